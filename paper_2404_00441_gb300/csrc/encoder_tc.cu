// encoder_tc.cu -- inference pass of the proposal encoder on the tcgen05
// tensor cores (BF16 operands, FP32 accumulation in tensor memory). The
// network and its arithmetic are those of learned.cu (weights and stored
// activations rounded to BF16, FP32 sums); only the order of the sums differs.
//
// Each CTA embeds its samples G at a time. Every convolution is an implicit
// GEMM whose M rows are output positions (sample, y, x) on a grid padded by
// one cell, N = 32 output channels and K = taps x input channels:
//
//  * an activation lives in shared memory as "phase planes": for a stride-2
//    consumer, the four (y mod 2, x mod 2) sub-grids of the map, each padded
//    with a leading zero row and column, one 16-byte row (8 channels) per
//    position and one plane per 8-channel chunk;
//  * the rows a tap (ky, kx) needs for consecutive output positions are then
//    consecutive rows of one plane at a constant row shift, so the MMA's A
//    operand is the plane itself at a shifted start address (K-major, no
//    swizzle, core matrices of 8 consecutive rows: SBO = 128 bytes, LBO =
//    the distance to the next chunk's plane). No im2col copy is made;
//  * the first layer (stride 1, C <= 8 input channels in one chunk) pairs
//    taps in one K = 16 step: the second chunk is the same plane at the next
//    tap's shift (LBO = shift difference x 16 bytes).
//
// The epilogue of each layer reads the accumulators with tcgen05.ld, adds the
// bias, applies ReLU, rounds to BF16 and scatters the rows into the next
// layer's phase planes; the last convolution writes the linear layer's A rows
// (one per sample); the linear layer's epilogue normalises the embedding.
#include <cuda_bf16.h>

#include <algorithm>

#include "ccw_internal.cuh"
#include "net_shape.cuh"
#include "tc_util.cuh"

namespace ccw {

// Geometry of one encoder shape (host-computed, passed by value).
struct EncTc {
  int C, tj, h2, h3, flat;
  int G;                 // samples per group (<= 8)
  int W1, R1, T1;        // layer 1: padded grid width tj + 2, rows per sample, M-tiles
  int W2, R2, T2;        // layer 2: h2 + 1, rows per sample, M-tiles (= a1 plane geometry)
  int W3, R3, T3;        // layer 3: h3 + 1, rows per sample, M-tiles (= a2 plane geometry)
  int P1, P2;            // rows per phase-chunk plane of a1 / a2
  int o_w1, o_w2, o_w3, o_wf, o_bias, o_a4, o_x, o_a1, o_a2, o_bar, smem;
  int x_guard;           // rows before the first row of the input plane
  uint32_t tmem_cols;
};

constexpr int kEncThreads = 256;
constexpr int kEncMaxG = 8;

// Byte offset of element (n, k) in a K-major B operand block of 16 K values
// and N rows: [N / 8][2 K-chunks][8 rows][8 values].
__device__ __forceinline__ int b_off(int n, int k) {
  return (n >> 3) * 256 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint16_t to_bf16_bits(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Row shift of tap (ky, kx) in a stride-2 layer's phase planes of width W,
// and the plane phase (py * 2 + px) it reads.
__device__ __forceinline__ int s2_shift(int ky, int kx, int W) {
  return (ky == 0 ? -W : 0) + (kx == 0 ? -1 : 0);
}
__device__ __forceinline__ int s2_phase(int ky, int kx) {
  return (ky == 1 ? 0 : 2) + (kx == 1 ? 0 : 1);
}

// Stages the BF16 weights in the B-operand layouts and the FP32 biases.
__device__ void enc_stage_weights(const float* __restrict__ P, const NetShape& s, const EncTc& g,
                                  unsigned char* sm) {
  const int tid = threadIdx.x;
  // layer 1: 5 tap pairs; K rows 0..7 = tap 2p, 8..15 = tap 2p + 1 (channel ci < C)
  for (int i = tid; i < 5 * 32 * 16; i += kEncThreads) {
    const int p = i / 512, co = (i / 16) % 32, k = i % 16;
    const int tap = 2 * p + (k >> 3), ci = k & 7;
    float v = 0.f;
    if (tap < 9 && ci < s.C) v = __ldg(P + s.o_w1 + (co * s.C + ci) * 9 + tap);
    *reinterpret_cast<uint16_t*>(sm + g.o_w1 + p * 1024 + b_off(co, k)) = to_bf16_bits(v);
  }
  // layers 2 and 3: (tap, 16-channel step q) blocks
  for (int l = 0; l < 2; ++l) {
    const float* w = P + (l == 0 ? s.o_w2 : s.o_w3);
    const int base = l == 0 ? g.o_w2 : g.o_w3;
    for (int i = tid; i < 32 * 32 * 9; i += kEncThreads) {
      // master order [co][ci][tap]: consecutive threads read consecutive words
      const int co = i / 288, ci = (i / 9) % 32, tap = i % 9;
      const int q = ci >> 4, k = ci & 15;
      *reinterpret_cast<uint16_t*>(sm + base + (tap * 2 + q) * 1024 + b_off(co, k)) =
          to_bf16_bits(__ldg(w + i));
    }
  }
  // linear: K index k = pos * 32 + co (pos = oy * h3 + ox), master [j][co][pos]
  const int hh = s.h3 * s.h3;
  for (int i = tid; i < 64 * s.flat; i += kEncThreads) {
    const int j = i / s.flat, r = i % s.flat;
    const int co = r / hh, pos = r % hh;
    const int k = pos * 32 + co;
    *reinterpret_cast<uint16_t*>(sm + g.o_wf + (k >> 4) * 2048 + b_off(j, k & 15)) =
        to_bf16_bits(__ldg(P + s.o_wf + i));
  }
  float* bias = reinterpret_cast<float*>(sm + g.o_bias);
  for (int i = tid; i < 160; i += kEncThreads) {
    float v;
    if (i < 32) v = __ldg(P + s.o_b1 + i);
    else if (i < 64) v = __ldg(P + s.o_b2 + i - 32);
    else if (i < 96) v = __ldg(P + s.o_b3 + i - 64);
    else v = __ldg(P + s.o_bf + i - 96);
    bias[i] = v;
  }
}

// 32 accumulator columns (one M-tile of a convolution) of this thread's lane:
// bias, ReLU, BF16, packed as four 16-byte rows of 8 channels.
__device__ __forceinline__ void enc_conv_row(uint32_t taddr, const float* bias, uint4 (&out)[4]) {
  uint32_t v[32];
  tmem_ld32(taddr, v);
  uint32_t w[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    float a0 = __uint_as_float(v[2 * c]) + bias[2 * c];
    float a1 = __uint_as_float(v[2 * c + 1]) + bias[2 * c + 1];
    a0 = a0 < 0.f ? 0.f : a0;
    a1 = a1 < 0.f ? 0.f : a1;
    w[c] = (uint32_t)to_bf16_bits(a0) | ((uint32_t)to_bf16_bits(a1) << 16);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

// The inference pass over samples x[N][C][tj][tj] -> unit embeddings
// emb[N][64], G samples per group, groups taken in turn by the CTAs.
// The weights' shared-memory image (offsets 0 .. o_a4 of the layout) built
// once in global memory, so that each CTA takes it with one bulk copy.
__global__ void k_enc_weight_image(const float* __restrict__ P, NetShape s, EncTc g,
                                   unsigned char* img) {
  enc_stage_weights(P, s, g, img);
}

// Where the samples come from: floats x[N][C][tj][tj], or the block counts
// of event records (rec + i * stride + counts_off, uint8 [C][tj][tj]) divided
// by 2^(d J) (zero for an empty event, which is never searched).
struct EncSrc {
  const float* x;
  const unsigned char* rec;
  int64_t stride;
  int counts_off;
  float inv;
};

__global__ void __launch_bounds__(kEncThreads, 1)
    k_encode_tc(const unsigned char* __restrict__ wimg, NetShape s, EncTc g, EncSrc src, int N,
                float* __restrict__ emb, int* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + g.o_bar);
  uint64_t* wbar = reinterpret_cast<uint64_t*>(sm + g.o_bar + 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + g.o_bar + 8);
  volatile int* flag = reinterpret_cast<volatile int*>(sm + g.o_bar + 12);
  pdl_trigger();
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(wbar, 1);
    *flag = 0;
    fence_mbar_init();
    // the weights and biases: one bulk copy of their image
    mbar_arrive_expect_tx(wbar, (uint32_t)g.o_a4);
    bulk_g2s(sm, wimg, (uint32_t)g.o_a4, wbar);
  }
  // every plane starts zero: the padding rows and columns are never written
  for (int i = g.o_a4 / 16 + tid; i < g.o_bar / 16; i += kEncThreads)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  // the predecessor's records are complete from here on, and every earlier
  // kernel has released its tensor memory (allocating before this wait could
  // block a predecessor's allocation on the same SM while this CTA waits)
  pdl_wait();
  if (warp == 0) tmem_alloc(tslot, g.tmem_cols);
  // one thread waits for the copy (the others wait at the barrier, not
  // polling beside it), then every thread observes the completed phase
  if (tid == 0 && !mbar_wait_bounded(wbar, 0u)) *flag = 1;
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  mbar_try_wait(wbar, 0u);
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const float* bias = reinterpret_cast<const float*>(sm + g.o_bias);
  const uint32_t sbase = smem_u32(sm);
  const int quarter = warp & 3, half = warp >> 2;
  const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
  const int tj = g.tj, tt = tj * tj;
  const int ngroups = (N + g.G - 1) / g.G;
  const uint32_t idesc32 = instr_desc(true, 128, 32), idesc64 = instr_desc(true, 128, 64);
  uint32_t phase = 0;

  // commit the MMAs issued by thread 0, wait (bounded) for them, and order
  // the accumulators and shared memory before what follows
  auto mma_done = [&]() -> bool {
    if (tid == 0) {
      mma_commit(bar);
      if (!mbar_wait_bounded(bar, phase)) *flag = 1;
    }
    __syncthreads();
    if (*flag) return false;
    mbar_try_wait(bar, phase);   // every thread observes the completed phase
    phase ^= 1u;
    tc_fence_after();
    return true;
  };
  // generic-proxy plane writes and accumulator reads before the next MMAs
  auto publish = [&]() {
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
  };

  for (int grp = blockIdx.x; grp < ngroups && !*flag; grp += gridDim.x) {
    const int n0 = grp * g.G, gr = min(g.G, N - n0);
    // ---- inputs -> interior rows of the layer-1 plane (8 channels a row)
#pragma unroll 4
    for (int i = tid; i < gr * tt; i += kEncThreads) {
      const int it = i / tt, r = i % tt, y = r / tj, xx = r % tj;
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      if (src.rec) {
        const unsigned char* rec = src.rec + (int64_t)(n0 + it) * src.stride;
        const bool known = reinterpret_cast<const int*>(rec)[kEvKnown] > 0;
        const unsigned char* cnt = rec + src.counts_off + r;
#pragma unroll
        for (int ci = 0; ci < 8; ++ci)
          if (ci < s.C && known)
            w[ci >> 1] |= (uint32_t)to_bf16_bits((float)cnt[ci * tt] * src.inv) << (16 * (ci & 1));
      } else {
        const float* xs = src.x + (int64_t)(n0 + it) * s.C * tt + r;
#pragma unroll
        for (int ci = 0; ci < 8; ++ci)
          if (ci < s.C) w[ci >> 1] |= (uint32_t)to_bf16_bits(__ldg(xs + ci * tt)) << (16 * (ci & 1));
      }
      const int row = g.x_guard + it * g.R1 + (y + 1) * g.W1 + xx + 1;
      *reinterpret_cast<uint4*>(sm + g.o_x + row * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    publish();

    // ---- layer 1: 5 tap pairs per M-tile
    if (tid == 0) {
      tc_fence_after();
      for (int j = 0; j < g.T1; ++j)
        for (int p = 0; p < 5; ++p) {
          const int ta = 2 * p;
          const int sa = (ta / 3 - 1) * g.W1 + (ta % 3 - 1);
          const int sb = p < 4 ? ((ta + 1) / 3 - 1) * g.W1 + ((ta + 1) % 3 - 1) : sa + 1;
          const uint32_t a_addr =
              sbase + (uint32_t)(g.o_x + (g.x_guard + 128 * j + sa) * 16);
          mma_f16(tmem + (uint32_t)(j * 32), smem_desc(a_addr, (uint32_t)(sb - sa) * 16u, 128u),
                  smem_desc(sbase + (uint32_t)(g.o_w1 + p * 1024), 128u, 256u), idesc32,
                  p > 0 ? 1u : 0u);
        }
    }
    if (!mma_done()) break;
    for (int j = half; j < g.T1; j += 2) {
      uint4 out[4];
      enc_conv_row(lane_base + (uint32_t)(j * 32), bias, out);
      const int m = 128 * j + quarter * 32 + lane;
      const int it = m / g.R1, r = m % g.R1, Y = r / g.W1, X = r % g.W1;
      if (it < gr && Y >= 1 && Y <= tj && X >= 1 && X <= tj) {
        const int y = Y - 1, xx = X - 1;
        const int ph = (y & 1) * 2 + (xx & 1);
        const int row = it * g.R2 + ((y >> 1) + 1) * g.W2 + (xx >> 1) + 1;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          *reinterpret_cast<uint4*>(sm + g.o_a1 + ((ph * 4 + c) * g.P1 + row) * 16) = out[c];
      }
    }
    publish();

    // ---- layers 2 and 3: 9 taps x 2 K steps per M-tile, A = shifted plane
    for (int l = 0; l < 2; ++l) {
      const int T = l == 0 ? g.T2 : g.T3, Pp = l == 0 ? g.P1 : g.P2;
      const int W = l == 0 ? g.W2 : g.W3;
      const int src = l == 0 ? g.o_a1 : g.o_a2, wgt = l == 0 ? g.o_w2 : g.o_w3;
      if (tid == 0) {
        tc_fence_after();
        for (int j = 0; j < T; ++j)
          for (int t = 0; t < 9; ++t) {
            const int ky = t / 3, kx = t % 3;
            const int ph = s2_phase(ky, kx), sh = s2_shift(ky, kx, W);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const uint32_t a_addr =
                  sbase + (uint32_t)(src + ((ph * 4 + 2 * q) * Pp + 128 * j + sh) * 16);
              mma_f16(tmem + (uint32_t)(j * 32), smem_desc(a_addr, (uint32_t)Pp * 16u, 128u),
                      smem_desc(sbase + (uint32_t)(wgt + (t * 2 + q) * 1024), 128u, 256u),
                      idesc32, (t | q) ? 1u : 0u);
            }
          }
      }
      if (!mma_done()) break;
      const int R = l == 0 ? g.R2 : g.R3;
      for (int j = half; j < T; j += 2) {
        uint4 out[4];
        enc_conv_row(lane_base + (uint32_t)(j * 32), bias + 32 * (l + 1), out);
        const int m = 128 * j + quarter * 32 + lane;
        const int it = m / R, r = m % R, Y = r / W, X = r % W;
        if (it < gr && Y >= 1 && X >= 1) {
          const int y = Y - 1, xx = X - 1;
          if (l == 0) {
            const int ph = (y & 1) * 2 + (xx & 1);
            const int row = it * g.R3 + ((y >> 1) + 1) * g.W3 + (xx >> 1) + 1;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              *reinterpret_cast<uint4*>(sm + g.o_a2 + ((ph * 4 + c) * g.P2 + row) * 16) = out[c];
          } else {
            // linear layer's A: row = sample, K = pos * 32 + channel
            const int pos = y * g.h3 + xx;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              *reinterpret_cast<uint4*>(sm + g.o_a4 + ((pos * 4 + c) * 8 + it) * 16) = out[c];
          }
        }
      }
      publish();
    }
    if (*flag) break;

    // ---- linear layer (M rows 0..G-1 real) and L2 normalisation
    if (tid == 0) {
      tc_fence_after();
      for (int k16 = 0; k16 < g.flat / 16; ++k16)
        mma_f16(tmem, smem_desc(sbase + (uint32_t)(g.o_a4 + k16 * 256), 128u, 128u),
                smem_desc(sbase + (uint32_t)(g.o_wf + k16 * 2048), 128u, 256u), idesc64,
                k16 > 0 ? 1u : 0u);
    }
    if (!mma_done()) break;
    if (warp == 0) {
      float z[64];
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + (uint32_t)c0, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) z[c0 + c] = __uint_as_float(v[c]) + bias[96 + c0 + c];
      }
      float q = 0.f;
#pragma unroll
      for (int c = 0; c < 64; ++c) q += z[c] * z[c];
      const float rn = 1.f / sqrtf(fmaxf(q, 1e-24f));
      if (lane < gr) {
        float4* dst = reinterpret_cast<float4*>(emb + (int64_t)(n0 + lane) * 64);
#pragma unroll
        for (int c = 0; c < 16; ++c)
          dst[c] = make_float4(z[4 * c] * rn, z[4 * c + 1] * rn, z[4 * c + 2] * rn,
                               z[4 * c + 3] * rn);
      }
    }
    tc_fence_before();
    __syncthreads();   // the next group reuses the planes and accumulators
  }
  if (*flag) {
    // a copy or commit never arrived: record it, give what is in flight one
    // more bounded wait, then free the tensor memory
    if (tid == 0) {
      if (status) atomicOr(status, kStatusTimeout);
      mbar_wait_bounded(wbar, 0u);
      mbar_wait_bounded(bar, phase);
    }
    __syncthreads();
  }
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, g.tmem_cols);
}

// Geometry and shared-memory layout for encoder shape (C, tj); false when
// the shape does not fit (then the FP32-lane kernels run).
static bool enc_tc_plan(int C, int tj, EncTc* out) {
  if (C < 1 || C > 8 || tj < 2) return false;
  const NetShape s = net_shape(C, tj);
  auto r8 = [](int v) { return (v + 7) & ~7; };
  for (int G = kEncMaxG; G >= 1; --G) {
    EncTc g{};
    g.C = C;
    g.tj = tj;
    g.h2 = s.h2;
    g.h3 = s.h3;
    g.flat = s.flat;
    g.G = G;
    g.W1 = tj + 2;
    g.R1 = g.W1 * g.W1;
    g.T1 = (G * g.R1 + 127) / 128;
    g.W2 = s.h2 + 1;
    g.R2 = g.W2 * g.W2;
    g.T2 = (G * g.R2 + 127) / 128;
    g.W3 = s.h3 + 1;
    g.R3 = g.W3 * g.W3;
    g.T3 = (G * g.R3 + 127) / 128;
    g.P1 = r8(G * g.R2);
    g.P2 = r8(G * g.R3);
    int o = 0;
    g.o_w1 = o;
    o += 5 * 1024;
    g.o_w2 = o;
    o += 18 * 1024;
    g.o_w3 = o;
    o += 18 * 1024;
    g.o_wf = o;
    o += (s.flat / 16) * 2048;
    g.o_bias = o;
    o += 160 * 4;
    g.o_a4 = o;
    o += s.flat * 16;                       // [flat / 8 chunks][8 rows of 16 bytes]
    g.x_guard = r8(g.W1 + 1);
    g.o_x = o;
    o += r8(g.x_guard + 128 * g.T1 + g.W1 + 2) * 16;
    g.o_a1 = o;
    o += (16 * g.P1 + std::max(0, 128 * g.T2 - g.P1)) * 16;
    g.o_a2 = o;
    o += (16 * g.P2 + std::max(0, 128 * g.T3 - g.P2)) * 16;
    g.o_bar = o;
    o += 32;   // MMA barrier, TMEM slot, flag, weight-copy barrier
    g.smem = o;
    int cols = std::max(std::max(g.T1, g.T2), g.T3) * 32;
    cols = std::max(cols, 64);
    uint32_t tc = 32;
    while ((int)tc < cols) tc <<= 1;
    g.tmem_cols = tc;
    if (tc > 512) continue;
    // the linear layer's A: row group i of K chunk c at (i + c) x 128 bytes,
    // so row group 0 holds the samples and groups 1..15 (rows that are not
    // samples) read at most 15 x 128 bytes past the block
    if (g.o_a4 + s.flat * 16 + 15 * 128 > g.o_bar) continue;
    // one CTA per SM when it takes more than half of the tensor memory
    if (tc > 256 && g.smem < 120 * 1024) g.smem = 120 * 1024;
    if (g.smem > 227 * 1024) continue;
    *out = g;
    return true;
  }
  return false;
}

// Bytes of the weight image of encoder shape (C, tj), 0 when the tensor-core
// pass does not take the shape.
int64_t enc_tc_image_bytes(int C, int tj) {
  EncTc g;
  return enc_tc_plan(C, tj, &g) ? g.o_a4 : 0;
}

// Writes the weight image of parameters P into img (enc_tc_image_bytes).
cudaError_t enc_tc_build_image(const float* P, int C, int tj, void* img, cudaStream_t st) {
  EncTc g;
  if (!enc_tc_plan(C, tj, &g)) return cudaErrorNotSupported;
  k_enc_weight_image<<<1, kEncThreads, 0, st>>>(P, net_shape(C, tj), g, (unsigned char*)img);
  return cudaGetLastError();
}

// Launches the tensor-core inference pass with the weight image wimg (built
// here into temporary memory when NULL); returns cudaErrorNotSupported
// (nothing launched) when the shape does not fit.
static cudaError_t encode_tc(const float* P, const void* wimg, int C, int tj, EncSrc src, int N,
                             float* emb, int* status, cudaStream_t st, bool pdl = false) {
  EncTc g;
  if (!enc_tc_plan(C, tj, &g)) return cudaErrorNotSupported;
  if (N <= 0) return cudaSuccess;
  static int configured = 0;
  if (g.smem > configured) {
    cudaError_t e =
        cudaFuncSetAttribute(k_encode_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
    if (e != cudaSuccess) return e;
    configured = g.smem;
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  void* tmp = nullptr;
  if (!wimg) {
    cudaError_t e = cudaMallocAsync(&tmp, (size_t)g.o_a4, st);
    if (e != cudaSuccess) return e;
    if ((e = enc_tc_build_image(P, C, tj, tmp, st)) != cudaSuccess) {
      cudaFreeAsync(tmp, st);
      return e;
    }
    wimg = tmp;
  }
  const int ngroups = (N + g.G - 1) / g.G;
  const int grid = ngroups < sms ? ngroups : sms;
  const cudaError_t e =
      launch_pdl(k_encode_tc, dim3(grid), dim3(kEncThreads), g.smem, st, pdl && !tmp,
                 (const unsigned char*)wimg, net_shape(C, tj), g, src, N, emb, status);
  if (tmp) cudaFreeAsync(tmp, st);
  return e;
}

cudaError_t net_infer_tc(const float* P, const void* wimg, int C, int tj, const float* x, int N,
                         float* emb, int* status, cudaStream_t st) {
  EncSrc src{};
  src.x = x;
  return encode_tc(P, wimg, C, tj, src, N, emb, status, st);
}

// The same pass on the block counts of event records (no separate input
// kernel): sample i = record rec + i * stride.
// With `pdl` the kernel is launched with programmatic stream serialization:
// its set-up overlaps the predecessor (the event kernel of the same step).
cudaError_t net_infer_tc_records(const float* P, const void* wimg, int C, int tj,
                                 const unsigned char* rec, int64_t stride, int counts_off,
                                 float inv, int N, float* emb, int* status, cudaStream_t st,
                                 bool pdl) {
  EncSrc src{};
  src.rec = rec;
  src.stride = stride;
  src.counts_off = counts_off;
  src.inv = inv;
  return encode_tc(P, wimg, C, tj, src, N, emb, status, st, pdl);
}

}  // namespace ccw
