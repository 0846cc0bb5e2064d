// events.cu -- phase A of a search step: the data event of every item and its
// level-J Haar approximation (Algorithm 1, lines 8-9).
//
// One CTA per item. The known cells of the template window are (hard datum
// if present, else the simulated value); their facies counts per s^d block
// are the scaled-Haar approximation of the facies indicator images of the
// overlap region. The one-hot score of a candidate with TI counts a_f is
//   sum_u sum_f a_f(x+u) b_f(u)
//     = sum_u sum_{f<F-1} a_f(x+u) (b_f(u) - b_{F-1}(u)) + s^d sum_u b_{F-1}(u)
// because the TI counts of a block sum to s^d; the kernel stores the F-1
// weights w_f = b_f - b_{F-1} and the constant. The literal score stores the
// block sums of the known codes. An empty data event is finished here: a
// uniform draw (Algorithm 1, lines 5-6) and, when simulating, the paste.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "device_util.cuh"

namespace ccw {

constexpr int kCntInts = 12;   // shared counters ahead of the block counts

template <int D, int MODE>
__global__ void __launch_bounds__(kThreads) k_events(const __grid_constant__ WaveArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const TiDev& t = a.ti;
  const int tid = threadIdx.x;
  const int nth = blockDim.x;   // a multiple of 32, at most kThreads
  const int item = blockIdx.x;
  const int T = t.T, Tj = t.Tj, s = t.s, rows = t.rows, TjP = t.TjP;
  float* Ws = reinterpret_cast<float*>(smem);
  int* cnt = reinterpret_cast<int*>(smem + t.nch * rows * TjP * 4);
  // cnt: 0 known, 1 const, 2 mask cells, 3 hd count, 4 bad, 8..11 overlap
  // strip k holds an incomplete block
  int* counts = cnt + kCntInts;   // [F][Tj^d] facies counts of the level-J blocks
  unsigned char* rec = a.ev.base + (int64_t)item * a.ev.stride;
  int* meta = reinterpret_cast<int*>(rec);
  uint32_t* rowmask = reinterpret_cast<uint32_t*>(rec + a.ev.mask_off);
  int2* hdl = reinterpret_cast<int2*>(rec + a.ev.hd_off);
  float* wout = reinterpret_cast<float*>(rec + a.ev.w_off);

  ItemPos it;
  const uint8_t* sg = nullptr;
  const uint8_t* de = nullptr;
  const uint8_t* hdw = nullptr;
  if (MODE == kModeSim) {
    it = decode_sim_item<D>(a, item);
    sg = it.sg;
  } else {
    const int64_t tv = (D == 3) ? (int64_t)T * T * T : (int64_t)T * T;
    de = a.de + (int64_t)item * tv;
    hdw = a.hd ? a.hd + (int64_t)item * tv : nullptr;
    if (MODE == kModeSearch) {
      it.r = a.ctr[2 * item];
      it.p = a.ctr[2 * item + 1];
    }
  }

  const int ncells = (D == 3) ? Tj * Tj * Tj : Tj * Tj;
  for (int i = tid; i < t.nch * rows * TjP; i += nth) Ws[i] = 0.f;
  if (tid < kCntInts) cnt[tid] = 0;
  pdl_trigger();
  pdl_wait();   // the previous step's pastes and reads of the records are done
  __syncthreads();
  // One thread per level-J block: it gathers the block's s^d cells (grid
  // value, or the hard datum where there is one), counts the facies in
  // registers, and writes the block's weights (Eq. CCW operand). Facies
  // counts sit in 16-bit lanes: facies 0-3 in `lo`, 4-7 in `hi`.
  int my_known = 0, my_const = 0, my_mask = 0, bad = 0;
  const int Oj = a.Oj;
  // 4-cell rows of a block are one aligned 32-bit word of the grid when the
  // window origin and the grid pitch are multiples of 4
  const bool words = MODE == kModeSim && s == 4 && ((it.o[0] | it.Gp[0]) & 3) == 0;
  for (int u = tid; u < ncells; u += nth) {
    const int ux = u % Tj, uy = (u / Tj) % Tj, uz = (D == 3) ? u / (Tj * Tj) : 0;
    uint64_t lo = 0, hi = 0;
    int cf[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // facies counts (word path)
    if (words) {
      // a block row is one 32-bit word of 4 codes: count each facies with
      // byte-wise compares (SWAR); hard data replace their bytes first
      for (int cz = 0; cz < ((D == 3) ? 4 : 1); ++cz)
#pragma unroll
        for (int cy = 0; cy < 4; ++cy) {
          const int qy = uy * 4 + cy, qz = uz * 4 + cz;
          const int gx0 = it.o[0] + ux * 4, gy = it.o[1] + qy, gz = it.o[2] + qz;
          uint32_t vw = *reinterpret_cast<const uint32_t*>(
              sg + gx0 + (int64_t)it.Gp[0] * (gy + (int64_t)it.Gp[1] * gz));
          if (it.overlay) {   // the group has hard data
            const int hy = gy - it.off[1], hz = gz - it.off[2];
            uint32_t hw = 0xFFFFFFFFu;
            if (hy >= 0 && hz >= 0 && hy < it.G[1] && hz < it.G[2]) {
              const uint8_t* orow = it.overlay + (int64_t)it.G[0] * (hy + (int64_t)it.G[1] * hz);
#pragma unroll
              for (int cx = 0; cx < 4; ++cx) {
                const int hx = gx0 + cx - it.off[0];
                const uint32_t h = (hx >= 0 && hx < it.G[0]) ? __ldg(orow + hx) : 0xFFu;
                hw = (hw & ~(0xFFu << (8 * cx))) | (h << (8 * cx));
              }
            }
            if (hw != 0xFFFFFFFFu) {
#pragma unroll
              for (int cx = 0; cx < 4; ++cx) {
                const uint32_t h = (hw >> (8 * cx)) & 0xFFu;
                if (h == CCW_UNKNOWN) continue;
                const int qx = ux * 4 + cx;
                const int k = atomicAdd(&cnt[3], 1);
                if (k < a.ev.hd_cap)
                  hdl[k] = make_int2(qx + t.tp[0] * (qy + t.tp[1] * qz),
                                     ((qx + T * (qy + T * qz)) << 8) | (int)h);
                if (h >= (uint32_t)t.F) bad |= kStatusBadCode;
              }
              const uint32_t keep = __vcmpeq4(hw, 0xFFFFFFFFu);   // 0xFF: no hard datum
              vw = (vw & keep) | (hw & ~keep);
            }
          }
          int seen = __popc(__vcmpeq4(vw, 0xFFFFFFFFu)) >> 3;   // unknown cells
#pragma unroll
          for (int f = 0; f < 8; ++f) {
            if (f >= t.F) break;
            const int n = __popc(__vcmpeq4(vw, 0x01010101u * (uint32_t)f)) >> 3;
            cf[f] += n;
            seen += n;
          }
          if (seen != 4) bad |= kStatusBadCode;   // a code >= F
        }
    } else
    for (int cz = 0; cz < ((D == 3) ? s : 1); ++cz)
      for (int cy = 0; cy < s; ++cy) {
        const int qy = uy * s + cy, qz = uz * s + cz;
#pragma unroll 4
        for (int cx = 0; cx < s; ++cx) {
          const int qx = ux * s + cx;
          uint8_t v, h = CCW_UNKNOWN;
          if (MODE == kModeSim) {
            const int gx = it.o[0] + qx, gy = it.o[1] + qy, gz = it.o[2] + qz;
            if (it.overlay) {   // the group has hard data
              const int hx = gx - it.off[0], hy = gy - it.off[1], hz = gz - it.off[2];
              if (hx >= 0 && hy >= 0 && hz >= 0 && hx < it.G[0] && hy < it.G[1] && hz < it.G[2])
                h = __ldg(it.overlay + hx + (int64_t)it.G[0] * (hy + (int64_t)it.G[1] * hz));
            }
            v = sg[gx + (int64_t)it.Gp[0] * (gy + (int64_t)it.Gp[1] * gz)];
            if (h != CCW_UNKNOWN) v = h;
          } else {
            const int q = qx + T * (qy + T * qz);
            v = __ldg(de + q);
            if (hdw) h = __ldg(hdw + q);
          }
          if (h != CCW_UNKNOWN) {
            const int k = atomicAdd(&cnt[3], 1);
            if (k < a.ev.hd_cap)
              hdl[k] = make_int2(qx + t.tp[0] * (qy + t.tp[1] * qz),
                                 ((qx + T * (qy + T * qz)) << 8) | (int)h);
            if (h >= t.F) bad |= kStatusBadCode;
          }
          if (v != CCW_UNKNOWN) {
            if (v >= t.F) {
              bad |= kStatusBadCode;
            } else {
              const uint64_t one = 1ull << (16 * (v & 3));
              if (v < 4) lo += one;
              else hi += one;
            }
          }
        }
      }
    int c = 0, csum = 0;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      if (f >= t.F) break;
      const int b = words ? cf[f] : (int)(((f < 4 ? lo : hi) >> (16 * (f & 3))) & 0xFFFF);
      counts[f * ncells + u] = b;
      c += b;
      csum += f * b;
    }
    if (D == 2 && a.learned && c != t.sd) {
      // this block keeps every overlap strip it lies in from being full
      if (ux < Oj) cnt[8] = 1;
      if (ux >= Tj - Oj) cnt[9] = 1;
      if (uy < Oj) cnt[10] = 1;
      if (uy >= Tj - Oj) cnt[11] = 1;
    }
    if (!c) continue;
    my_known += c;
    ++my_mask;
    const int row = u / Tj;
    if (t.score_mode == 0) {
      const int blast = counts[(t.F - 1) * ncells + u];
      for (int f = 0; f < t.F - 1; ++f)
        Ws[(f * rows + row) * TjP + ux] = (float)(counts[f * ncells + u] - blast);
      my_const += t.sd * blast;
    } else {
      Ws[row * TjP + ux] = (float)csum;
    }
  }
  if (MODE == kModeSim && a.vt_ext > 0 && it.overlay) {
    // non-causal conditioning (Sec. 4.4): the hard data of the virtual
    // template, the window grown by vt_ext cells along the forward direction
    // of the path, outside the window. Path-frame offsets v are mirrored
    // along the axes the path runs backwards; the data only join the
    // mismatch count (record flag kHdVirtual: never pasted).
    const int E = a.vt_ext, W = T + E;
    // the cells of the grown window outside the window, in path frame:
    // 2D: rows vy >= T (every vx), then vx >= T of rows vy < T;
    // 3D: planes vz >= T, then rows vy >= T of planes vz < T, then vx >= T
    const int nA = (D == 3) ? W * W * E : W * E;
    const int nB = (D == 3) ? T * E * W : T * E;
    const int nC = (D == 3) ? T * T * E : 0;
    const int nv = nA + nB + nC;
    constexpr int kB = 4;   // cells per thread whose overlay loads are in flight together
    for (int v0 = tid; v0 < nv; v0 += kB * nth) {
      int h[kB], off[kB];
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        h[b] = CCW_UNKNOWN;
        off[b] = 0;
        const int v = v0 + b * nth;
        if (v >= nv) continue;
        int vx, vy, vz = 0;
        if (D == 2) {
          if (v < nA) {
            vy = T + v / W;
            vx = v % W;
          } else {
            vy = (v - nA) / E;
            vx = T + (v - nA) % E;
          }
        } else if (v < nA) {
          vz = T + v / (W * W);
          vy = (v / W) % W;
          vx = v % W;
        } else if (v < nA + nB) {
          const int r = v - nA;
          vz = r / (E * W);
          vy = T + (r / W) % E;
          vx = r % W;
        } else {
          const int r = v - nA - nB;
          vz = r / (T * E);
          vy = (r / E) % T;
          vx = T + r % E;
        }
        const int qx = (it.flips & 1u) ? T - 1 - vx : vx;
        const int qy = (it.flips & 2u) ? T - 1 - vy : vy;
        const int qz = (D == 3 && (it.flips & 4u)) ? T - 1 - vz : vz;
        const int hx = it.o[0] + qx - it.off[0], hy = it.o[1] + qy - it.off[1],
                  hz = it.o[2] + qz - it.off[2];
        if (hx < 0 || hy < 0 || hz < 0 || hx >= it.G[0] || hy >= it.G[1] || hz >= it.G[2])
          continue;
        h[b] = __ldg(it.overlay + hx + (int64_t)it.G[0] * (hy + (int64_t)it.G[1] * hz));
        off[b] = qx + t.tp[0] * (qy + t.tp[1] * qz);
      }
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        if (h[b] == CCW_UNKNOWN) continue;
        const int k = atomicAdd(&cnt[3], 1);
        if (k < a.ev.hd_cap) hdl[k] = make_int2(off[b], kHdVirtual | h[b]);
        if (h[b] >= t.F) bad |= kStatusBadCode;
      }
    }
  }
  my_known = __reduce_add_sync(0xffffffffu, my_known);
  my_const = __reduce_add_sync(0xffffffffu, my_const);
  my_mask = __reduce_add_sync(0xffffffffu, my_mask);
  bad = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
  if ((tid & 31) == 0) {
    if (my_known) atomicAdd(&cnt[0], my_known);
    if (my_const) atomicAdd(&cnt[1], my_const);
    if (my_mask) atomicAdd(&cnt[2], my_mask);
    if (bad) atomicOr(&cnt[4], bad);
  }
  __syncthreads();
  if (MODE == kModeSim && it.counts)
    for (int i = tid; i < t.F * ncells; i += nth) it.counts[i] = (uint8_t)counts[i];
  if (a.learned) {
    uint8_t* rc = rec + a.ev.counts_off;
    for (int i = tid; i < t.F * ncells; i += nth) rc[i] = (uint8_t)min(counts[i], 255);
  }
  // chunk masks of the template rows and the weights, to the record
  for (int row = tid; row < rows; row += nth) {
    uint32_t m = 0;
    for (int ch = 0; ch < t.nch; ++ch) {
      const float* wr = Ws + (ch * rows + row) * TjP;
      for (int ux = 0; ux < Tj; ++ux)
        if (wr[ux] != 0.f) m |= 1u << (ux >> 2);
    }
    rowmask[row] = m;
  }
  {
    const float4* src = reinterpret_cast<const float4*>(Ws);
    float4* dst = reinterpret_cast<float4*>(wout);
    for (int i = tid; i < t.nch * rows * TjP / 4; i += nth) dst[i] = src[i];
  }
  if (a.bmat) {
    // the weights as the B operand of the tensor-core CCF: item n is row
    // n % nt of N-tile n / nt; K step k = (ch * rows + row) * ks/16 + k16
    // holds taps 16 k16 .. 16 k16 + 15 of that template row, as two 8 x 8
    // core matrices (kc = 0, 1) in the canonical K-major layout
    const int nt = a.nt, k16n = a.ks / 16;
    const int ntile = item / nt, ni = item % nt;
    unsigned char* base = reinterpret_cast<unsigned char*>(a.bmat) +
                          (int64_t)ntile * a.ksteps * 32 * nt + (ni / 8) * 256 + (ni % 8) * 16;
    for (int i = tid; i < a.ksteps * 2; i += nth) {
      const int k = i >> 1, kc = i & 1;
      const int k16 = k % k16n, rc = k / k16n;
      const float* wr = Ws + rc * TjP;
      uint32_t packed[4];
#pragma unroll
      for (int e2 = 0; e2 < 4; ++e2) {
        const int kx0 = 16 * k16 + 8 * kc + 2 * e2;
        const float w0 = kx0 < Tj ? wr[kx0] : 0.f;
        const float w1 = kx0 + 1 < Tj ? wr[kx0 + 1] : 0.f;
        uint16_t h0, h1;
        if (a.precision == 2) {
          h0 = __bfloat16_as_ushort(__float2bfloat16_rn(w0));
          h1 = __bfloat16_as_ushort(__float2bfloat16_rn(w1));
        } else {
          h0 = __half_as_ushort(__float2half_rn(w0));
          h1 = __half_as_ushort(__float2half_rn(w1));
        }
        packed[e2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
      }
      *reinterpret_cast<uint4*>(base + (int64_t)k * 32 * nt + kc * 128) =
          make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
  }
  const int known = cnt[0];
  if (tid == 0) {
    meta[kEvKnown] = known;
    meta[kEvConst] = cnt[1];
    meta[kEvMaskCells] = cnt[2];
    meta[kEvNHd] = min(cnt[3], a.ev.hd_cap);
    // overlap strips fully known (2D, learned proposal): bit k unless a
    // block of strip k was incomplete
    meta[kEvMaskType] = (D == 2 && a.learned && Oj > 0)
                            ? ((cnt[8] ? 0 : 1) | (cnt[9] ? 0 : 2) | (cnt[10] ? 0 : 4) |
                               (cnt[11] ? 0 : 8))
                            : 0;
    meta[kEvResolved] = 0;
    const int bad = cnt[4] | (cnt[3] > a.ev.hd_cap ? kStatusHdOverflow : 0);
    if (bad) atomicOr(a.status, bad);
  }
  if (known != 0 || MODE == kModeMap) return;

  // empty data event: uniform draw (Algorithm 1, lines 5-6)
  const uint64_t seed = (MODE == kModeSim) ? a.call->seed : a.seed;
  const uint32_t u = draw_word(seed, it.r, it.p, 0u);
  const int pk = (int)mul_shift(u, t.P);
  if (MODE == kModeSearch) {
    if (tid < a.K) {
      a.topk_idx[item * a.K + tid] = -1;
      a.topk_score[item * a.K + tid] = 0;
      a.topk_mis[item * a.K + tid] = 0;
    }
    if (tid == 0) a.pick[item] = pk;
    return;
  }
  const CallDev* c = a.call;
  if (it.log && tid < c->log_stride) {
    int32_t* e = it.log;
    e[tid] = (tid == 0) ? pk
                        : (tid == 3 ? (CCW_LOG_FLAG_UNIFORM | CCW_LOG_FLAG_DONE)
                                    : (tid < 3 ? 0 : -1));
  }
  const PasteGeom g = sim_paste_geom<D>(a, it);
  if (D == 2 && a.allshift)
    paste_crop2(g, t.ti, t.tp[0], a.fd0, pk, T, nth, tid);
  else
    paste_pixels<D>(g, pk, t.J, nth, tid);
  __syncthreads();
  paste_hard_data<D>(g, hdl, min(cnt[3], a.ev.hd_cap), T, nth, tid);
}

// Standalone Inverse-DWT paste (ccw_idwt_paste): one CTA per batch element.
template <int D>
__global__ void __launch_bounds__(kThreads)
    k_idwt_paste(const int16_t* pyr, int nc0, int nc1, int cd0, int cd1, int Tj, int J, int64_t P,
                 const int32_t* picks, const int32_t* origins, uint8_t* grid, int gx, int gy,
                 int gz, int* status) {
  const int b = blockIdx.x;
  const int pk = picks[b];
  if (pk < 0 || pk >= P) {
    if (threadIdx.x == 0) atomicOr(status, kStatusBadCode);
    return;
  }
  PasteGeom g;
  g.pyr = pyr;
  g.nc0 = nc0;
  g.nc1 = nc1;
  g.cd0 = cd0;
  g.cd1 = cd1;
  g.Tj = Tj;
  g.grid = grid;
  g.g[0] = gx;
  g.g[1] = gy;
  g.g[2] = gz;
  g.o[0] = origins[3 * b];
  g.o[1] = origins[3 * b + 1];
  g.o[2] = (D == 3) ? origins[3 * b + 2] : 0;
  paste_pixels<D>(g, pk, J, kThreads, threadIdx.x);
}

cudaError_t launch_idwt_paste(int d, int J, const int16_t* pyr, const int nc[3], const int cd[3],
                              int Tj, int64_t P, int B, const int32_t* picks,
                              const int32_t* origins, uint8_t* grid, const int gdim[3],
                              int* status, cudaStream_t st) {
  if (d == 2)
    k_idwt_paste<2><<<B, kThreads, 0, st>>>(pyr, nc[0], nc[1], cd[0], cd[1], Tj, J, P, picks,
                                            origins, grid, gdim[0], gdim[1], gdim[2], status);
  else
    k_idwt_paste<3><<<B, kThreads, 0, st>>>(pyr, nc[0], nc[1], cd[0], cd[1], Tj, J, P, picks,
                                            origins, grid, gdim[0], gdim[1], gdim[2], status);
  return cudaGetLastError();
}

int events_smem_bytes(int nch, int rows, int TjP, int F, int ncells) {
  return nch * rows * TjP * 4 + kCntInts * 4 + F * ncells * 4;   // cnt, then the counts
}

template <int D, int MODE>
static cudaError_t launch_events_t(const WaveArgs& a, bool pdl, cudaStream_t st) {
  const int ncells = a.ti.rows * a.ti.Tj;
  const int smem = events_smem_bytes(a.ti.nch, a.ti.rows, a.ti.TjP, a.ti.F, ncells);
  auto fn = k_events<D, MODE>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  // one thread per level-J block up to kThreads (fewer threads per CTA let
  // more CTAs share an SM when the template has few blocks)
  const int nth = std::min(kThreads, std::max(96, (ncells + 31) / 32 * 32));   // >= 4 + K log words
  return launch_pdl(fn, dim3(a.n_items), dim3(nth), smem, st, pdl, a);
}

cudaError_t launch_events(int mode, const WaveArgs& a, bool pdl, cudaStream_t st) {
  if (a.ti.d == 2) {
    if (mode == kModeSim) return launch_events_t<2, kModeSim>(a, pdl, st);
    if (mode == kModeSearch) return launch_events_t<2, kModeSearch>(a, pdl, st);
    return launch_events_t<2, kModeMap>(a, pdl, st);
  }
  if (mode == kModeSim) return launch_events_t<3, kModeSim>(a, pdl, st);
  if (mode == kModeSearch) return launch_events_t<3, kModeSearch>(a, pdl, st);
  return launch_events_t<3, kModeMap>(a, pdl, st);
}

}  // namespace ccw
