// proposal.cu -- inference of the learned proposal (not part of the paper):
// embed each data event with the encoder, propose the n_prop TI candidates
// whose embedding (under the same overlap mask type) is nearest, re-rank the
// proposals with the exact masked CCF of Eq. CCW and the hard-data
// mismatches, and settle the item when the proposals' embedding scores are
// well separated; otherwise the item falls back to the full search.
#include <algorithm>

#include "device_util.cuh"
#include "tc_util.cuh"

namespace ccw {

// learned.cu
cudaError_t net_infer(const float* P, int C, int tj, const float* x, int N, float* act,
                      float* emb, cudaStream_t st, int* status = nullptr, int path = 0,
                      const void* wimg = nullptr);

// Is level-J cell (ux, uy) inside the overlap strips of mask type `type`?
__device__ __forceinline__ bool in_mask(int type, int ux, int uy, int Tj, int Oj) {
  return ((type & 1) && ux < Oj) || ((type & 2) && ux >= Tj - Oj) || ((type & 4) && uy < Oj) ||
         ((type & 8) && uy >= Tj - Oj);
}

__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Overlap mask type of a data event from its block counts (2D): bit k set
// when strip k (0 low x, 1 high x, 2 low y, 3 high y; Oj blocks wide) is
// fully known, i.e. every block holds 2^(2J) known cells.
__device__ inline int mask_type_of(const uint8_t* cnt, int F, int Tj, int Oj, int sd) {
  if (Oj <= 0) return 0;
  int type = 0;
  for (int k = 0; k < 4; ++k) {
    bool full = true;
    for (int i = 0; i < Oj * Tj && full; ++i) {
      const int along = i / Tj, across = i % Tj;
      const int ux = (k == 0) ? along : (k == 1) ? Tj - 1 - along : across;
      const int uy = (k == 2) ? along : (k == 3) ? Tj - 1 - along : across;
      int c = 0;
      for (int f = 0; f < F; ++f) c += cnt[f * Tj * Tj + ux + Tj * uy];
      full = (c == sd);
    }
    if (full) type |= 1 << k;
  }
  return type;
}

// Proposals exist only for a non-empty mask of strips with at most one
// strip per axis (the shapes a raster or mirrored raster path produces).
__device__ __forceinline__ bool usable_type(int type) {
  return type != 0 && (type & 3) != 3 && (type & 12) != 12;
}

// Encoder input of TI candidate c under mask type `type`: facies counts of
// the level-J blocks inside the mask divided by 2^(d J), zero outside.
__device__ inline void window_input(const TiDev& t, int Oj, int type, int64_t c, float* x,
                                    int tid, int nthreads, bool round) {
  const int C = t.F, tj = t.Tj;
  const int cx = (int)(c % t.cd[0]), cy = (int)(c / t.cd[0]);
  const float inv = 1.f / (float)t.sd;
  for (int u = tid; u < tj * tj; u += nthreads) {
    const int ux = u % tj, uy = u / tj;
    const bool m = in_mask(type, ux, uy, tj, Oj);
    float rest = (float)t.sd;
    for (int f = 0; f < C - 1; ++f) {
      const float v =
          m ? t.planes[(int64_t)f * t.plane_vol + (cx + ux) + (int64_t)t.px * (cy + uy)] : 0.f;
      x[f * tj * tj + u] = round ? bf(v * inv) : v * inv;
      rest -= v;
    }
    x[(C - 1) * tj * tj + u] = m ? (round ? bf(rest * inv) : rest * inv) : 0.f;
  }
}

// Encoder inputs of the step's items: the block counts of the event record
// divided by 2^(d J) (zero for an empty event, which is never searched).
__global__ void k_event_inputs(const __grid_constant__ WaveArgs a, float* __restrict__ x) {
  const TiDev& t = a.ti;
  const int item = blockIdx.x;
  const int nc = t.F * t.Tj * t.Tj;
  pdl_trigger();
  pdl_wait();   // the event records of this step are complete
  const unsigned char* rec = a.ev.base + (int64_t)item * a.ev.stride;
  const uint8_t* cnt = rec + a.ev.counts_off;
  const bool known = reinterpret_cast<const int*>(rec)[kEvKnown] > 0;
  const float inv = 1.f / (float)t.sd;
  float* xi = x + (int64_t)item * nc;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) xi[i] = known ? cnt[i] * inv : 0.f;
}

// Encoder inputs of TI candidates c0 .. c0 + n - 1 under mask type `type`.
__global__ void k_window_inputs(const __grid_constant__ WaveArgs a, int type, int64_t c0,
                                float* __restrict__ x) {
  const TiDev& t = a.ti;
  const int nc = t.F * t.Tj * t.Tj;
  window_input(t, a.Oj, type, c0 + blockIdx.x, x + (int64_t)blockIdx.x * nc, threadIdx.x,
               blockDim.x, false);
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                          int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

// ---------------------------------------------------------------------------
// Nearest neighbours: scores s_c = table[type][c] . bf16(e) over every
// candidate (BF16 table rows and query, FP32 sums),
// the n_prop best by (score desc, index asc), and the relative gap
// (s_1 - s_nprop) / max(|s_1|, eps). A two-level histogram over [-1, 1]
// finds a threshold that keeps at least n_prop and at most kCollect
// candidates; those are ranked exactly.
// ---------------------------------------------------------------------------
constexpr int kNnThreads = 256;
constexpr int kBins = 1024;
constexpr int kCollect = 512;
constexpr int kScoreCache = 6144;   // candidates whose scores stay in shared memory
constexpr int kSortSmall = 128;     // survivors sorted in registers (4 per lane)

__device__ __forceinline__ float nn_score(const __nv_bfloat16* row, const float* e) {
  float s0 = 0.f, s1 = 0.f;
  const uint4* r = reinterpret_cast<const uint4*>(row);
#pragma unroll
  for (int q = 0; q < 8; ++q) {   // 8 BF16 values per 16-byte load
    const uint4 v = __ldg(r + q);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const float lo = __uint_as_float(w[h] << 16), hi = __uint_as_float(w[h] & 0xFFFF0000u);
      s0 = fmaf(lo, e[8 * q + 2 * h], s0);
      s1 = fmaf(hi, e[8 * q + 2 * h + 1], s1);
    }
  }
  return s0 + s1;
}

__global__ void __launch_bounds__(kNnThreads) k_nnsel(const __grid_constant__ WaveArgs a) {
  __shared__ float e[64];
  __shared__ int hist[kBins];
  __shared__ float cs[kCollect];
  __shared__ int ci[kCollect];
  __shared__ float cache[kScoreCache];
  __shared__ int sh_i[4];
  __shared__ float sh_f[4];
  const TiDev& t = a.ti;
  const int tid = threadIdx.x;
  const int item = blockIdx.x;
  pdl_trigger();
  pdl_wait();
  const int* meta = reinterpret_cast<const int*>(a.ev.base + (int64_t)item * a.ev.stride);
  const int type = meta[kEvMaskType];
  const bool known = meta[kEvKnown] > 0;
  unsigned long long* stats = a.call ? a.call->learn_stats : nullptr;
  if (!known || !usable_type(type)) {
    if (tid == 0) {
      a.prop_gap[item] = -1.f;   // no proposals: full search
      if (stats && known) atomicAdd(&stats[0], 1ull);
    }
    return;
  }
  if (tid == 0 && stats) {
    atomicAdd(&stats[0], 1ull);
    atomicAdd(&stats[1], 1ull);
  }
  if (tid < 64) e[tid] = bf(a.emb[(int64_t)item * 64 + tid]);   // the BF16 query
  for (int b = tid; b < kBins; b += kNnThreads) hist[b] = 0;
  __syncthreads();
  const __nv_bfloat16* tab = a.tables + (int64_t)type * t.P * 64;
  const int np = (int)min((int64_t)a.n_prop, t.P);
  // Threshold search: a histogram of the scores over [lo, hi] (two levels)
  // gives a score thr with at least np candidates at or above it and, when
  // possible, at most kCollect. The exact ranking below checks both counts,
  // so rounding in the binning can only cost a fallback, never a wrong list.
  float lo = -1.5f, hi = 1.5f;
  int above_prev = 0;
  float thr = lo;
  const bool cached = t.P <= kScoreCache;
  for (int level = 0; level < 2; ++level) {
    const float scale = kBins / (hi - lo);
    // warp-uniform trip count; lanes of a warp that fall in the same bin
    // add once (the scores cluster, so plain atomics would serialize)
    for (int64_t cb = 0; cb < t.P; cb += kNnThreads) {
      const int64_t c = cb + tid;
      int b = -1;
      if (c < t.P) {
        float sc;
        if (cached && level > 0) {
          sc = cache[c];
        } else {
          sc = nn_score(tab + c * 64, e);
          if (cached) cache[c] = sc;
        }
        if (sc >= lo && sc < hi) b = min(kBins - 1, max(0, (int)((sc - lo) * scale)));
      }
      const unsigned same = __match_any_sync(0xffffffffu, b);
      if (b >= 0 && (tid & 31) == __ffs(same) - 1) atomicAdd(&hist[b], __popc(same));
    }
    __syncthreads();
    if (tid == 0) {
      int above = above_prev;
      int b = kBins - 1;
      for (; b > 0; --b) {
        if (above + hist[b] >= np) break;
        above += hist[b];
      }
      sh_i[0] = b;
      sh_i[1] = above;   // scores in bins above b (and above the window)
      sh_i[2] = hist[b];
    }
    __syncthreads();
    const int bsel = sh_i[0], above = sh_i[1], inbin = sh_i[2];
    thr = lo + bsel / scale;
    if (above + inbin <= kCollect || level == 1) break;
    // refine inside the selected bin
    const float nlo = thr, nhi = lo + (bsel + 1) / scale;
    above_prev = above;
    __syncthreads();
    for (int bb = tid; bb < kBins; bb += kNnThreads) hist[bb] = 0;
    __syncthreads();
    lo = nlo;
    hi = nhi;
  }
  if (tid == 0) sh_i[3] = 0;
  __syncthreads();
  for (int64_t cb = 0; cb < t.P; cb += kNnThreads) {
    const int64_t c = cb + tid;
    float sc = 0.f;
    bool keep = false;
    if (c < t.P) {
      sc = cached ? cache[c] : nn_score(tab + c * 64, e);
      keep = sc >= thr;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    int base = 0;
    if ((tid & 31) == 0 && bal) base = atomicAdd(&sh_i[3], __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) {
      const int k = base + __popc(bal & ((1u << (tid & 31)) - 1u));
      if (k < kCollect) {
        cs[k] = sc;
        ci[k] = (int)c;
      }
    }
  }
  __syncthreads();
  const int total = sh_i[3];
  const int ncoll = min(total, kCollect);
  if (total > kCollect || ncoll < np) {
    if (tid == 0) a.prop_gap[item] = -1.f;   // threshold not usable: full search
    return;
  }
  // exact rank of each collected candidate: score desc, index asc
  for (int k = tid; k < ncoll; k += kNnThreads) {
    int rank = 0;
    for (int j = 0; j < ncoll; ++j)
      rank += (cs[j] > cs[k]) || (cs[j] == cs[k] && ci[j] < ci[k]);
    if (rank < np) a.prop[(int64_t)item * a.n_prop + rank] = ci[k];
    if (rank == 0) sh_f[1] = cs[k];
    if (rank == np - 1) sh_f[2] = cs[k];
  }
  __syncthreads();
  if (tid == 0) {
    const float s1 = sh_f[1], sn = sh_f[2];
    a.prop_gap[item] = (s1 - sn) / fmaxf(fabsf(s1), 1e-6f);
  }
}

// ---------------------------------------------------------------------------
// The same selection for kNnG data events per CTA: each table row is loaded
// once into registers and dotted with every event of its mask type (the
// events of a wavefront mostly share one), the scores kept in shared memory;
// then one warp per event finds the threshold with the same two-level
// histogram (so the same events fall back to the full search) and ranks the
// survivors with a bitonic sort of (score descending, index ascending) keys.
// For tables of at most kScoreCache windows.
// ---------------------------------------------------------------------------
constexpr int kNnG = 4;

// The row's 64 BF16 values (8 x 16-byte words) dotted with e in the order of
// nn_score (even and odd terms summed apart): the same score bit for bit.
__device__ __forceinline__ float nn_score_regs(const uint4 (&r)[8], const float* e) {
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint32_t w[4] = {r[q].x, r[q].y, r[q].z, r[q].w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const float lo = __uint_as_float(w[h] << 16), hi = __uint_as_float(w[h] & 0xFFFF0000u);
      s0 = fmaf(lo, e[8 * q + 2 * h], s0);
      s1 = fmaf(hi, e[8 * q + 2 * h + 1], s1);
    }
  }
  return s0 + s1;
}

// Ascending order of these keys = score descending, then index ascending.
__device__ __forceinline__ uint64_t nn_rank_key(float sc, int idx) {
  uint32_t u = __float_as_uint(sc);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // ascending with the score
  return ((uint64_t)(~u) << 32) | (uint32_t)idx;
}

struct NnMultiSmem {
  float e[kNnG][64];
  int hist[kNnG][kBins];
  uint64_t keys[kNnG][kCollect];
  int type[kNnG], ok[kNnG], cnt[kNnG];
};

__device__ __forceinline__ float nn_key_score(uint64_t k) {
  const uint32_t ord = ~(uint32_t)(k >> 32);
  return __uint_as_float((ord & 0x80000000u) ? (ord & 0x7FFFFFFFu) : ~ord);
}

// Selection of one data event by one warp from its scores sc[0 .. P): a
// two-level histogram over [-1.5, 1.5) finds a threshold that keeps at least
// n_prop and at most kCollect windows; the survivors' keys (score
// descending, index ascending) are sorted (bitonic, the smallest power of two
// >= their count and >= 64) and the first n_prop written with the gap.
// hist: kBins ints, keys: kCollect words of this warp's shared memory.
// The n_prop best of ncoll <= 32 NPL survivor keys (keys[0 .. ncoll)):
// bitonic sort in registers (element e = NPL lane + r), proposals written,
// gap written by lane 0 and returned to every lane. One warp.
template <int NPL>
__device__ __noinline__ float nn_sort_regs_warp(const WaveArgs& a, int item,
                                                   const uint64_t* keys, int ncoll, int np,
                                                   int lane) {
  uint64_t x[NPL];
#pragma unroll
  for (int r = 0; r < NPL; ++r) {
    const int e = NPL * lane + r;
    x[r] = e < ncoll ? keys[e] : kNoKey;
  }
#pragma unroll
  for (int k = 2; k <= 32 * NPL; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= NPL) {
#pragma unroll
        for (int r = 0; r < NPL; ++r) {
          const int e = NPL * lane + r;
          const uint64_t y = __shfl_xor_sync(0xffffffffu, x[r], j / NPL);
          const bool up = (e & k) == 0, lower = (e & j) == 0;
          x[r] = (lower == up) ? (x[r] < y ? x[r] : y) : (x[r] > y ? x[r] : y);
        }
      } else {
#pragma unroll
        for (int r = 0; r < NPL; ++r)
          if ((r & j) == 0) {
            const int e = NPL * lane + r;
            const bool up = (e & k) == 0;
            const uint64_t u = x[r], v = x[r ^ j];
            if ((u > v) == up) {
              x[r] = v;
              x[r ^ j] = u;
            }
          }
      }
    }
  uint64_t xn = x[0];
  const int rn = (np - 1) % NPL;
#pragma unroll
  for (int r = 0; r < NPL; ++r) {
    const int e = NPL * lane + r;
    if (e < np) a.prop[(int64_t)item * a.n_prop + e] = (int)(x[r] & 0xFFFFFFFFu);
    xn = r == rn ? x[r] : xn;
  }
  const uint64_t k1 = __shfl_sync(0xffffffffu, x[0], 0);
  const uint64_t kn = __shfl_sync(0xffffffffu, xn, (np - 1) / NPL);
  const float s1 = nn_key_score(k1), sn = nn_key_score(kn);
  const float gap = (s1 - sn) / fmaxf(fabsf(s1), 1e-6f);
  if (lane == 0) a.prop_gap[item] = gap;
  return gap;
}

// Level-0 histogram bin of score v (-1 outside [-1.5, 1.5)).
__device__ __forceinline__ int nn_bin0(float v) {
  const float lo = -1.5f, hi = 1.5f, scale = kBins / (hi - lo);
  return (v >= lo && v < hi) ? min(kBins - 1, max(0, (int)((v - lo) * scale))) : -1;
}

__device__ __forceinline__ float nn_select_warp(const WaveArgs& a, int item, const float* sc, int P,
                                             int* hist, uint64_t* keys, int lane,
                                             bool hist_ready = false) {
  const TiDev& t = a.ti;
  const int np = (int)min((int64_t)a.n_prop, t.P);
  float lo = -1.5f, hi = 1.5f;
  int above_prev = 0;
  float thr = lo;
  for (int level = 0; level < 2; ++level) {
    const float scale = kBins / (hi - lo);
    // hist_ready: the caller built the level-0 histogram (nn_bin0)
    if (level > 0 || !hist_ready) {
      for (int b = lane; b < kBins; b += 32) hist[b] = 0;
      __syncwarp();
      for (int cb = 0; cb < P; cb += 32) {
        const int c = cb + lane;
        int b = -1;
        if (c < P) {
          const float v = sc[c];
          if (v >= lo && v < hi) b = min(kBins - 1, max(0, (int)((v - lo) * scale)));
        }
        const unsigned same = __match_any_sync(0xffffffffu, b);
        if (b >= 0 && lane == __ffs(same) - 1) atomicAdd(&hist[b], __popc(same));
      }
    }
    __syncwarp();
    // the highest bin b >= 1 whose count with everything above reaches np
    // (else bin 0): lane L holds bins 32L .. 32L + 31
    int part = 0;
    for (int k = 0; k < 32; ++k) part += hist[32 * lane + k];
    int suffix = part;   // bins of this lane and the lanes above it
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_down_sync(0xffffffffu, suffix, o);
      if (lane + o < 32) suffix += v;
    }
    const int above_lanes = suffix - part;   // bins of the lanes above this one
    int run = above_prev + above_lanes, fb = -1, fabove = 0;
    for (int k = 31; k >= 0; --k) {
      const int b = 32 * lane + k;
      if (b > 0 && run + hist[b] >= np && fb < 0) {
        fb = b;
        fabove = run;
      }
      run += hist[b];
      if (b == 0 && fb < 0) {
        fb = -2;   // reached bin 0 without a hit: bin 0 with `run - hist[0]` above
        fabove = run - hist[0];
      }
    }
    const unsigned hits = __ballot_sync(0xffffffffu, fb >= 0);
    int bsel, above;
    if (hits) {
      const int src = 31 - __clz(hits);
      bsel = __shfl_sync(0xffffffffu, fb, src);
      above = __shfl_sync(0xffffffffu, fabove, src);
    } else {
      bsel = 0;
      above = __shfl_sync(0xffffffffu, fabove, 0);
    }
    const int inbin = hist[bsel];
    thr = lo + bsel / scale;
    // refine past kSortSmall survivors: the proposals and the fallback
    // decisions are those of refining past kCollect (the finer threshold
    // keeps a subset that still holds the n_prop best), the sort is cheaper
    if (above + inbin <= kSortSmall || level == 1) break;
    const float nlo = thr, nhi = lo + (bsel + 1) / scale;
    above_prev = above;
    __syncwarp();
    lo = nlo;
    hi = nhi;
  }
  // survivors: keys (score descending, index ascending)
  int total = 0;
  for (int cb = 0; cb < P; cb += 32) {
    const int c = cb + lane;
    const bool keep = c < P && sc[c] >= thr;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int k = total + __popc(bal & ((1u << lane) - 1u));
      if (k < kCollect) keys[k] = nn_rank_key(sc[c] + 0.f, c);
    }
    total += __popc(bal);
  }
  const int ncoll = min(total, kCollect);
  if (total > kCollect || ncoll < np) {
    if (lane == 0) a.prop_gap[item] = -1.f;   // threshold not usable: full search
    return -1.f;
  }
  __syncwarp();
  // sorted in registers by the warp
  if (ncoll <= kSortSmall) return nn_sort_regs_warp<4>(a, item, keys, ncoll, np, lane);
  if (ncoll <= 2 * kSortSmall) return nn_sort_regs_warp<8>(a, item, keys, ncoll, np, lane);
  return nn_sort_regs_warp<16>(a, item, keys, ncoll, np, lane);
}

// The exact re-rank of k_rerank done by the selecting warp right after its
// selection (simulation mode): Eq. CCW on the event's level-J weights for the
// n_prop proposals (two per lane), the hard-data mismatches, the K best keys
// in the item's first partial list, and the item marked resolved. wsm holds
// at least nch * rows * Tj floats, ksm at least K words (this warp's).
__device__ __forceinline__ void nn_rerank_warp(const WaveArgs& a, int item, float gap, float* wsm,
                                               uint64_t* ksm, int lane) {
  const TiDev& t = a.ti;
  unsigned char* rec = a.ev.base + (int64_t)item * a.ev.stride;
  int* meta = reinterpret_cast<int*>(rec);
  if (meta[kEvKnown] == 0 || gap < 0.f || gap < a.call->gap_theta) return;
  const int np = (int)min((int64_t)a.n_prop, t.P);
  const int K = a.K;
  const int Kp = (int)min((int64_t)K, (int64_t)np);
  const float* W = reinterpret_cast<const float*>(rec + a.ev.w_off);
  const int2* hdl = reinterpret_cast<const int2*>(rec + a.ev.hd_off);
  const int nhd = meta[kEvNHd], cons = meta[kEvConst];
  const int nw = t.nch * t.rows * t.Tj;
  for (int i = lane; i < nw; i += 32) {
    const int ux = i % t.Tj, r = i / t.Tj;
    wsm[i] = W[r * t.TjP + ux];
  }
  __syncwarp();
  // both proposals of the lane row by row, eight loads in flight
  int cq[2], cxq[2], cyq[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int pi = lane + 32 * q;
    cq[q] = pi < np ? a.prop[(int64_t)item * a.n_prop + pi] : 0;
    cxq[q] = cq[q] % t.cd[0];
    cyq[q] = cq[q] / t.cd[0];
  }
  float acc[2] = {0.f, 0.f};
  for (int ch = 0; ch < t.nch; ++ch) {
    const float* plane = t.planes + (int64_t)(t.plane0 + ch) * t.plane_vol;
    for (int row = 0; row < t.rows; ++row) {
      const float* wr = wsm + (ch * t.rows + row) * t.Tj;
      const float* p0 = plane + cxq[0] + (int64_t)t.px * (cyq[0] + row);
      const float* p1 = plane + cxq[1] + (int64_t)t.px * (cyq[1] + row);
      // integer-valued products: the sums are exact in any order
      float s0 = 0.f, s1 = 0.f, u0 = 0.f, u1 = 0.f;
      int ux = 0;
      for (; ux + 4 <= t.Tj; ux += 4) {
        const float a0 = __ldg(p0 + ux), a1 = __ldg(p0 + ux + 1);
        const float a2 = __ldg(p0 + ux + 2), a3 = __ldg(p0 + ux + 3);
        const float b0 = __ldg(p1 + ux), b1 = __ldg(p1 + ux + 1);
        const float b2 = __ldg(p1 + ux + 2), b3 = __ldg(p1 + ux + 3);
        const float w0 = wr[ux], w1 = wr[ux + 1], w2 = wr[ux + 2], w3 = wr[ux + 3];
        s0 = fmaf(w0, a0, s0);
        s1 = fmaf(w1, a1, s1);
        s0 = fmaf(w2, a2, s0);
        s1 = fmaf(w3, a3, s1);
        u0 = fmaf(w0, b0, u0);
        u1 = fmaf(w1, b1, u1);
        u0 = fmaf(w2, b2, u0);
        u1 = fmaf(w3, b3, u1);
      }
      for (; ux < t.Tj; ++ux) {
        s0 = fmaf(wr[ux], __ldg(p0 + ux), s0);
        u0 = fmaf(wr[ux], __ldg(p1 + ux), u0);
      }
      acc[0] += s0 + s1;
      acc[1] += u0 + u1;
    }
  }
  uint64_t key[2] = {kNoKey, kNoKey};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (lane + 32 * q >= np) continue;
    const uint8_t* tb =
        t.ti + (int64_t)t.s * cxq[q] + (int64_t)t.tp[0] * ((int64_t)t.s * cyq[q]);
    int mis = 0;
    for (int k = 0; k < nhd; ++k) {
      const int2 e = hdl[k];
      mis += (__ldg(tb + e.x) != (uint8_t)(e.y & 0xFF));
    }
    key[q] = make_key(mis, __float2int_rn(acc[q]) + cons, cq[q]);
  }
  // the Kp smallest keys, in order
  uint64_t prev = 0;
  for (int r = 0; r < Kp; ++r) {
    uint64_t m = kNoKey;
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if ((r == 0 || key[q] > prev) && key[q] < m) m = key[q];
    m = warp_min_u64(m);
    prev = m;
    if (lane == 0) ksm[r] = m;
  }
  __syncwarp();
  unsigned long long* dst = a.part + (int64_t)item * a.n_parts * K;
  for (int i = lane; i < a.n_parts * K; i += 32) {
    const int p = i / K, r = i % K;
    dst[i] = (p == 0 && r < Kp) ? ksm[r] : kNoKey;
  }
  if (lane == 0) {
    meta[kEvResolved] = 1;
    if (a.call->learn_stats) atomicAdd(&a.call->learn_stats[2], 1ull);
  }
}

__global__ void __launch_bounds__(kNnThreads) k_nnsel_multi(const __grid_constant__ WaveArgs a) {
  extern __shared__ unsigned char nn_smem[];
  NnMultiSmem& S = *reinterpret_cast<NnMultiSmem*>(nn_smem);
  float* cache = reinterpret_cast<float*>(nn_smem + sizeof(NnMultiSmem));   // [kNnG][P]
  const TiDev& t = a.ti;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.x * kNnG;
  const int P = (int)t.P;
  pdl_trigger();
  pdl_wait();
  unsigned long long* stats = a.call ? a.call->learn_stats : nullptr;
  if (tid < kNnG) {
    const int item = i0 + tid;
    int type = -1, ok = 0;
    if (item < a.n_items) {
      const int* meta = reinterpret_cast<const int*>(a.ev.base + (int64_t)item * a.ev.stride);
      type = meta[kEvMaskType];
      const bool known = meta[kEvKnown] > 0;
      ok = known && usable_type(type);
      if (!ok) a.prop_gap[item] = -1.f;   // no proposals: full search
      if (stats && known) atomicAdd(&stats[0], 1ull);
      if (stats && ok) atomicAdd(&stats[1], 1ull);
    }
    S.type[tid] = ok ? type : -1;
    S.ok[tid] = ok;
  }
  for (int i = tid; i < kNnG * 64; i += kNnThreads) {
    const int g = i / 64, item = i0 + g;
    S.e[g][i % 64] = item < a.n_items ? bf(a.emb[(int64_t)item * 64 + i % 64]) : 0.f;
  }
  __syncthreads();
  // scores: every row of a type present in the group, loaded once
  for (int g = 0; g < kNnG; ++g) {
    const int type = S.type[g];
    if (type < 0) continue;
    bool first = true;
    for (int h = 0; h < g; ++h) first &= S.type[h] != type;
    if (!first) continue;   // already scored with an earlier event of this type
    const uint4* tab = reinterpret_cast<const uint4*>(a.tables + (int64_t)type * t.P * 64);
    for (int c = tid; c < P; c += kNnThreads) {
      uint4 r[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) r[q] = __ldg(tab + (int64_t)c * 8 + q);
#pragma unroll
      for (int h = 0; h < kNnG; ++h)
        if (S.type[h] == type) cache[h * P + c] = nn_score_regs(r, S.e[h]);
    }
  }
  __syncthreads();
  if (warp >= kNnG || !S.ok[warp]) return;
  // selection: one warp per event
  const float gap =
      nn_select_warp(a, i0 + warp, cache + warp * P, P, S.hist[warp], S.keys[warp], lane);
  if (a.fuse_rerank)
    nn_rerank_warp(a, i0 + warp, gap, reinterpret_cast<float*>(S.hist[warp]), S.keys[warp], lane);
}

// ---------------------------------------------------------------------------
// The same selection with the scores from the tcgen05 tensor cores: the
// tables are kept a second time in the MMA's K-major core-matrix layout, one
// 16 KB block per 128 windows ([16 row groups][8 K chunks][8 rows][16 bytes],
// zero rows past P); a CTA takes G = 8 or 12 data events (MMA N = 16,
// columns G..15 zero; one warp per event, at least 8), and for each mask type
// among them streams that type's blocks through 2-8 shared-memory stages
// (bulk copies) into one MMA chain (M = 128 windows, K = 64), the scores of
// every block in their own tensor memory columns. The scores then move to
// shared memory, and the selection runs in CTA-wide phases; the survivors'
// keys take the stages' space once the MMAs are done. Twelve events per CTA
// let a wavefront of up to 12 x (SM count) events run in one round of CTAs.
// For tables of at most kNnTcMaxP windows.
// ---------------------------------------------------------------------------
constexpr int kNnTcMaxP = 24 * 128;
constexpr int kNnTcBlock = 128 * 64;   // BF16 values per 128-window block
constexpr int kNnTcMaxStages = 8;
constexpr int kNnTcSmemMax = 227 * 1024;

// Histograms of the tensor-core selector: bin b at b + b / 32, so that lane L
// reading its 32 bins 32 L .. 32 L + 31 touches 32 different banks.
constexpr int kBinsPad = kBins + kBins / 32;
__device__ __forceinline__ int hpad(int b) { return b + (b >> 5); }

template <int G>
struct NnTcSmem {
  uint64_t bar_load[kNnTcMaxStages], bar_mma[kNnTcMaxStages], bar_done;
  uint32_t tslot;
  int flag;
  int type[G], ok[G];
  // per event: threshold, level-1 range, count above it, survivors, state
  float thr[G], lo1[G], hi1[G];
  int above0[G], need1[G], cnt[G];
  float gap[G];
  int hist[G][kBinsPad];
};

// Threads of k_nnsel_tc<G>: one warp per event, at least 8 warps.
template <int G>
__host__ __device__ constexpr int nn_tc_threads() {
  return G > 8 ? 32 * G : 256;
}

// Offset (bytes) of element (row, k) of a K-major operand block with 8-row
// groups of all 8 K chunks: [rows / 8][8 chunks][8 rows][16 bytes].
__host__ __device__ __forceinline__ int nn_tc_off(int row, int k) {
  return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// k_nnsel_tc<G>'s shared memory for P windows: the fixed part, the B
// operand, then as many 16 KB stages as fit beside the scores (at least 2,
// and enough to hold the survivors' keys, G x kCollect words, afterwards).
template <int G>
__host__ __device__ inline int nn_tc_head() {
  return ((int)sizeof(NnTcSmem<G>) + 127) & ~127;
}
template <int G>
__host__ __device__ inline int nn_tc_min_stages() {
  const int k = (G * kCollect * 8 + 16383) / 16384;
  return k < 2 ? 2 : k;
}
template <int G>
__host__ __device__ inline int nn_tc_stages(int64_t P) {
  const int64_t room = kNnTcSmemMax - nn_tc_head<G>() - 2048 - (int64_t)sizeof(float) * G * P;
  const int64_t n = room / 16384;
  const int lo = nn_tc_min_stages<G>();
  return (int)(n < lo ? lo : n > kNnTcMaxStages ? kNnTcMaxStages : n);
}
template <int G>
__host__ __device__ inline int nn_tc_smem(int64_t P) {
  return nn_tc_head<G>() + 2048 + nn_tc_stages<G>(P) * 16384 + (int)(sizeof(float) * G * P);
}

// The threshold bin of a padded histogram (one warp, lane L taking bins
// 32 L .. 32 L + 31): the highest bin b >= 1 whose count together with
// everything above it (above_prev lies above the histogram's range) reaches
// np, else bin 0; `above` is the count above that bin. The search of
// nn_select_warp on the padded layout.
__device__ __forceinline__ void nn_threshold_pad(const int* hist, int np, int above_prev, int lane,
                                                 int& bsel, int& above) {
  const int* hl = hist + 33 * lane;   // bins 32 lane .. 32 lane + 31
  int part = 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) part += hl[k];
  int suffix = part;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_down_sync(0xffffffffu, suffix, o);
    if (lane + o < 32) suffix += v;
  }
  int run = above_prev + suffix - part, fb = -1, fabove = 0;
#pragma unroll
  for (int k = 31; k >= 0; --k) {
    const int b = 32 * lane + k, h = hl[k];
    if (b > 0 && run + h >= np && fb < 0) {
      fb = b;
      fabove = run;
    }
    run += h;
    if (b == 0 && fb < 0) {
      fb = -2;
      fabove = run - h;
    }
  }
  const unsigned hits = __ballot_sync(0xffffffffu, fb >= 0);
  if (hits) {
    const int src = 31 - __clz(hits);
    bsel = __shfl_sync(0xffffffffu, fb, src);
    above = __shfl_sync(0xffffffffu, fabove, src);
  } else {
    bsel = 0;
    above = __shfl_sync(0xffffffffu, fabove, 0);
  }
}

// Selection for the CTA's G events in CTA-wide phases, with the
// thresholds, survivors and proposals of nn_select_warp: each warp finds its
// event's threshold (level 0 from the histogram the epilogue built, level 1
// over the threshold bin when more than kSortSmall would survive), all
// threads then build the level-1 histograms and collect every event's
// survivors; each warp sorts its event's survivors (up to kCollect, in
// keys[h * kCollect ..]) in registers. Sets S.gap[h] (-1: the event falls
// back to the full search).
template <int G>
__device__ __forceinline__ void nn_select_cta_tc(const WaveArgs& a, NnTcSmem<G>& S,
                                                 const float* cache, uint64_t* keys, int P,
                                                 int i0, int tid, int warp, int lane) {
  constexpr int NT = nn_tc_threads<G>();
  const int np = (int)min((int64_t)a.n_prop, a.ti.P);
  const bool mine = warp < G && S.ok[warp];
  if (mine) {
    const float lo = -1.5f, hi = 1.5f, scale = kBins / (hi - lo);
    int bsel, above;
    nn_threshold_pad(S.hist[warp], np, 0, lane, bsel, above);
    const int inbin = S.hist[warp][hpad(bsel)];
    const float thr = lo + bsel / scale;
    if (lane == 0) {
      S.thr[warp] = thr;
      S.need1[warp] = above + inbin > kSortSmall;
      S.lo1[warp] = thr;
      S.hi1[warp] = lo + (bsel + 1) / scale;
      S.above0[warp] = above;
    }
  } else if (warp < G && lane == 0) {
    S.need1[warp] = 0;
  }
  if (warp < G && lane == 0) S.cnt[warp] = 0;
  __syncthreads();
  bool any = false;
#pragma unroll
  for (int h = 0; h < G; ++h) any |= S.ok[h] && S.need1[h];
  if (any) {
    for (int i = tid; i < G * kBinsPad; i += NT) {
      const int h = i / kBinsPad;
      if (S.ok[h] && S.need1[h]) (&S.hist[0][0])[i] = 0;
    }
    __syncthreads();
    for (int h = 0; h < G; ++h) {
      if (!S.ok[h] || !S.need1[h]) continue;
      const float lo = S.lo1[h], hi = S.hi1[h], scale = kBins / (hi - lo);
      const float* sc = cache + h * P;
      for (int c = tid; c < P; c += NT) {
        const float v = sc[c];
        if (v >= lo && v < hi)
          atomicAdd(&S.hist[h][hpad(min(kBins - 1, max(0, (int)((v - lo) * scale))))], 1);
      }
    }
    __syncthreads();
    if (mine && S.need1[warp]) {
      const float lo = S.lo1[warp], hi = S.hi1[warp], scale = kBins / (hi - lo);
      int bsel, above;
      nn_threshold_pad(S.hist[warp], np, S.above0[warp], lane, bsel, above);
      if (lane == 0) S.thr[warp] = lo + bsel / scale;
    }
    __syncthreads();
  }
  // survivors of every event, their keys in any order (sorted below)
  for (int h = 0; h < G; ++h) {
    if (!S.ok[h]) continue;
    const float thr = S.thr[h];
    const float* sc = cache + h * P;
    for (int c = tid; c < P; c += NT) {
      const float v = sc[c];
      if (v >= thr) {
        const int k = atomicAdd(&S.cnt[h], 1);
        if (k < kCollect) keys[h * kCollect + k] = nn_rank_key(v + 0.f, c);
      }
    }
  }
  __syncthreads();
  if (mine) {
    const int item = i0 + warp;
    const int total = S.cnt[warp], ncoll = min(total, kCollect);
    if (total > kCollect || ncoll < np) {
      if (lane == 0) {
        a.prop_gap[item] = -1.f;   // threshold not usable: full search
        S.gap[warp] = -1.f;
      }
    } else {
      // every survivor set sorted by its own warp in registers
      uint64_t* kw = keys + warp * kCollect;
      const float gap = ncoll <= kSortSmall ? nn_sort_regs_warp<4>(a, item, kw, ncoll, np, lane)
                        : ncoll <= 2 * kSortSmall
                            ? nn_sort_regs_warp<8>(a, item, kw, ncoll, np, lane)
                            : nn_sort_regs_warp<16>(a, item, kw, ncoll, np, lane);
      if (lane == 0) S.gap[warp] = gap;
    }
  } else if (warp < G && lane == 0) {
    S.gap[warp] = -1.f;
  }
  __syncthreads();
}

__global__ void k_tables_mma(const __nv_bfloat16* __restrict__ tables, int64_t P, int nblk,
                             __nv_bfloat16* __restrict__ out) {
  const int64_t n = (int64_t)16 * nblk * kNnTcBlock;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    // i enumerates the source order (type, window, k) over the padded rows
    const int k = (int)(i % 64);
    const int64_t r = (i / 64) % ((int64_t)nblk * 128), type = i / 64 / ((int64_t)nblk * 128);
    const __nv_bfloat16 v = r < P ? tables[(type * P + r) * 64 + k] : __float2bfloat16_rn(0.f);
    const int64_t blk = type * nblk + r / 128;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(out) +
                                      blk * (int64_t)kNnTcBlock * 2 +
                                      nn_tc_off((int)(r % 128), k)) = v;
  }
}

template <int G>
__global__ void __launch_bounds__(nn_tc_threads<G>(), 1)
    k_nnsel_tc(const __grid_constant__ WaveArgs a) {
  constexpr int NT = nn_tc_threads<G>();
  extern __shared__ __align__(128) unsigned char nn_smem[];
  NnTcSmem<G>& S = *reinterpret_cast<NnTcSmem<G>*>(nn_smem);
  const TiDev& t = a.ti;
  const int P = (int)t.P;
  const int NS = nn_tc_stages<G>(P);
  unsigned char* eb = nn_smem + nn_tc_head<G>();                       // B: 16 rows
  unsigned char* stage = eb + 2048;                                    // NS x 16 KB
  float* cache = reinterpret_cast<float*>(stage + NS * 16384);        // [G][P]
  // the survivors' keys [G][kCollect] over the stages, once the MMAs are done
  uint64_t* keys = reinterpret_cast<uint64_t*>(stage);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.x * G;
  const int nblk = (P + 127) / 128;
  pdl_trigger();
  // set-up that reads nothing the predecessor writes, while it finishes
  for (int i = tid; i < G * kBinsPad; i += NT) (&S.hist[0][0])[i] = 0;
  uint32_t ncols = 32;
  while ((int)ncols < nblk * 16) ncols <<= 1;
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init(&S.bar_load[k], 1);
      mbar_init(&S.bar_mma[k], 1);
    }
    mbar_init(&S.bar_done, 1);
    S.flag = 0;
    fence_mbar_init();
  }
  // the embeddings and event records are complete, and every earlier kernel
  // has released its tensor memory (allocating before this wait could block
  // a predecessor's allocation on the same SM while this CTA waits for it)
  pdl_wait();
  if (warp == 0) tmem_alloc(&S.tslot, ncols);
  unsigned long long* stats = a.call ? a.call->learn_stats : nullptr;
  if (tid < G) {
    const int item = i0 + tid;
    int type = -1, ok = 0;
    if (item < a.n_items) {
      const int* meta = reinterpret_cast<const int*>(a.ev.base + (int64_t)item * a.ev.stride);
      type = meta[kEvMaskType];
      const bool known = meta[kEvKnown] > 0;
      ok = known && usable_type(type);
      if (!ok) a.prop_gap[item] = -1.f;   // no proposals: full search
      if (stats && known) atomicAdd(&stats[0], 1ull);
      if (stats && ok) atomicAdd(&stats[1], 1ull);
    }
    S.type[tid] = ok ? type : -1;
    S.ok[tid] = ok;
  }
  // B operand: the BF16 query of event h in row h (rows G..15 zero)
  for (int i = tid; i < 16 * 64; i += NT) {
    const int h = i / 64, k = i % 64, item = i0 + h;
    const float v = (h < G && item < a.n_items) ? a.emb[(int64_t)item * 64 + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(eb + nn_tc_off(h, k)) = __float2bfloat16_rn(v);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tslot;
  const uint32_t idesc = instr_desc(true, 128, 16);
  const uint32_t eb_addr = smem_u32(eb), st_addr = smem_u32(stage);
  // warp w reads tensor memory lanes 32 (w % 4) ..; the NT / 128 warps of a
  // lane quarter take every (NT / 128)-th block
  const int quarter = warp & 3, part = warp >> 2, parts = NT / 128;
  const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
  // blocks are numbered over all passes (b = passes * nblk + j): block b
  // uses stage b % NS, the (b / NS)-th use of that stage's barriers
  int issued = 0;   // thread 0: blocks whose copy was issued
  uint32_t passes = 0;
  for (int g = 0; g < G; ++g) {
    const int type = S.type[g];
    if (type < 0) continue;
    bool first = true;
    for (int h = 0; h < g; ++h) first &= S.type[h] != type;
    if (!first) continue;   // scored with an earlier event of this type
    const int b0 = (int)passes * nblk;
    // CTAs start at different blocks of the table so that they do not all
    // read the same L2 lines at the same time
    const int start = (int)((blockIdx.x * 5u) % (unsigned)nblk);
    volatile int* vflag = &S.flag;
    if (tid == 0) {
      // copies: block b into stage b % NS once the MMAs of block b - NS,
      // the stage's previous use, are done
      const __nv_bfloat16* tab = a.tables_mma + (int64_t)type * nblk * kNnTcBlock;
      for (int b = b0; b < b0 + nblk; ++b) {
        const int sidx = b % NS;
        if (b >= NS && !mbar_wait_bounded(&S.bar_mma[sidx], (uint32_t)(b / NS - 1) & 1u)) {
          *vflag = 1;
          break;
        }
        if (*vflag) break;
        mbar_arrive_expect_tx(&S.bar_load[sidx], 16384u);
        bulk_g2s(stage + sidx * 16384, tab + (int64_t)((start + b - b0) % nblk) * kNnTcBlock,
                 16384u, &S.bar_load[sidx]);
        issued = b + 1;
      }
    } else if (tid == 32) {
      // MMAs: block b's scores into columns 16 x (its table block); each
      // thread alone polls its barriers (the others wait at the CTA barrier)
      bool ok = true;
      for (int b = b0; b < b0 + nblk; ++b) {
        const int sidx = b % NS;
        if (*vflag || !mbar_wait_bounded(&S.bar_load[sidx], (uint32_t)(b / NS) & 1u)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t col = (uint32_t)(((start + b - b0) % nblk) * 16);
#pragma unroll
        for (int k16 = 0; k16 < 4; ++k16)
          mma_f16(tmem + col,
                  smem_desc(st_addr + (uint32_t)(sidx * 16384 + k16 * 256), 128u, 1024u),
                  smem_desc(eb_addr + (uint32_t)(k16 * 256), 128u, 1024u), idesc,
                  k16 > 0 ? 1u : 0u);
        mma_commit(&S.bar_mma[sidx]);
      }
      if (!ok) *vflag = 1;
      mma_commit(&S.bar_done);
      if (!mbar_wait_bounded(&S.bar_done, passes & 1u)) *vflag = 1;
    }
    __syncthreads();
    if (S.flag) break;
    mbar_try_wait(&S.bar_done, passes & 1u);   // every thread observes the phase
    ++passes;
    tc_fence_after();
    for (int j = part; j < nblk; j += parts) {
      uint32_t v[16];
      tmem_ld16(lane_base + (uint32_t)(j * 16), v);
      const int c = 128 * j + quarter * 32 + lane;
      if (c < P) {
        // scores to shared memory, and the level-0 histogram of each event
#pragma unroll
        for (int h = 0; h < G; ++h)
          if (S.type[h] == type) {
            const float sc = __uint_as_float(v[h]);
            cache[h * P + c] = sc;
            const int b = nn_bin0(sc);
            if (b >= 0) atomicAdd(&S.hist[h][hpad(b)], 1);
          }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  const bool failed = S.flag != 0;
  if (failed && tid == 0) {
    // a copy or commit never arrived: let what is in flight land (bounded)
    if (a.status) atomicOr(a.status, kStatusTimeout);
    mbar_wait_bounded(&S.bar_done, passes & 1u);
    // the last copy issued into each stage (an earlier one has landed)
    for (int b = issued - NS > 0 ? issued - NS : 0; b < issued; ++b)
      mbar_wait_bounded(&S.bar_load[b % NS], (uint32_t)(b / NS) & 1u);
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
  if (failed) {
    if (warp < G && lane == 0 && i0 + warp < a.n_items)
      a.prop_gap[i0 + warp] = -1.f;   // no proposals: full search
    return;
  }
  nn_select_cta_tc<G>(a, S, cache, keys, P, i0, tid, warp, lane);
  if (a.fuse_rerank && warp < G && S.ok[warp])
    nn_rerank_warp(a, i0 + warp, S.gap[warp], reinterpret_cast<float*>(S.hist[warp]),
                   keys + warp * kCollect, lane);
}

// Event records from explicit block counts (the query entry point): known
// cells, mask type and counts, as the event kernel writes them.
__global__ void k_records_from_counts(const __grid_constant__ WaveArgs a, const uint8_t* counts,
                                      int32_t* type_out) {
  __shared__ int red[kWarps];
  const TiDev& t = a.ti;
  const int tid = threadIdx.x, item = blockIdx.x;
  const int nc = t.F * t.Tj * t.Tj;
  const uint8_t* src = counts + (int64_t)item * nc;
  unsigned char* rec = a.ev.base + (int64_t)item * a.ev.stride;
  int known = 0;
  for (int i = tid; i < nc; i += blockDim.x) {
    const uint8_t v = src[i];
    rec[a.ev.counts_off + i] = v;
    known += v;
  }
  for (int o = 16; o > 0; o >>= 1) known += __shfl_xor_sync(0xffffffffu, known, o);
  if ((tid & 31) == 0) red[tid >> 5] = known;
  __syncthreads();
  if (tid == 0) {
    int k = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) k += red[w];
    int* meta = reinterpret_cast<int*>(rec);
    const int type = mask_type_of(src, t.F, t.Tj, a.Oj, t.sd);
    meta[kEvKnown] = k;
    meta[kEvMaskType] = type;
    meta[kEvResolved] = 0;
    if (type_out) type_out[item] = type;
  }
}

// Encoder inputs for training: what 0 from block counts, 1 TI windows.
__global__ void k_inputs(const __grid_constant__ WaveArgs a, int what, const uint8_t* counts,
                         const int32_t* cand, int32_t* type, int n, float* out) {
  const TiDev& t = a.ti;
  const int i = blockIdx.x;
  if (i >= n) return;
  const int nc = t.F * t.Tj * t.Tj;
  float* x = out + (int64_t)i * nc;
  if (what == 0) {
    const uint8_t* src = counts + (int64_t)i * nc;
    const float inv = 1.f / (float)t.sd;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) x[k] = src[k] * inv;
    if (threadIdx.x == 0 && type) type[i] = mask_type_of(src, t.F, t.Tj, a.Oj, t.sd);
  } else {
    const int ty = type[i];
    const int64_t c = cand[i];
    if (c < 0 || c >= t.P || ty < 0 || ty > 15) {   // out of range: zeros
      for (int k = threadIdx.x; k < nc; k += blockDim.x) x[k] = 0.f;
      return;
    }
    window_input(t, a.Oj, ty, c, x, threadIdx.x, blockDim.x, false);
  }
}

// ---------------------------------------------------------------------------
// Exact re-rank of the proposals (Eq. CCW on the level-J weights of the
// event record, hard-data mismatches of Sec. 4.4), K best by the ranking
// key. Settles the item (per-part lists for the finish kernel, resolved
// flag) when the embedding gap is at least gap_theta.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rerank(const __grid_constant__ WaveArgs a) {
  __shared__ uint64_t keys[CCW_MAX_TOPK];
  __shared__ uint64_t red[9];
  const TiDev& t = a.ti;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int item = blockIdx.x;
  pdl_trigger();
  pdl_wait();
  unsigned char* rec = a.ev.base + (int64_t)item * a.ev.stride;
  int* meta = reinterpret_cast<int*>(rec);
  const float gap = a.prop_gap[item];
  // gap < 0: no proposals were written for this item
  if (meta[kEvKnown] == 0 || gap < 0.f || gap < a.call->gap_theta) return;
  const int np = (int)min((int64_t)a.n_prop, t.P);
  const int K = a.K;
  const int Kp = (int)min((int64_t)K, (int64_t)np);
  const float* W = reinterpret_cast<const float*>(rec + a.ev.w_off);
  const int2* hdl = reinterpret_cast<const int2*>(rec + a.ev.hd_off);
  const int nhd = meta[kEvNHd], cons = meta[kEvConst];
  // 4 threads per proposal, rows split among them
  const int pi = tid >> 2, part = tid & 3;
  uint64_t key = kNoKey;
  float acc = 0.f;
  int c = -1;
  if (pi < np) {
    c = a.prop[(int64_t)item * a.n_prop + pi];
    const int cx = c % t.cd[0], cy = c / t.cd[0];
    for (int ch = 0; ch < t.nch; ++ch) {
      const float* plane = t.planes + (int64_t)(t.plane0 + ch) * t.plane_vol;
      for (int row = part; row < t.rows; row += 4) {
        const float* wr = W + (ch * t.rows + row) * t.TjP;
        const float* pr = plane + (cx) + (int64_t)t.px * (cy + row);
        // integer-valued products: the sum is exact in any order, so four
        // partial sums keep four loads in flight
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int ux = 0;
        for (; ux + 4 <= t.Tj; ux += 4) {
          const float p0 = __ldg(pr + ux), p1 = __ldg(pr + ux + 1);
          const float p2 = __ldg(pr + ux + 2), p3 = __ldg(pr + ux + 3);
          s0 = fmaf(wr[ux], p0, s0);
          s1 = fmaf(wr[ux + 1], p1, s1);
          s2 = fmaf(wr[ux + 2], p2, s2);
          s3 = fmaf(wr[ux + 3], p3, s3);
        }
        for (; ux < t.Tj; ++ux) s0 = fmaf(wr[ux], __ldg(pr + ux), s0);
        acc += (s0 + s1) + (s2 + s3);
      }
    }
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (pi < np && part == 0) {
    const uint8_t* tb = t.ti + (int64_t)t.s * (c % t.cd[0]) +
                        (int64_t)t.tp[0] * ((int64_t)t.s * (c / t.cd[0]));
    int mis = 0;
    for (int k = 0; k < nhd; ++k) {
      const int2 e = hdl[k];
      mis += (__ldg(tb + e.x) != (uint8_t)(e.y & 0xFF));
    }
    key = make_key(mis, __float2int_rn(acc) + cons, c);
  }
  // K smallest keys of the proposals
  uint64_t prev = 0;
  for (int r = 0; r < Kp; ++r) {
    uint64_t m = (r == 0 || key > prev) ? key : kNoKey;
    m = warp_min_u64(m);
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = lane < 8 ? red[lane] : kNoKey;
      w = warp_min_u64(w);
      if (lane == 0) red[8] = w;
    }
    __syncthreads();
    prev = red[8];
    if (tid == 0) keys[r] = prev;
    __syncthreads();
  }
  // the item's lists: the proposals' K best in the first part, empty others
  unsigned long long* dst = a.part + (int64_t)item * a.n_parts * K;
  for (int i = tid; i < a.n_parts * K; i += 256) {
    const int p = i / K, r = i % K;
    dst[i] = (p == 0 && r < Kp) ? keys[r] : kNoKey;
  }
  if (tid == 0) {
    meta[kEvResolved] = 1;
    if (a.call->learn_stats) atomicAdd(&a.call->learn_stats[2], 1ull);
  }
}

// ---------------------------------------------------------------------------
int64_t enc_tc_image_bytes(int C, int tj);
bool net_infer_fused_fits(int C, int tj);
cudaError_t net_infer_tc_records(const float* P, const void* wimg, int C, int tj,
                                 const unsigned char* rec, int64_t stride, int counts_off,
                                 float inv, int N, float* emb, int* status, cudaStream_t st,
                                 bool pdl);

// Kernel launches of one launch_encode_items.
int encode_items_launches(int F, int Tj, bool img) {
  if (img && enc_tc_image_bytes(F, Tj) > 0) return 1;
  return 1 + (net_infer_fused_fits(F, Tj) ? 1 : 5);
}

cudaError_t launch_encode_items(const WaveArgs& a, float* x, float* act, bool pdl,
                                cudaStream_t st) {
  if (a.enc_img && enc_tc_image_bytes(a.ti.F, a.ti.Tj) > 0)
    // the tensor-core pass reads the block counts from the event records
    return net_infer_tc_records(a.net, a.enc_img, a.ti.F, a.ti.Tj, a.ev.base, a.ev.stride,
                                a.ev.counts_off, 1.f / (float)a.ti.sd, a.n_items, a.emb,
                                a.status, st, pdl);
  cudaError_t e = launch_pdl(k_event_inputs, dim3(a.n_items), dim3(128), 0, st, pdl, a, x);
  if (e != cudaSuccess) return e;
  return net_infer(a.net, a.ti.F, a.ti.Tj, x, a.n_items, act, a.emb, st, a.status, 0,
                   a.enc_img);
}

// Table of mask type `type`: embeddings of every candidate window, in
// chunks of `chunk` candidates through the scratch x, act, emb.
cudaError_t launch_encode_tables(const WaveArgs& a, int type, __nv_bfloat16* tables, float* x,
                                 float* act, float* emb, int chunk, cudaStream_t st) {
  for (int64_t c0 = 0; c0 < a.ti.P; c0 += chunk) {
    const int n = (int)std::min<int64_t>(chunk, a.ti.P - c0);
    k_window_inputs<<<n, 128, 0, st>>>(a, type, c0, x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = net_infer(a.net, a.ti.F, a.ti.Tj, x, n, act, emb, st, a.status, 0, a.enc_img)) !=
        cudaSuccess)
      return e;
    k_to_bf16<<<256, 256, 0, st>>>(emb, tables + ((int64_t)type * a.ti.P + c0) * 64,
                                   (int64_t)n * 64);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_tables_mma(const __nv_bfloat16* tables, int64_t P, __nv_bfloat16* out,
                              cudaStream_t st) {
  const int nblk = (int)((P + 127) / 128);
  k_tables_mma<<<1024, 256, 0, st>>>(tables, P, nblk, out);
  return cudaGetLastError();
}

int64_t tables_mma_elems(int64_t P) {
  return P <= kNnTcMaxP ? (int64_t)16 * ((P + 127) / 128) * kNnTcBlock : 0;
}

static int g_nn_path = 0;   // ccw_set_nn_path

// Does launch_nnsel also re-rank (simulation calls whose weights fit the
// warp's scratch)? Then no k_rerank launch follows.
bool nnsel_fuses_rerank_shape(int64_t P, int nch, int rows, int Tj, int n_prop) {
  return g_nn_path != 2 && P <= kScoreCache && nch * rows * Tj <= kBins && n_prop <= 64;
}
bool nnsel_fuses_rerank(const WaveArgs& a) {
  return a.call != nullptr && a.part != nullptr &&
         nnsel_fuses_rerank_shape(a.ti.P, a.ti.nch, a.ti.rows, a.ti.Tj, a.n_prop);
}

template <int G>
static cudaError_t launch_nnsel_tc(const WaveArgs& a, bool pdl, cudaStream_t st) {
  // one CTA per SM when the scores take more than half of the tensor memory
  int smem = nn_tc_smem<G>(a.ti.P);
  if ((a.ti.P + 127) / 128 * 16 > 256 && smem < 120 * 1024) smem = 120 * 1024;
  static int configured = 0;
  if (smem > configured) {
    cudaError_t e =
        cudaFuncSetAttribute(k_nnsel_tc<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  return launch_pdl(k_nnsel_tc<G>, dim3((a.n_items + G - 1) / G), dim3(nn_tc_threads<G>()),
                    smem, st, pdl, a);
}

cudaError_t launch_nnsel(const WaveArgs& a0, bool pdl, cudaStream_t st) {
  WaveArgs a = a0;
  a.fuse_rerank = nnsel_fuses_rerank(a0) ? 1 : 0;
  if ((g_nn_path == 0 || g_nn_path == 3) && a.tables_mma && a.ti.P <= kNnTcMaxP) {
    // twelve events per CTA when eight would need more CTAs than there are
    // SMs (and they fit beside the scores), else eight
    static int sms = 0;
    if (!sms) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = 1;
    }
    const bool g12 = nn_tc_smem<12>(a.ti.P) <= kNnTcSmemMax &&
                     (g_nn_path == 3 || a.n_items > 8 * sms);
    return g12 ? launch_nnsel_tc<12>(a, pdl, st) : launch_nnsel_tc<8>(a, pdl, st);
  }
  if ((g_nn_path <= 1 || g_nn_path == 3) && a.ti.P <= kScoreCache) {
    const int smem = (int)(sizeof(NnMultiSmem) + sizeof(float) * kNnG * a.ti.P);
    static int configured = 0;
    if (smem > configured) {
      cudaError_t e =
          cudaFuncSetAttribute(k_nnsel_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      configured = smem;
    }
    return launch_pdl(k_nnsel_multi, dim3((a.n_items + kNnG - 1) / kNnG), dim3(kNnThreads),
                      smem, st, pdl, a);
  }
  return launch_pdl(k_nnsel, dim3(a.n_items), dim3(kNnThreads), 0, st, pdl, a);
}

cudaError_t launch_records_from_counts(const WaveArgs& a, const uint8_t* counts,
                                      int32_t* type_out, cudaStream_t st) {
  k_records_from_counts<<<a.n_items, 256, 0, st>>>(a, counts, type_out);
  return cudaGetLastError();
}

cudaError_t launch_inputs(const WaveArgs& a, int what, const uint8_t* counts, const int32_t* cand,
                          int32_t* type, int n, float* out, cudaStream_t st) {
  for (int i0 = 0; i0 < n; i0 += 65535) {
    const int c = std::min(65535, n - i0);
    const int nc = a.ti.F * a.ti.Tj * a.ti.Tj;
    k_inputs<<<c, 128, 0, st>>>(a, what, counts ? counts + (int64_t)i0 * nc : nullptr,
                                cand ? cand + i0 : nullptr, type ? type + i0 : nullptr, c,
                                out + (int64_t)i0 * nc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_rerank(const WaveArgs& a, bool pdl, cudaStream_t st) {
  return launch_pdl(k_rerank, dim3(a.n_items), dim3(256), 0, st, pdl, a);
}

}  // namespace ccw

extern "C" int ccw_set_nn_path(int32_t path) {
  if (path < 0 || path > 3) return CCW_EINVAL;
  ccw::g_nn_path = path;
  return CCW_OK;
}
