// proposal.cu -- inference of the learned proposal (not part of the paper):
// embed each data event with the encoder, propose the n_prop TI candidates
// whose embedding (under the same overlap mask type) is nearest, re-rank the
// proposals with the exact masked CCF of Eq. CCW and the hard-data
// mismatches, and settle the item when the proposals' embedding scores are
// well separated; otherwise the item falls back to the full search.
#include <algorithm>

#include "device_util.cuh"

namespace ccw {

// learned.cu
cudaError_t net_infer(const float* P, int C, int tj, const float* x, int N, float* act,
                      float* emb, cudaStream_t st);

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
// Nearest neighbours: scores s_c = table[type][c] . e over every candidate,
// the n_prop best by (score desc, index asc), and the relative gap
// (s_1 - s_nprop) / max(|s_1|, eps). A two-level histogram over [-1, 1]
// finds a threshold that keeps at least n_prop and at most kCollect
// candidates; those are ranked exactly.
// ---------------------------------------------------------------------------
constexpr int kNnThreads = 256;
constexpr int kBins = 1024;
constexpr int kCollect = 512;
constexpr int kScoreCache = 6144;   // candidates whose scores stay in shared memory

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
  if (tid < 64) e[tid] = a.emb[(int64_t)item * 64 + tid];
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
    S.e[g][i % 64] = item < a.n_items ? a.emb[(int64_t)item * 64 + i % 64] : 0.f;
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
  const int g = warp, item = i0 + g;
  const float* sc = cache + g * P;
  int* hist = S.hist[g];
  uint64_t* keys = S.keys[g];
  const int np = (int)min((int64_t)a.n_prop, t.P);
  float lo = -1.5f, hi = 1.5f;
  int above_prev = 0;
  float thr = lo;
  for (int level = 0; level < 2; ++level) {
    for (int b = lane; b < kBins; b += 32) hist[b] = 0;
    __syncwarp();
    const float scale = kBins / (hi - lo);
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
    __syncwarp();
    // the highest bin b >= 1 whose count with everything above reaches np
    // (else bin 0): lane L holds bins 32L .. 32L + 31
    int part = 0;
    for (int k = 0; k < 32; ++k) part += hist[32 * lane + k];
    int above_lanes = 0;   // bins of the lanes above this one
    for (int L = 31; L > 0; --L) {
      const int v = __shfl_sync(0xffffffffu, part, L);
      if (L > lane) above_lanes += v;
    }
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
    if (above + inbin <= kCollect || level == 1) break;
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
    return;
  }
  for (int k = ncoll + lane; k < kCollect; k += 32) keys[k] = kNoKey;
  __syncwarp();
  // bitonic sort of kCollect keys, ascending
  for (int k = 2; k <= kCollect; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < kCollect; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const uint64_t x = keys[i], y = keys[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            keys[i] = y;
            keys[l] = x;
          }
        }
      }
      __syncwarp();
    }
  for (int r = lane; r < np; r += 32)
    a.prop[(int64_t)item * a.n_prop + r] = (int)(keys[r] & 0xFFFFFFFFu);
  if (lane == 0) {
    const float s1 = nn_key_score(keys[0]), sn = nn_key_score(keys[np - 1]);
    a.prop_gap[item] = (s1 - sn) / fmaxf(fabsf(s1), 1e-6f);
  }
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
        for (int ux = 0; ux < t.Tj; ++ux) acc = fmaf(wr[ux], __ldg(pr + ux), acc);
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
cudaError_t launch_encode_items(const WaveArgs& a, float* x, float* act, bool pdl,
                                cudaStream_t st) {
  cudaError_t e = launch_pdl(k_event_inputs, dim3(a.n_items), dim3(128), 0, st, pdl, a, x);
  if (e != cudaSuccess) return e;
  return net_infer(a.net, a.ti.F, a.ti.Tj, x, a.n_items, act, a.emb, st);
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
    if ((e = net_infer(a.net, a.ti.F, a.ti.Tj, x, n, act, emb, st)) != cudaSuccess) return e;
    k_to_bf16<<<256, 256, 0, st>>>(emb, tables + ((int64_t)type * a.ti.P + c0) * 64,
                                   (int64_t)n * 64);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_nnsel(const WaveArgs& a, bool pdl, cudaStream_t st) {
  if (a.ti.P <= kScoreCache) {
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
