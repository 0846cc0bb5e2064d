// ccw_internal.cuh -- shared definitions of the CUDA library (not part of the
// public ABI; see include/ccw.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ccw.h"

namespace ccw {

// Device status bits (ccw_ti_status).
enum : int {
  kStatusBadCode = 1,
  kStatusHdOverflow = 2,
  kStatusTimeout = 4,
};

constexpr int kThreads = 256;     // threads per CTA of the search kernel
constexpr int kRx = 4;            // consecutive x-candidates per thread
constexpr int kMaxHd = 1024;      // hard data kept per template window
constexpr int kMaxLevel2D = 4;
constexpr int kMaxLevel3D = 2;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): the round multiplies
// counter words 0 and 2 by two odd 32-bit constants, keeps the high and low
// halves, and mixes the high halves with the other two words and the key;
// the key advances by the Weyl increments (golden ratio, sqrt(3) - 1)
// between rounds.
// ---------------------------------------------------------------------------
struct U32x4 {
  uint32_t v[4];
};

__host__ __device__ inline U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, uint32_t k0, uint32_t k1) {
  constexpr uint32_t kMulA = 0xD2511F53u;
  constexpr uint32_t kMulB = 0xCD9E8D57u;
  constexpr uint32_t kWeylA = 0x9E3779B9u;
  constexpr uint32_t kWeylB = 0xBB67AE85u;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint64_t pa = (uint64_t)kMulA * c0;
    const uint64_t pb = (uint64_t)kMulB * c2;
    const uint32_t a_hi = (uint32_t)(pa >> 32), a_lo = (uint32_t)pa;
    const uint32_t b_hi = (uint32_t)(pb >> 32), b_lo = (uint32_t)pb;
    c0 = b_hi ^ c1 ^ k0;
    c1 = b_lo;
    c2 = a_hi ^ c3 ^ k1;
    c3 = a_lo;
    k0 += kWeylA;
    k1 += kWeylB;
  }
  U32x4 r;
  r.v[0] = c0;
  r.v[1] = c1;
  r.v[2] = c2;
  r.v[3] = c3;
  return r;
}

// First Philox word of counter (a, b, purpose, 0) under the 64-bit seed.
__host__ __device__ inline uint32_t draw_word(uint64_t seed, uint32_t a, uint32_t b,
                                              uint32_t purpose) {
  return philox4x32_10(a, b, purpose, 0u, (uint32_t)seed, (uint32_t)(seed >> 32)).v[0];
}

// floor(u * n / 2^32)
__host__ __device__ inline int64_t mul_shift(uint32_t u, int64_t n) {
  return (int64_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

// ---------------------------------------------------------------------------
// Ranking key: one 64-bit word, smaller = better, so a plain unsigned
// minimum implements (mismatch asc, score desc, index asc):
//   [63:48] mismatches (saturated), [47:24] (2^24 - 1 - score), [23:0] index.
// Valid because 0 <= score < 2^24 and P_c <= 2^24 (checked at prepare).
// ---------------------------------------------------------------------------
__host__ __device__ inline uint64_t make_key(int mis, int score, int idx) {
  const uint64_t m = (uint64_t)(mis > 0xFFFF ? 0xFFFF : mis);
  return (m << 48) | ((uint64_t)(0xFFFFFF - score) << 24) | (uint64_t)idx;
}
__host__ __device__ inline int key_index(uint64_t k) { return (int)(k & 0xFFFFFF); }
__host__ __device__ inline int key_score(uint64_t k) {
  return 0xFFFFFF - (int)((k >> 24) & 0xFFFFFF);
}
__host__ __device__ inline int key_mis(uint64_t k) { return (int)(k >> 48); }
constexpr uint64_t kNoKey = ~0ull;

// ---------------------------------------------------------------------------
// Kernel arguments.
// ---------------------------------------------------------------------------
enum Mode : int { kModeSim = 0, kModeSearch = 1, kModeMap = 2 };

struct SearchArgs {
  // training image
  const float* planes;     // nch level-J planes, each ncv floats
  const uint8_t* ti;       // cropped fine TI
  const int16_t* pyr;      // per-block Haar coefficients [ncv][s^d]
  int nch;                 // channels scored (F-1 one-hot, 1 literal)
  int F, J, s, sd, T, Tj, TjP, d, score_mode;
  int n[3], nc[3], cd[3];
  int64_t ncv, P;
  int tiles[3], n_tiles;   // candidate tiles per axis, total
  // items of this launch
  int n_items;
  const int2* items;       // sim: (realization slot, patch) pairs
  // simulation state
  uint8_t* sg;             // [n_real][Gp] padded grids, 255 = not simulated
  const uint8_t* overlay;  // [G] hard data, 255 = none
  int G[3], Gp[3], np[3], S, path_random, real_base;
  int64_t gp_vol, n_patches;
  // explicit data events
  const uint8_t* de;
  const uint8_t* hd;
  const uint32_t* ctr;
  // selection
  int K;
  uint64_t seed;
  unsigned long long* part;     // [n_items][n_tiles][K]
  unsigned int* counters;       // [n_items]
  // outputs
  int32_t* topk_idx;
  int32_t* topk_score;
  int32_t* topk_mis;
  int32_t* pick;
  int32_t* log;
  int log_stride;
  int32_t* map_score;
  int32_t* map_mis;
  int* status;
  unsigned long long* work;     // profiling: [0] candidate evals, [1] MACs (or NULL)
};

}  // namespace ccw
