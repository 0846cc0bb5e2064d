// ccw_internal.cuh -- shared definitions of the CUDA library (not part of the
// public ABI; see include/ccw.h for that).
#pragma once

#include <cuda_bf16.h>
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

constexpr int kThreads = 256;     // threads per CTA (at most, for event and finish kernels)
constexpr int kWarps = kThreads / 32;
constexpr int kRx = 4;            // consecutive x-candidates per thread
constexpr int kMaxHd = 1024;      // hard data kept per template window
constexpr int kMaxCutTempl = 128; // largest template of the boundary-cut paste
constexpr int kMaxLevel2D = 4;
constexpr int kMaxLevel3D = 2;
constexpr int kTcMaxMt = 4;       // M-tiles per CTA of the tensor-core CCF
constexpr int kTilePersist = 1 << 30;   // ccf_tile flag: one cooperative kernel per call
constexpr int kMaxChunks = 32;    // 4-wide tap chunks per template row (Tj <= 128)

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

// The prepared training image as the kernels see it.
struct TiDev {
  const float* planes;  // [F planes][nc2][nc1][px] floats: counts of facies 0..F-2, code sums
  int px;               // plane row pitch (floats, multiple of 4, zero padded)
  int64_t plane_vol;    // floats per plane
  int plane0, nch;      // planes scored by the active score mode
  const uint8_t* ti;    // cropped fine TI, cell (0, 0, 0) of a copy padded by T cells
                        // of 255 on both sides of every axis (pitches tp)
  const int16_t* pyr;   // per-block Haar coefficients [ncv][sd]
  int F, J, s, sd, T, Tj, TjP, chunks, rows, d, score_mode;
  int n[3], nc[3], cd[3];
  int tp[3];            // row and plane pitches of the padded fine TI
  int64_t ncv, P;
  int tile[3];          // candidates per CTA tile along x, y, z
  int tiles[3], n_tiles;
};

// Per-item event records written by the event kernel (phase A) and read by
// the CCF kernel (phase B). Record of item i starts at base + i * stride:
//   int32 meta[16] (kEv*), uint32 rowmask[rows] (bit g: 4-wide tap chunk g
//   holds a non-zero weight in some channel), int2 hd[hd_cap] (.x: offset of
//   the hard datum in the padded fine TI relative to a candidate's first
//   cell; .y: (offset in the template window << 8) | code, or kHdVirtual |
//   code for a datum of the virtual template outside the window),
//   float w[nch][rows][TjP], uint8 counts[F][Tj^d] (facies counts of the
//   level-J blocks, saturated at 255).
// meta[kEvMaskType]: overlap strips fully known in 2D (bit 0 low x, 1 high x,
// 2 low y, 3 high y); meta[kEvResolved]: 1 when the learned proposal settled
// the item (the full CCF then skips it).
enum { kEvKnown = 0, kEvConst = 1, kEvMaskCells = 2, kEvNHd = 3, kEvMaskType = 4,
       kEvResolved = 5 };
// Hard-data record flag: the datum lies in the virtual template (non-causal
// conditioning), outside the window, so it is counted but never pasted.
constexpr int kHdVirtual = (int)0x80000000u;
struct EvDev {
  unsigned char* base;
  int64_t stride;
  int mask_off, hd_off, w_off, counts_off, hd_cap;
};

// One grid size of a simulation batch (device array, rewritten every call).
struct SimGroup {
  uint8_t* sg;             // [n_real][Gp] padded grids, 255 = not simulated
  const uint8_t* overlay;  // [G] hard data of this group, 255 = none
  int G[3], Gp[3], np[3];
  int64_t gp_vol, n_patches;
  int real_base;           // id of the group's first realization
  int32_t* log;            // [n_real][n_patches][log_stride] or NULL
  uint8_t* counts;         // [n_real][n_patches][F][Tj^d] data-event block counts or NULL
};

// Per-call values of a simulation, read from device memory so that a
// captured wave graph can be replayed with another seed or output.
struct CallDev {
  uint64_t seed;
  int path_random;
  int log_stride;
  unsigned long long* work;  // profiling counters [2] or NULL
  float gap_theta;           // learned proposal: relative gap that settles a patch
  unsigned long long* learn_stats;  // learned proposal counters [3] or NULL
};

// All-shift (polyphase) candidates: the TI's level-J planes of one phase
// (block origins at phase + s u) and their 8-shift copies for the tensor
// cores. A candidate's ranking index is its fine origin's raster index over
// the fine candidate grid.
struct PhaseDev {
  const void* z8_f16;
  const void* z8_bf16;
  int64_t z8_nq;        // core matrices per plane of the 8-shift copies
  int px8, mtiles, a_nq, n_mgroups;
  int cd0, cd1;         // candidate grid of the phase (level-J origins)
  int ph0, ph1;         // the phase (fine offset of block origins, < s)
  int part_base;        // first partial key list of the phase per item
};

struct WaveArgs {
  TiDev ti;
  EvDev ev;
  const SimGroup* groups;   // simulation mode
  int S;                    // patch stride T - OR
  const CallDev* call;      // simulation mode
  const int4* items;        // simulation: (group, realization slot, patch, 0)
  int n_items;
  int nb;                   // items per CTA in the CCF kernel
  // explicit data events (search / map)
  const uint8_t* de;
  const uint8_t* hd;
  const uint32_t* ctr;
  uint64_t seed;
  // tensor-core path (precision 1: FP16, 2: BF16)
  int precision;
  const void* z8;           // [F planes][z8_nq][8][8] 16-bit 8-shift view of the planes
  int64_t z8_nq;            // core matrices per plane
  int px8;                  // line pitch of the planes (multiple of 8)
  int ks;                   // taps per template row padded to a multiple of 16
  int ksteps;               // K steps of 16 taps: nch * rows * ks / 16
  int mtiles;               // 128-position M-tiles over the candidate lines
  int mt;                   // M-tiles per CTA
  int n_mgroups;            // CTAs along M
  int nt;                   // items per N-tile
  int a_nq;                 // core matrices of one channel's A region per CTA
  int tc_lane_epi;          // 1: epilogue with lanes on candidates (else per-thread lists)
  int tcs_stages;           // shared-memory stages of the streamed tensor-core kernel
  int tcs_rows;             // template rows ky per stage of the streamed kernel
  void* bmat;               // [N-tiles][ksteps][nt/8][2][8][8] 16-bit weights
  // selection
  int K;
  int n_parts;              // per-item partial lists written by the CCF kernel
  unsigned long long* part;     // [n_items][n_parts][K] partial ranking keys
  // outputs
  int32_t* topk_idx;
  int32_t* topk_score;
  int32_t* topk_mis;
  int32_t* pick;
  int32_t* map_score;
  int32_t* map_mis;
  int* status;
  unsigned long long* work;     // profiling counters for search/map mode (or NULL)
  // learned proposal (simulation mode)
  int learned;
  const float* net;         // encoder parameters (FP32)
  const void* enc_img;      // their tensor-core weight image, or NULL
  const __nv_bfloat16* tables;  // [16 mask types][P][64] unit embeddings of TI windows
  const __nv_bfloat16* tables_mma;  // the same in 128-window MMA blocks, or NULL
  float* emb;               // [n_items][64] item embeddings
  float* enc_x;             // [n_items][F][Tj^2] encoder inputs
  float* enc_act;           // encoder activations of the step's items
  int* prop;                // [n_items][n_prop] proposals
  float* prop_gap;          // [n_items] relative embedding gap of the proposals
  int n_prop;
  int fuse_rerank;          // the selector re-ranks its own proposals (no k_rerank)
  int Oj;                   // overlap in level-J blocks
  // paste and conditioning variants (simulation mode)
  int vt_ext;               // cells the virtual template extends the window forward
  int cut;                  // 1: minimum-error boundary cut at paste (2D)
  // one cooperative kernel for all wavefronts of a call (persist.cu)
  const int64_t* wave_off;  // [n_waves + 1] first item of every wavefront in `items`
  int n_waves;
  unsigned* gbar;           // [2]: grid-barrier arrivals, abort flag (zeroed per call)
  uint32_t spin_limit;      // polls of a grid-barrier wait before it gives up
  int gw;                   // threads per item in the gather and paste phases
  unsigned long long* phase_ns;  // [3] summed phase durations (profiling) or NULL
  // all-shift candidates (2D, tensor cores): CCF CTAs of phase blockIdx.z
  int allshift;
  const PhaseDev* phases;   // [n_phases] device array
  int n_phases;
  int fd0;                  // fine candidate grid width (n0 - T + 1)
};

}  // namespace ccw
