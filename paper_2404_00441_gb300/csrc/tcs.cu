// tcs.cu -- phase B of a search step on the tensor cores with streamed
// operands: the masked cross-correlation of Eq. CCW (Algorithm 1, line 10)
// as the contraction S[c, n] = sum_k A[c, k] B[n, k] of tc.cu, for training
// images whose Hankel view is too large to hold whole in shared memory (3D,
// where a template row is a (ky, kz) pair) and as a tiling choice in 2D.
//
// Candidate positions are read as a line L = x + px8 (y + nc1 z) of the
// level-J grid (px8 a multiple of 8). For the 128 positions L0..L0+127 of an
// M-tile, template row (ky, kz) and taps [16 k16, 16 k16 + 16):
//   A[m, kx] = plane[L0 + m + px8 (ky + nc1 kz) + 16 k16 + kx],
// whose 8 x 8 core matrices are the 17 consecutive entries q0 .. q0 + 16 of
// the 8-shift copy z8 (q0 = (L0 + px8 (ky + nc1 kz) + 16 k16) / 8). A stage
// holds one slice (channel, kz, block of R consecutive rows ky): the A
// operands of its rows, all taps and the CTA's mt M-tiles are one contiguous
// run of the 8-shift copy (one bulk copy), and the items' B tiles of its K
// steps (canonical K-major, written by the event kernel) another. A ring of 2-3 shared-memory stages
// is filled by one producer thread and drained by one MMA thread;
// tcgen05.commit on a stage's "empty" barrier hands it back. Accumulators: mt
// M-tiles x nt FP32 columns of tensor memory. Epilogue: per-thread K-lists
// (K <= 8) as in tc.cu, or the full map.
#include "tc_util.cuh"

namespace ccw {

constexpr int kTcsThreads = 256;
constexpr int kTcsMaxStages = 4;
constexpr int kTcsRegK = 8;

// Core matrices of one stage's A run: mt M-tiles, R rows of pitch px8/8,
// k16n groups of 16 taps.
__host__ __device__ inline int tcs_a_nq(int mt, int R, int px8, int k16n) {
  return 16 * (mt - 1) + (R - 1) * px8 / 8 + 2 * (k16n - 1) + 17;
}

struct TcsSmem {
  int bar_off, meta_off, stage_off, stage_bytes, b_in_stage, s_off, c_off, w_off, m_off, bytes;
};

__host__ __device__ inline TcsSmem tcs_smem(int mt, int nt, int R, int px8, int k16n,
                                            int stages) {
  TcsSmem L;
  int off = 0;
  L.bar_off = off;   // full[kTcsMaxStages], empty[...], done, TMEM slot, flags
  off += 256;
  L.meta_off = off;
  off += ((nt * 16 + 127) / 128) * 128;
  L.stage_off = off;
  L.b_in_stage = tcs_a_nq(mt, R, px8, k16n) * 128;   // a multiple of 128
  L.stage_bytes = ((L.b_in_stage + R * k16n * 32 * nt + 127) / 128) * 128;
  off += stages * L.stage_bytes;
  L.s_off = off;
  const int ntc = nt < 32 ? nt : 32;   // items per epilogue chunk
  const int s_bytes = 128 * (ntc + 4) * 4, l_bytes = kTcsThreads * kTcsRegK * 8;
  off += (((s_bytes > l_bytes ? s_bytes : l_bytes) + 127) / 128) * 128;
  L.c_off = off;
  off += kTcMaxMt * 128 * 8;
  L.w_off = off;   // the K-th best key of every thread's list [nseg][ntc]
  off += kTcsThreads * 8;
  // uint16 mismatch tile [128][ntc + 2] of the epilogue: over the stages
  // (idle once every MMA has completed) when they are large enough
  const int m_bytes = 128 * (ntc + 2) * 2;
  if (stages * L.stage_bytes >= m_bytes) {
    L.m_off = L.stage_off;
  } else {
    L.m_off = off;
    off += ((m_bytes + 127) / 128) * 128;
  }
  L.bytes = off + 128;   // slack for aligning the dynamic shared memory base
  return L;
}

int tcs_smem_bytes(int mt, int nt, int R, int px8, int k16n, int stages) {
  return tcs_smem(mt, nt, R, px8, k16n, stages).bytes;
}

template <int MODE, bool BF16>
__global__ void __launch_bounds__(kTcsThreads) k_ccf_tcs(const __grid_constant__ WaveArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const TiDev& t = a.ti;
  const int nt = a.nt, K = a.K;
  const int k16n = a.ks / 16;
  const int stages = a.tcs_stages;
  const int R = a.tcs_rows;   // template rows ky per slice
  const TcsSmem L = tcs_smem(a.mt, nt, R, a.px8, k16n, stages);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint64_t* empty = full + kTcsMaxStages;
  uint64_t* done = full + 2 * kTcsMaxStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 2 * kTcsMaxStages + 1);
  volatile int* flag = reinterpret_cast<volatile int*>(full + 2 * kTcsMaxStages + 2);
  int4* meta = reinterpret_cast<int4*>(smem + L.meta_off);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quarter = warp & 3, parity = warp >> 2;
  const int mg = blockIdx.x, ntile = blockIdx.y;
  const int64_t L_start = (int64_t)mg * a.mt * 128;
  const int n_mt = min(a.mt, a.mtiles - mg * a.mt);
  const int Kp = (int)((int64_t)K < t.P ? K : t.P);
  const uint32_t b_bytes = 32u * (uint32_t)nt;
  const int ksteps = a.ksteps;
  const int kz_n = t.rows / t.Tj;              // 1 in 2D
  const int parts = (t.Tj + R - 1) / R;        // row blocks per (channel, kz)
  const int n_slices = t.nch * kz_n * parts;   // stages of work: (channel, kz, block)

  // geometry of slice i: channel, rows r0 .. r0 + ri - 1 at kz; bytes of its
  // A run and B tiles; first core matrix of the A run; first K step
  const unsigned char* z8 = reinterpret_cast<const unsigned char*>(a.z8);
  auto slice = [&](int i, uint32_t& ab, uint32_t& bb, const unsigned char*& asrc,
                   int64_t& k0) {
    const int rb = i % parts, ck = i / parts;
    const int ch = ck / kz_n, kz = ck % kz_n;
    const int r0 = rb * R, ri = min(R, t.Tj - r0);
    ab = (uint32_t)tcs_a_nq(a.mt, ri, a.px8, k16n) * 128u;
    bb = (uint32_t)(ri * k16n) * b_bytes;
    const int64_t q0 = (L_start + (int64_t)a.px8 * ((int64_t)t.nc[1] * kz + r0)) / 8;
    asrc = z8 + ((int64_t)(t.plane0 + ch) * a.z8_nq + q0) * 128;
    k0 = ((int64_t)ch * t.rows + (int64_t)kz * t.Tj + r0) * k16n;
  };
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
    flag[0] = 0;
    // the A runs of the first slices (the TI, not this step's data) load
    // while the previous kernel finishes
    for (int i = 0; i < stages && i < n_slices; ++i) {
      uint32_t ab, bb;
      const unsigned char* asrc;
      int64_t k0;
      slice(i, ab, bb, asrc, k0);
      mbar_arrive_expect_tx(&full[i], ab + bb);
      bulk_g2s(smem + L.stage_off + i * L.stage_bytes, asrc, ab, &full[i]);
    }
  }
  pdl_trigger();
  pdl_wait();   // event records and B operands of this step are complete
  for (int i = tid; i < nt; i += kTcsThreads) {
    const int item = ntile * nt + i;
    int4 m = make_int4(0, 0, 0, 0);
    if (item < a.n_items) {
      const int* em = reinterpret_cast<const int*>(a.ev.base + (int64_t)item * a.ev.stride);
      m.x = em[kEvKnown];
      m.y = em[kEvConst];
      m.z = em[kEvNHd];
      m.w = (MODE == kModeMap) ? 1 : (m.x > 0 && !em[kEvResolved]);
    }
    meta[i] = m;
  }
  unsigned long long* work = (MODE == kModeSim) ? a.call->work : a.work;
  if (work && mg == 0 && MODE != kModeMap) {
    for (int i = tid; i < nt; i += kTcsThreads) {
      const int item = ntile * nt + i;
      if (item >= a.n_items) continue;
      const int* em = reinterpret_cast<const int*>(a.ev.base + (int64_t)item * a.ev.stride);
      if (em[kEvKnown] <= 0 || em[kEvResolved]) continue;
      atomicAdd(&work[0], (unsigned long long)t.P);
      atomicAdd(&work[1], (unsigned long long)t.P * em[kEvMaskCells] * t.nch);
    }
  }
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(a.mt * nt)) ncols <<= 1;
  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // ---- slice loop: producer (thread 0) and MMA issuer (thread 32) ---------
  if (tid == 0) {
    const unsigned char* bsrc =
        reinterpret_cast<const unsigned char*>(a.bmat) + (int64_t)ntile * ksteps * b_bytes;
    int issued = 0;
    for (int i = 0; i < n_slices; ++i) {
      const int s = i % stages;
      if (i >= stages && !mbar_wait_bounded(&empty[s], (uint32_t)(((i / stages) - 1) & 1))) {
        flag[0] = 1;
        break;
      }
      if (flag[0]) break;
      unsigned char* st = smem + L.stage_off + s * L.stage_bytes;
      uint32_t ab, bb;
      const unsigned char* asrc;
      int64_t k0;
      slice(i, ab, bb, asrc, k0);
      if (i >= stages) {   // the first slices' A runs are already on their way
        mbar_arrive_expect_tx(&full[s], ab + bb);
        bulk_g2s(st, asrc, ab, &full[s]);
      }
      bulk_g2s(st + L.b_in_stage, bsrc + k0 * b_bytes, bb, &full[s]);
      issued = i + 1;
    }
    if (flag[0]) {
      // let the copies that may still be in flight land
      for (int i = issued - stages > 0 ? issued - stages : 0; i < issued; ++i)
        mbar_wait_bounded(&full[i % stages], (uint32_t)((i / stages) & 1));
    }
  } else if (tid == 32) {
    const uint32_t idesc = instr_desc(BF16, 128, nt);
    const uint32_t base = smem_u32(smem + L.stage_off);
    const int row_q = a.px8 / 8;   // core matrices between template rows
    for (int i = 0; i < n_slices; ++i) {
      const int s = i % stages;
      if (!mbar_wait_bounded(&full[s], (uint32_t)((i / stages) & 1))) {
        flag[0] = 1;
        break;
      }
      tc_fence_after();
      const uint32_t st = base + (uint32_t)(s * L.stage_bytes);
      const int ri = min(R, t.Tj - (i % parts) * R);
      for (int ky = 0; ky < ri; ++ky)
        for (int k16 = 0; k16 < k16n; ++k16) {
          const uint64_t bd = smem_desc(
              st + (uint32_t)L.b_in_stage + (uint32_t)(ky * k16n + k16) * b_bytes, 128u, 256u);
          const uint32_t acc = (i > 0 || ky > 0 || k16 > 0) ? 1u : 0u;
          for (int j = 0; j < n_mt; ++j) {
            const uint64_t ad =
                smem_desc(st + (uint32_t)((16 * j + ky * row_q + 2 * k16) * 128), 128u, 128u);
            mma_f16(tmem + (uint32_t)(j * nt), ad, bd, idesc, acc);
          }
        }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
    if (!mbar_wait_bounded(done, 0u)) flag[0] = 1;
  }
  __syncthreads();
  const bool failed = flag[0] != 0;

  // ---- epilogue: scores of one M-tile through shared memory; thread
  // (item n, segment) keeps its item's K best keys in registers or writes
  // the map --------------------------------------------------------------
  if (!failed) {
    mbar_try_wait(done, 0u);
    tc_fence_after();
    float* S = reinterpret_cast<float*>(smem + L.s_off);
    int2* cand = reinterpret_cast<int2*>(smem + L.c_off);
    for (int i = tid; i < n_mt * 128; i += kTcsThreads) {
      const int64_t Lpos = L_start + i;
      const int cx = (int)(Lpos % a.px8);
      const int64_t rest = Lpos / a.px8;
      const int cy = (int)(rest % t.nc[1]), cz = (int)(rest / t.nc[1]);
      const bool valid = cx < t.cd[0] && cy < t.cd[1] && cz < t.cd[2];
      cand[i] = make_int2(valid ? cx + t.cd[0] * (cy + t.cd[1] * cz) : -1,
                          t.s * cx + t.tp[0] * (t.s * cy + t.tp[1] * (t.s * cz)));
    }
    __syncthreads();   // cand is read by every warp from here on
    // items in chunks of ntc columns: the score tile stays small for any nt
    const int ntc = nt < 32 ? nt : 32;
    const int spc = ntc + 4;
    const int n = tid % ntc, nseg = kTcsThreads / ntc, seg = tid / ntc;
    const int seg_len = 128 / nseg;
    const int m = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const int half = ntc / 2;
    uint64_t* seglists = reinterpret_cast<uint64_t*>(S);
    uint16_t* Mt = reinterpret_cast<uint16_t*>(smem + L.m_off);
    uint64_t* worsts = reinterpret_cast<uint64_t*>(smem + L.w_off);
#pragma unroll 1
    for (int cc = 0; cc < nt / ntc; ++cc) {
      const int col = cc * ntc + n;
      const int4 mt4 = meta[col];
      const int item = ntile * nt + col;
      const int2* hdl = reinterpret_cast<const int2*>(
          a.ev.base + (int64_t)(item < a.n_items ? item : 0) * a.ev.stride + a.ev.hd_off);
      uint64_t lst[kTcsRegK];
#pragma unroll
      for (int i = 0; i < kTcsRegK; ++i) lst[i] = kNoKey;
      uint64_t worst = kNoKey;
      // the same decision in every thread: hard data per item of the chunk
      int hd_sum = 0;
      for (int i = 0; i < ntc; ++i) hd_sum += meta[cc * ntc + i].z;
      const bool hd_tile = hd_sum >= 2 * ntc;
#pragma unroll 1
      for (int j = 0; j < n_mt; ++j) {
#pragma unroll 1
        for (int c0 = parity * half; c0 < (parity + 1) * half; c0 += 8) {
          uint32_t v[8];
          tmem_ld8(lane_base + (uint32_t)(j * nt + cc * ntc + c0), v);
          float4* dst = reinterpret_cast<float4*>(S + m * spc + c0);
          dst[0] = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]),
                               __uint_as_float(v[2]), __uint_as_float(v[3]));
          dst[1] = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]),
                               __uint_as_float(v[6]), __uint_as_float(v[7]));
        }
        // many hard data: count mismatches with coalesced loads first
        if (hd_tile) mismatch_tile(a, meta, ntile, nt, cc * ntc, ntc, cand + j * 128, Mt, ntc + 2);
        __syncthreads();
        // for K > 1: the smallest K-th best over the item's segment lists of
        // the previous M-tiles bounds the keys worth inserting (every list's
        // K-th best is at or above the item's K-th best)
        uint64_t bound = kNoKey;
        if (MODE != kModeMap && K > 1 && j > 0)
          for (int g = 0; g < nseg; ++g) {
            const uint64_t w2 = worsts[g * ntc + n];
            bound = w2 < bound ? w2 : bound;
          }
        if (mt4.w)
          scan_segment<MODE, kTcsRegK>(a, S, spc, n, cand + j * 128, seg * seg_len, seg_len,
                                       mt4, hdl, item, K, lst, worst, hd_tile ? Mt : nullptr,
                                       ntc + 2, bound);
        if (MODE != kModeMap && K > 1) worsts[seg * ntc + n] = worst;
        __syncthreads();   // S is rewritten next
      }
      if (MODE != kModeMap) {
        // segment lists of the chunk's items (over S), one warp per item merges
#pragma unroll
        for (int i = 0; i < kTcsRegK; ++i)
          if (i < K) seglists[(seg * ntc + n) * kTcsRegK + i] = lst[i];
        __syncthreads();
        for (int nn = warp; nn < ntc; nn += kTcsThreads / 32) {
          if (!meta[cc * ntc + nn].w) continue;
          const int item2 = ntile * nt + cc * ntc + nn;
          unsigned long long* part = a.part + ((int64_t)item2 * a.n_parts + mg) * K;
          int head = 0;
          const bool has = lane < nseg;
          for (int r = 0; r < Kp; ++r) {
            const uint64_t mine =
                (has && head < Kp) ? seglists[(lane * ntc + nn) * kTcsRegK + head] : kNoKey;
            const uint64_t best = warp_min_u64(mine);
            if (has && best != kNoKey && mine == best) ++head;
            if (lane == 0) part[r] = best;
          }
        }
        __syncthreads();   // the lists' space is the next chunk's score tile
      }
    }
  }
  if (failed && tid == 0) atomicOr(a.status, kStatusTimeout);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

template <int MODE, bool BF16>
static cudaError_t launch_t(const WaveArgs& a, int smem, bool pdl, cudaStream_t st) {
  auto fn = k_ccf_tcs<MODE, BF16>;
  static int configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  dim3 grid(a.n_mgroups, (a.n_items + a.nt - 1) / a.nt);
  return launch_pdl(fn, grid, dim3(kTcsThreads), smem, st, pdl, a);
}

cudaError_t launch_ccf_tcs(int mode, const WaveArgs& a, int smem, bool pdl, cudaStream_t st) {
  const bool bf = a.precision == 2;
  if (mode == kModeSim)
    return bf ? launch_t<kModeSim, true>(a, smem, pdl, st)
              : launch_t<kModeSim, false>(a, smem, pdl, st);
  if (mode == kModeSearch)
    return bf ? launch_t<kModeSearch, true>(a, smem, pdl, st)
              : launch_t<kModeSearch, false>(a, smem, pdl, st);
  return bf ? launch_t<kModeMap, true>(a, smem, pdl, st)
            : launch_t<kModeMap, false>(a, smem, pdl, st);
}

}  // namespace ccw
