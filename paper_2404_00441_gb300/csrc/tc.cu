// tc.cu -- phase B of a search step on the 5th-generation tensor cores
// (tcgen05, sm_103a): the masked cross-correlation of Eq. CCW (Algorithm 1,
// line 10) of a batch of data events as one contraction
//     S[c, n] = sum_k A[c, k] B[n, k],
// c over candidates, n over the data events (items) of the step, k over
// (channel, template row, tap). FP16 or BF16 operands, FP32 accumulation in
// tensor memory; exact because every operand is an integer within the
// format's exact range and every partial sum is an integer below 2^24 (both
// checked on the host).
//
// Layout (2D). The candidate positions of the level-J TI are read as a line
// of pitch px8 (a multiple of 8): position L = x + px8 y. For the 128
// positions L0..L0+127 of one M-tile, template row ky and taps kx in
// [16 k16, 16 k16 + 16), A[m, kx] = plane[L0 + m + ky px8 + kx]. With the
// 8-shift copy z8[q][r][e] = plane[8q + r + e] prepared with the TI, the
// 8 x 8 core matrix (m-group i, k-group j) of that tile is z8[q0 + i + j] with
// q0 = (L0 + ky px8)/8 + 2 k16: a no-swizzle K-major operand whose core
// matrices are 128 bytes apart along both M and K. One bulk copy per channel
// brings every core matrix a CTA needs into shared memory. B (the items'
// weights) is written by the event kernel directly in the canonical K-major
// layout and arrives with one more bulk copy.
//
// Each CTA owns mt (<= 4) consecutive M-tiles and one N-tile of nt items.
// The accumulators of its M-tiles (128 lanes x nt columns of FP32 each) live
// side by side in tensor memory. Two epilogues turn the scores into ranking
// keys with the hard-data mismatches and keep the K best per item: (a) for
// K <= 8, each M-tile's scores move through a shared-memory tile and thread
// (item, segment) keeps its item's K best in registers (scan_segment); (b)
// otherwise, or on request, each of 8 warps reads one lane quarter (a
// candidate per lane and M-tile) and every other item and selects with warp
// shuffles. The CTA merges the partial lists into one K-list per item.
#include "tc_util.cuh"

namespace ccw {

constexpr int kTcThreads = 256;   // 8 warps: TMEM lane quarter w % 4, item parity w / 4
constexpr int kTcRegK = 8;        // K up to this keeps per-thread lists in registers

struct TcSmem {
  int bar_off, meta_off, list_off, a_off, b_off, s_off, c_off, bytes;
};

__host__ __device__ inline TcSmem tc_smem(int nch, int a_nq, int ksteps, int nt, int K,
                                          int lane_epi) {
  TcSmem L;
  int off = 0;
  L.bar_off = off;
  off += 128;
  L.meta_off = off;               // per item: known, const, n_hd, active
  off += ((nt * 16 + 127) / 128) * 128;
  L.list_off = off;               // [8 warps][nt][K] best keys of each warp
  off += ((8 * nt * K * 8 + 127) / 128) * 128;
  L.a_off = off;
  off += nch * a_nq * 128;
  L.b_off = off;
  off += ksteps * 32 * nt;
  L.s_off = L.c_off = off;
  if (K <= kTcRegK && !lane_epi) {
    // one M-tile of scores, [128][nt + 4] floats; later the thread lists
    off = ((off + 127) / 128) * 128;
    L.s_off = off;
    const int s_bytes = 128 * (nt + 4) * 4, l_bytes = kTcThreads * kTcRegK * 8;
    off += ((s_bytes > l_bytes ? s_bytes : l_bytes) + 127) / 128 * 128;
    L.c_off = off;   // (candidate index, TI offset) of every row of the CTA's M-tiles
    off += kTcMaxMt * 128 * 8;
  }
  L.bytes = off + 128;   // slack for aligning the dynamic shared memory base
  return L;
}

int tc_smem_bytes(int nch, int a_nq, int ksteps, int nt, int K, int lane_epi) {
  return tc_smem(nch, a_nq, ksteps, nt, K, lane_epi).bytes;
}

enum { kTcBarA = 0, kTcBarB = 1, kTcBarMma = 2 };

template <int MODE, bool BF16>
__global__ void __launch_bounds__(kTcThreads) k_ccf_tc(const __grid_constant__ WaveArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const TiDev& t = a.ti;
  const int nt = a.nt, K = a.K, nch = t.nch;
  const TcSmem L = tc_smem(nch, a.a_nq, a.ksteps, nt, K, a.tc_lane_epi);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.bar_off + 64);
  int* flag = reinterpret_cast<int*>(smem + L.bar_off + 72);
  int4* meta = reinterpret_cast<int4*>(smem + L.meta_off);
  uint64_t* lists = reinterpret_cast<uint64_t*>(smem + L.list_off);
  unsigned char* As = smem + L.a_off;
  unsigned char* Bs = smem + L.b_off;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quarter = warp & 3, parity = warp >> 2;
  const int mg = blockIdx.x, ntile = blockIdx.y;
  // the candidate geometry: the TI's decimated level-J planes, or phase
  // blockIdx.z of the all-shift candidates (block origins at phase + s u;
  // ranking index = the fine origin's index over the fine candidate grid)
  int mtiles = a.mtiles, px8 = a.px8, a_nq = a.a_nq, cd0 = t.cd[0], cd1 = t.cd[1];
  int ph0 = 0, ph1 = 0, part_base = 0;
  int64_t z8_nq = a.z8_nq;
  const void* z8v = a.z8;
  if (a.allshift) {
    const PhaseDev& ph = a.phases[blockIdx.z];
    if (mg >= ph.n_mgroups) return;   // the whole CTA, before any barrier
    mtiles = ph.mtiles;
    px8 = ph.px8;
    a_nq = ph.a_nq;
    cd0 = ph.cd0;
    cd1 = ph.cd1;
    ph0 = ph.ph0;
    ph1 = ph.ph1;
    part_base = ph.part_base;
    z8_nq = ph.z8_nq;
    z8v = a.precision == 2 ? ph.z8_bf16 : ph.z8_f16;
  }
  auto cand_index = [&](int cx, int cy) {
    return a.allshift ? (t.s * cx + ph0) + a.fd0 * (t.s * cy + ph1) : cx + cd0 * cy;
  };
  auto cand_offset = [&](int cx, int cy) {
    return (t.s * cx + ph0) + t.tp[0] * (t.s * cy + ph1);
  };
  const int64_t L_start = (int64_t)mg * a.mt * 128;
  const int n_mt = min(a.mt, mtiles - mg * a.mt);
  const int Kp = (int)((int64_t)K < t.P ? K : t.P);
  const uint32_t a_bytes = (uint32_t)a_nq * 128u;
  const uint32_t b_bytes = (uint32_t)a.ksteps * 32u * (uint32_t)nt;

  // ---- barriers and the (static) A region --------------------------------
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
    flag[0] = 0;
    mbar_arrive_expect_tx(&bar[kTcBarA], (uint32_t)nch * a_bytes);
    const unsigned char* z8 = reinterpret_cast<const unsigned char*>(z8v);
    for (int ch = 0; ch < nch; ++ch) {
      const unsigned char* src =
          z8 + ((int64_t)(t.plane0 + ch) * z8_nq + L_start / 8) * 128;
      bulk_g2s(As + (int64_t)ch * a_bytes, src, a_bytes, &bar[kTcBarA]);
    }
  }
  pdl_trigger();
  pdl_wait();   // event records and weights of this step are complete
  if (tid == 0) {
    mbar_arrive_expect_tx(&bar[kTcBarB], b_bytes);
    bulk_g2s(Bs, reinterpret_cast<const unsigned char*>(a.bmat) + (int64_t)ntile * b_bytes,
             b_bytes, &bar[kTcBarB]);
  }
  int searched = 0;   // items of this thread that need the search
  for (int i = tid; i < nt; i += kTcThreads) {
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
    searched |= m.w;
  }
  // an N-tile none of whose items needs the search (no data, or settled by
  // the learned proposal) writes nothing: its copies land and it returns
  if (!__syncthreads_or(searched)) {
    if (tid == 0 && (!mbar_wait_bounded(&bar[kTcBarA], 0u) ||
                     !mbar_wait_bounded(&bar[kTcBarB], 0u)) && a.status)
      atomicOr(a.status, kStatusTimeout);
    return;
  }
  unsigned long long* work = (MODE == kModeSim) ? a.call->work : a.work;
  if (work && mg == 0 && blockIdx.z == 0 && MODE != kModeMap) {
    // profiling: candidate evaluations and algorithmic multiply-adds (data
    // cells of the template times channels) of every item, counted once
    for (int i = tid; i < nt; i += kTcThreads) {
      const int item = ntile * nt + i;
      if (item >= a.n_items) continue;
      const int* em = reinterpret_cast<const int*>(a.ev.base + (int64_t)item * a.ev.stride);
      if (em[kEvKnown] <= 0 || em[kEvResolved]) continue;
      atomicAdd(&work[0], (unsigned long long)t.P);
      atomicAdd(&work[1], (unsigned long long)t.P * em[kEvMaskCells] * nch);
    }
  }
  // TMEM: one nt-column accumulator per M-tile
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(a.mt * nt)) ncols <<= 1;
  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // ---- MMAs of every M-tile, one commit ------------------------------------
  if (tid == 0) {
    if (!mbar_wait_bounded(&bar[kTcBarA], 0u) || !mbar_wait_bounded(&bar[kTcBarB], 0u)) {
      flag[0] = 1;
    } else {
      tc_fence_after();
      // K steps (channel, template row, 16 taps) in order, the M-tiles'
      // independent accumulators taking turns so that consecutive MMAs do
      // not wait on each other's accumulation; addresses advance by constants
      const uint32_t idesc = instr_desc(BF16, 128, nt);
      const int k16n = a.ks / 16;
      const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
      const uint32_t b_step = 32u * (uint32_t)nt, row_bytes = (uint32_t)px8 * 16u;
      uint32_t kidx = 0, b_addr = b_base;
      for (int ch = 0; ch < nch; ++ch) {
        uint32_t a_row = a_base + (uint32_t)ch * a_bytes;
        for (int row = 0; row < t.rows; ++row, a_row += row_bytes)
          for (int k16 = 0; k16 < k16n; ++k16, ++kidx, b_addr += b_step) {
            const uint64_t bd = smem_desc(b_addr, 128u, 256u);
            for (int j = 0; j < n_mt; ++j) {
              const uint64_t ad =
                  smem_desc(a_row + (uint32_t)(16 * j + 2 * k16) * 128u, 128u, 128u);
              mma_f16(tmem + (uint32_t)(j * nt), ad, bd, idesc, kidx > 0 ? 1u : 0u);
            }
          }
      }
      mma_commit(&bar[kTcBarMma]);
    }
  }
  __syncthreads();
  bool failed = flag[0] != 0;
  if (!failed) {
    if (tid == 0 && !mbar_wait_bounded(&bar[kTcBarMma], 0u)) flag[0] = 1;
    __syncthreads();
    failed = flag[0] != 0;
  }

  // ---- epilogue, K <= kTcRegK: scores move from tensor memory to shared
  // memory one M-tile at a time; thread (item n, segment) then scans its
  // item's column over a segment of candidates, turning scores into ranking
  // keys (with the hard-data mismatches) and keeping its K best in
  // registers; the segment lists of each item merge into the CTA's list.
  const bool reg_lists = MODE != kModeMap && K <= kTcRegK && !a.tc_lane_epi;
  if (!failed && reg_lists) {
    mbar_try_wait(&bar[kTcBarMma], 0u);
    tc_fence_after();
    float* S = reinterpret_cast<float*>(smem + L.s_off);
    int2* cand = reinterpret_cast<int2*>(smem + L.c_off);
    const int sp = nt + 4;
    for (int i = tid; i < n_mt * 128; i += kTcThreads) {
      const int64_t Lpos = L_start + i;
      const int cx = (int)(Lpos % px8), cy = (int)(Lpos / px8);
      const bool valid = cx < cd0 && cy < cd1;
      cand[i] = make_int2(valid ? cand_index(cx, cy) : -1, cand_offset(cx, cy));
    }
    const int n = tid % nt, nseg = kTcThreads / nt, seg = tid / nt;
    const int seg_len = 128 / nseg;
    const int4 mt4 = meta[n];
    const int item = ntile * nt + n;
    const int2* hdl = reinterpret_cast<const int2*>(
        a.ev.base + (int64_t)(item < a.n_items ? item : 0) * a.ev.stride + a.ev.hd_off);
    uint64_t lst[kTcRegK];
#pragma unroll
    for (int i = 0; i < kTcRegK; ++i) lst[i] = kNoKey;
    uint64_t worst = kNoKey;
    const int m = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const int half = nt / 2;
#pragma unroll 1
    for (int j = 0; j < n_mt; ++j) {
#pragma unroll 1
      for (int c0 = parity * half; c0 < (parity + 1) * half; c0 += 8) {
        uint32_t v[8];
        tmem_ld8(lane_base + (uint32_t)(j * nt + c0), v);
        float4* dst = reinterpret_cast<float4*>(S + m * sp + c0);
        dst[0] = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]),
                             __uint_as_float(v[2]), __uint_as_float(v[3]));
        dst[1] = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]),
                             __uint_as_float(v[6]), __uint_as_float(v[7]));
      }
      __syncthreads();
      if (mt4.w && MODE != kModeMap && K == 1 && mt4.z == 0) {
        // K = 1 without hard data: the segment's best score, the first
        // (lowest index) of equal ones since candidate indices rise with
        // the rows; one key for the segment
        const int2* cj = cand + j * 128;
        float best = -3.0e38f;
        int bi = -1;
#pragma unroll 4
        for (int r = seg * seg_len; r < (seg + 1) * seg_len; ++r) {
          const float v = S[r * sp + n];
          const int ci = cj[r].x;
          if (ci >= 0 && v > best) {
            best = v;
            bi = ci;
          }
        }
        if (bi >= 0) {
          const uint64_t key = make_key(0, __float2int_rn(best) + mt4.y, bi);
          if (key < worst) {
            lst[0] = key;
            worst = key;
          }
        }
      } else if (mt4.w) {
        scan_segment<MODE, kTcRegK>(a, S, sp, n, cand + j * 128, seg * seg_len, seg_len, mt4,
                                    hdl, item, K, lst, worst);
      }
      __syncthreads();   // S is rewritten by the next M-tile
    }
    // segment lists -> shared memory (over S), then one warp per item merges
    uint64_t* seglists = reinterpret_cast<uint64_t*>(S);
#pragma unroll
    for (int i = 0; i < kTcRegK; ++i)
      if (i < K) seglists[(seg * nt + n) * kTcRegK + i] = lst[i];
    __syncthreads();
    for (int nn = warp; nn < nt; nn += 8) {
      if (!meta[nn].w) continue;
      const int item2 = ntile * nt + nn;
      unsigned long long* part = a.part + ((int64_t)item2 * a.n_parts + part_base + mg) * K;
      int head = 0;
      const bool has = lane < nseg;
      for (int r = 0; r < Kp; ++r) {
        const uint64_t mine =
            (has && head < Kp) ? seglists[(lane * nt + nn) * kTcRegK + head] : kNoKey;
        const uint64_t best = warp_min_u64(mine);
        if (has && best != kNoKey && mine == best) ++head;
        if (lane == 0) part[r] = best;
      }
    }
  }

  // ---- epilogue (maps, K > kTcRegK): lane = candidate of each M-tile, warps
  // split the items ----
  if (!failed && !reg_lists) {
    mbar_try_wait(&bar[kTcBarMma], 0u);
    tc_fence_after();
    const int m = quarter * 32 + lane;
    int cidx[kTcMaxMt];
    const uint8_t* tb[kTcMaxMt];
#pragma unroll
    for (int j = 0; j < kTcMaxMt; ++j) {
      const int64_t Lpos = L_start + 128 * j + m;
      const int cx = (int)(Lpos % px8), cy = (int)(Lpos / px8);
      const bool valid = j < n_mt && cx < cd0 && cy < cd1;
      cidx[j] = valid ? cand_index(cx, cy) : -1;
      tb[j] = t.ti + cand_offset(cx, cy);
    }
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
    for (int n = parity; n < nt; n += 2) {
      const int4 mt4 = meta[n];
      if (!mt4.w) continue;
      uint32_t v[kTcMaxMt];
#pragma unroll
      for (int j = 0; j < kTcMaxMt; ++j)
        v[j] = (j < n_mt) ? tmem_ld1(lane_base + (uint32_t)(j * nt + n)) : 0u;
      tmem_wait_ld();
      const int item = ntile * nt + n;
      const int2* hdl = reinterpret_cast<const int2*>(a.ev.base + (int64_t)item * a.ev.stride +
                                                      a.ev.hd_off);
      // hard-data mismatches of the M-tiles' candidates, loads overlapped
      int misj[kTcMaxMt];
#pragma unroll
      for (int j = 0; j < kTcMaxMt; ++j) misj[j] = 0;
#pragma unroll 1
      for (int k = 0; k < mt4.z; ++k) {
        const int2 e = __ldg(hdl + k);
        const uint8_t code = (uint8_t)(e.y & 0xFF);
#pragma unroll
        for (int j = 0; j < kTcMaxMt; ++j)
          if (cidx[j] >= 0) misj[j] += (__ldg(tb[j] + e.x) != code);
      }
      uint64_t keys[kTcMaxMt];
#pragma unroll
      for (int j = 0; j < kTcMaxMt; ++j) {
        keys[j] = kNoKey;
        if (cidx[j] < 0) continue;
        const int score = __float2int_rn(__uint_as_float(v[j])) + mt4.y;
        const int mis = misj[j];
        if (MODE == kModeMap) {
          a.map_score[(int64_t)item * t.P + cidx[j]] = mt4.x ? score : 0;
          if (a.map_mis) a.map_mis[(int64_t)item * t.P + cidx[j]] = mt4.x ? mis : 0;
        } else {
          keys[j] = make_key(mis, score, cidx[j]);
        }
      }
      if (MODE == kModeMap) continue;
      // the K best of this warp's 32 x n_mt candidates
      uint64_t* lst = lists + ((int64_t)warp * nt + n) * K;
      uint64_t prev = 0;
#pragma unroll 1
      for (int r = 0; r < Kp; ++r) {
        uint64_t best = kNoKey;
#pragma unroll
        for (int j = 0; j < kTcMaxMt; ++j)
          if ((r == 0 || keys[j] > prev) && keys[j] < best) best = keys[j];
        best = warp_min_u64(best);
        if (lane == 0) lst[r] = best;
        prev = best;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (!failed && !reg_lists && MODE != kModeMap) {
    // merge the lists of the 4 warps that saw each item into the CTA's list
    for (int n = warp; n < nt; n += 8) {
      if (!meta[n].w) continue;
      const int item = ntile * nt + n;
      const int p = n & 1;   // the warps of parity p handled item n
      unsigned long long* part = a.part + ((int64_t)item * a.n_parts + part_base + mg) * K;
      uint64_t prev = 0;
      for (int r = 0; r < Kp; ++r) {
        uint64_t best = kNoKey;
        for (int e = lane; e < 4 * Kp; e += 32) {
          const int w = 4 * p + e / Kp;
          const uint64_t val = lists[((int64_t)w * nt + n) * K + (e % Kp)];
          if ((r == 0 || val > prev) && val < best) best = val;
        }
        best = warp_min_u64(best);
        if (lane == 0) part[r] = best;
        prev = best;
      }
    }
  }
  if (failed && tid == 0) {
    atomicOr(a.status, kStatusTimeout);
    // let the copies and MMAs in flight finish before the CTA exits
    mbar_wait_bounded(&bar[kTcBarA], 0u);
    mbar_wait_bounded(&bar[kTcBarB], 0u);
    mbar_wait_bounded(&bar[kTcBarMma], 0u);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

template <int MODE, bool BF16>
static cudaError_t launch_t(const WaveArgs& a, int smem, bool pdl, cudaStream_t st) {
  auto fn = k_ccf_tc<MODE, BF16>;
  static int configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  dim3 grid(a.n_mgroups, (a.n_items + a.nt - 1) / a.nt, a.allshift ? a.n_phases : 1);
  return launch_pdl(fn, grid, dim3(kTcThreads), smem, st, pdl, a);
}

cudaError_t launch_ccf_tc(int mode, const WaveArgs& a, int smem, bool pdl, cudaStream_t st) {
  const bool bf = a.precision == 2;
  if (mode == kModeSim)
    return bf ? launch_t<kModeSim, true>(a, smem, pdl, st) : launch_t<kModeSim, false>(a, smem, pdl, st);
  if (mode == kModeSearch)
    return bf ? launch_t<kModeSearch, true>(a, smem, pdl, st)
              : launch_t<kModeSearch, false>(a, smem, pdl, st);
  return bf ? launch_t<kModeMap, true>(a, smem, pdl, st) : launch_t<kModeMap, false>(a, smem, pdl, st);
}

}  // namespace ccw
