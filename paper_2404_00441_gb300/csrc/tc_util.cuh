// tc_util.cuh -- inline-PTX wrappers of the 5th-generation tensor-core
// (tcgen05) and bulk-copy instructions shared by the tensor-core CCF kernels.
#pragma once

#include "device_util.cuh"

namespace ccw {

// ---------------------------------------------------------------------------
// tcgen05 / bulk-copy wrappers (PTX ISA: tcgen05.*, cp.async.bulk)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: start address, leading (K direction) and
// stride (M/N direction) byte offsets between 8 x 16-byte core matrices, no
// swizzle, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = F16 or BF16, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t instr_desc(bool bf16, int M, int N) {
  return (1u << 4) | (bf16 ? (1u << 7) | (1u << 10) : 0u) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 8 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One 32-bit TMEM column of this thread's lane (completion not awaited).
__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr) {
  uint32_t v;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr));
  return v;
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


// Epilogue scan of the tensor-core CCF kernels: candidates r0 .. r0+len-1
// (len a multiple of kScanBatch) of one M-tile for item column n. Scores come from
// the shared-memory tile S (row pitch sp floats); `cand` holds (candidate
// index or -1, offset of the candidate's first cell in the fine TI) per row.
// Hard-data mismatches (Sec. 4.4) are counted for kScanBatch candidates at a
// time so that their TI loads overlap. Each key enters the thread's sorted list lst
// (K <= KL best; `worst` is its K-th entry), or the map is written. Keys
// at or above `bound` are dropped (see the caller).

// Hard-data mismatches (Sec. 4.4) of one M-tile's 128 candidates for the
// items in columns c0 .. c0+ntc-1, into the uint16 tile Mt[row][column]
// (pitch spm): each warp takes items in turn, its lanes take candidates, so
// the TI loads of a warp are consecutive cells (coalesced).
__device__ __forceinline__ void mismatch_tile(const WaveArgs& a, const int4* meta, int ntile,
                                              int nt, int c0, int ntc, const int2* cand,
                                              uint16_t* Mt, int spm) {
  const TiDev& t = a.ti;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int2 cr[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) cr[i] = cand[lane + 32 * i];
  for (int nl = warp; nl < ntc; nl += nw) {
    const int4 q = meta[c0 + nl];
    if (!q.w || q.z == 0) continue;
    const int2* hd = reinterpret_cast<const int2*>(
        a.ev.base + (int64_t)(ntile * nt + c0 + nl) * a.ev.stride + a.ev.hd_off);
    int mv[4] = {0, 0, 0, 0};
#pragma unroll 1
    for (int k = 0; k < q.z; ++k) {
      const int2 e = __ldg(hd + k);
      const uint8_t code = (uint8_t)(e.y & 0xFF);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (cr[i].x >= 0) mv[i] += (__ldg(t.ti + cr[i].y + e.x) != code);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) Mt[(lane + 32 * i) * spm + nl] = (uint16_t)min(mv[i], 0xFFFF);
  }
}

// The same count for the items of a chunk whose hard-data lists were first
// staged in shared memory (item nl's list at hs + hoff[nl], meta[nl].z
// entries): each lane keeps 4 candidates, and 4 hard data at a time put 16
// TI loads in flight, none of them waiting on a global load of the list.
__device__ __forceinline__ void mismatch_tile_staged(const TiDev& t, const int4* meta, int ntc,
                                                     const int* hoff, const int2* hs,
                                                     const int2* cand, uint16_t* Mt, int spm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int2 cr[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) cr[i] = cand[lane + 32 * i];
  for (int nl = warp; nl < ntc; nl += nw) {
    const int4 q = meta[nl];
    if (!q.w || q.z == 0) continue;
    const int2* hd = hs + hoff[nl];
    int mv[4] = {0, 0, 0, 0};
    int k = 0;
#pragma unroll 1
    for (; k + 4 <= q.z; k += 4) {
      int2 e[4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) e[kk] = hd[k + kk];
      uint8_t v[4][4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          v[kk][i] = cr[i].x >= 0 ? __ldg(t.ti + cr[i].y + e[kk].x) : (uint8_t)(e[kk].y & 0xFF);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int i = 0; i < 4; ++i) mv[i] += v[kk][i] != (uint8_t)(e[kk].y & 0xFF);
    }
#pragma unroll 1
    for (; k < q.z; ++k) {
      const int2 e = hd[k];
      const uint8_t code = (uint8_t)(e.y & 0xFF);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (cr[i].x >= 0) mv[i] += (__ldg(t.ti + cr[i].y + e.x) != code);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) Mt[(lane + 32 * i) * spm + nl] = (uint16_t)min(mv[i], 0xFFFF);
  }
}

// Stages the hard-data lists of the chunk's items (columns c0 .. c0+ntc-1 of
// N-tile ntile) in shared memory: hoff[nl] = first entry of item nl in hs.
// Returns false (nothing staged) when they hold more than cap entries.
// Needs a barrier before hs is read.
__device__ __forceinline__ bool stage_hard_data(const WaveArgs& a, const int4* meta, int ntile,
                                                int nt, int c0, int ntc, int* hoff, int2* hs,
                                                int cap) {
  int total = 0;
  for (int i = 0; i < ntc; ++i) total += meta[c0 + i].w ? meta[c0 + i].z : 0;
  if (total > cap) return false;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((int)threadIdx.x < ntc) {
    int off = 0;
    for (int i = 0; i < (int)threadIdx.x; ++i) off += meta[c0 + i].w ? meta[c0 + i].z : 0;
    hoff[threadIdx.x] = off;
  }
  for (int nl = warp; nl < ntc; nl += nw) {
    const int4 q = meta[c0 + nl];
    if (!q.w || q.z == 0) continue;
    int off = 0;
    for (int i = 0; i < nl; ++i) off += meta[c0 + i].w ? meta[c0 + i].z : 0;
    const int2* src = reinterpret_cast<const int2*>(
        a.ev.base + (int64_t)(ntile * nt + c0 + nl) * a.ev.stride + a.ev.hd_off);
    for (int k = lane; k < q.z; k += 32) hs[off + k] = __ldg(src + k);
  }
  return true;
}

constexpr int kScanBatch = 4;

template <int MODE, int KL>
__device__ __forceinline__ void scan_segment(const WaveArgs& a, const float* S, int sp, int n,
                                             const int2* cand, int r0, int len, int4 mt4,
                                             const int2* hdl, int64_t item, int K,
                                             uint64_t (&lst)[KL], uint64_t& worst,
                                             const uint16_t* Mt = nullptr, int spm = 0,
                                             uint64_t bound = ~0ull) {
  const TiDev& t = a.ti;
#pragma unroll 1
  for (int rb = r0; rb < r0 + len; rb += kScanBatch) {
    int2 ci[kScanBatch];
    int mis[kScanBatch];
#pragma unroll
    for (int u = 0; u < kScanBatch; ++u) {
      ci[u] = cand[rb + u];
      mis[u] = (Mt && mt4.z) ? Mt[(rb + u) * spm + n] : 0;   // counted beforehand
    }
#pragma unroll 1
    for (int k = 0; k < (Mt ? 0 : mt4.z); ++k) {
      const int2 e = __ldg(hdl + k);
      const uint8_t code = (uint8_t)(e.y & 0xFF);
#pragma unroll
      for (int u = 0; u < kScanBatch; ++u)
        if (ci[u].x >= 0) mis[u] += (__ldg(t.ti + ci[u].y + e.x) != code);
    }
#pragma unroll
    for (int u = 0; u < kScanBatch; ++u) {
      if (ci[u].x < 0) continue;
      const int score = __float2int_rn(S[(rb + u) * sp + n]) + mt4.y;
      if (MODE == kModeMap) {
        a.map_score[item * t.P + ci[u].x] = mt4.x ? score : 0;
        if (a.map_mis) a.map_mis[item * t.P + ci[u].x] = mt4.x ? mis[u] : 0;
        continue;
      }
      const uint64_t key = make_key(mis[u], score, ci[u].x);
      // `bound`: a key above the K-th best of another thread's list for
      // this item can never be among the item's K best
      if (key < worst && key < bound) {
        if (K == 1) {
          lst[0] = key;
          worst = key;
        } else {
          uint64_t x = key;
#pragma unroll
          for (int i = 0; i < KL; ++i) {
            const uint64_t lo = lst[i] < x ? lst[i] : x;
            x = lst[i] < x ? x : lst[i];
            lst[i] = lo;
          }
          worst = lst[0];
#pragma unroll
          for (int i = 1; i < KL; ++i)
            if (i < K) worst = lst[i];
        }
      }
    }
  }
}

}  // namespace ccw
