// persist.cu -- every wavefront of a 2D simulation call in one cooperative
// kernel, with the masked cross-correlation of Eq. CCW on the tensor cores.
//
// The three phases of a wavefront step (Algorithm 1, lines 8-14) run inside
// one launch, separated by grid-wide barriers:
//   A  data events (lines 8-9): each item (a patch of one realization) is
//      gathered by a group of gw threads (one warp up to the whole CTA); its
//      level-J facies counts become the weights of Eq. CCW, written straight
//      into the B operand of the contraction; an empty event is drawn and
//      pasted here (lines 5-6);
//   B  the contraction S[c, n] = sum_k A[c, k] B[n, k] (line 10) of every
//      candidate c with every item n of the wavefront, tcgen05.mma kind::f16
//      into tensor memory, then hard-data mismatches and the K best ranking
//      keys of each item per CTA (line 11, Sec. 4.4);
//   C  per item: merge of the CTAs' keys, Philox draw (line 12), Inverse-DWT
//      paste and hard data (lines 13-14).
// CTA b owns the fixed M-group b mod n_mg (mt consecutive 128-candidate
// M-tiles), so its part of the TI's 8-shift copy (the A operand, the Hankel
// view of tc.cu) is copied into shared memory once per call and stays there
// for every wavefront; the CTAs sharing an M-group split the wavefront's
// N-tiles (nt items each). One CTA per SM; the grid is the SM count, launched
// cooperatively so that every CTA is resident and the barriers can complete.
// Every barrier and mbarrier wait is bounded: on expiry the kernel records
// kStatusTimeout, raises the abort flag that ends every other CTA's waits,
// waits (bounded) for its own copies and MMAs and frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_util.cuh"

namespace ccw {

constexpr int kPThreads = 256;
constexpr int kPRegK = 8;              // K <= 8: per-thread K-lists in registers
constexpr int kPCntInts = 12;          // per-item counters ahead of the block counts
constexpr int kPMinSmem = 120 * 1024;  // dynamic shared memory floor: one CTA per SM
constexpr int kPHdStage = 512;         // hard data of a chunk staged in shared memory

// ---------------------------------------------------------------------------
// Shared-memory layout (host and device)
// ---------------------------------------------------------------------------
struct PLayout {
  int bar, meta, cand, a, u;   // byte offsets; u = phase-local union region
  int grp_a, grp_c;            // per-group bytes in phases A and C
  int b, s, w, m, h;           // phase B offsets inside u
  int bytes;
};

__host__ __device__ inline int p_align(int v, int a) { return (v + a - 1) / a * a; }

__host__ __device__ inline PLayout p_layout(int nch, int a_nq, int mt, int nt, int ksteps, int F,
                                            int ncells, int T, int gw) {
  PLayout L;
  int off = 0;
  L.bar = off;   // a_full, b_full, mma_done, tmem slot, flags
  off += 256;
  L.meta = off;
  off += p_align(nt * 16, 128);
  L.cand = off;
  off += p_align(mt * 128 * 8, 128);
  L.a = off;
  off += nch * a_nq * 128;
  L.u = off;
  const int groups = kPThreads / gw;
  L.grp_a = p_align((kPCntInts + F * ncells) * 4, 16);
  const int ua = groups * L.grp_a;
  L.b = 0;
  const int ntc = nt < 32 ? nt : 32;
  L.s = p_align(ksteps * 32 * nt, 128);
  const int sb = 128 * (ntc + 4) * 4, lb = kPThreads * kPRegK * 8;
  L.w = L.s + p_align(sb > lb ? sb : lb, 128);
  L.m = L.w + kPThreads * 8;
  L.h = L.m + p_align(128 * (ntc + 2) * 2, 128);   // hd offsets [32], then entries
  const int ub = L.h + 128 + kPHdStage * 8;
  // phase C, per group: staged coefficients (T^2 int16), top-K keys, the
  // selected key, reduction slots
  L.grp_c = p_align(p_align(T * T * 2, 16) + CCW_MAX_TOPK * 8 + 8 + 16 * 8, 128);
  const int uc = groups * L.grp_c;
  int um = ua > ub ? ua : ub;
  um = um > uc ? um : uc;
  off += um;
  L.bytes = off + 128;   // slack for aligning the dynamic shared memory base
  return L;
}

int persist_smem_bytes(int nch, int a_nq, int mt, int nt, int ksteps, int F, int ncells, int T,
                       int gw) {
  const int b = p_layout(nch, a_nq, mt, nt, ksteps, F, ncells, T, gw).bytes;
  return b < kPMinSmem ? kPMinSmem : b;
}

// ---------------------------------------------------------------------------
// Grid barrier and groups
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Orders this thread's generic-proxy global writes with later async-proxy
// (bulk copy) reads of the same memory.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Waits until every CTA has arrived `target` / gridDim.x times in total.
// Returns false when this CTA's wait gave up (the abort flag is then set) or
// another CTA had given up.
__device__ bool grid_sync(const WaveArgs& a, unsigned target, volatile int* sflag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_add(&a.gbar[0], 1u);
    int ok = 0;
    for (uint32_t i = 0; i < a.spin_limit; ++i) {
      if (ld_acquire(&a.gbar[0]) >= target) {
        ok = 1;
        break;
      }
      if (ld_acquire(&a.gbar[1]) != 0u) break;
      if (i >= 64) __nanosleep(64);
    }
    if (!ok) {
      atomicExch(&a.gbar[1], 1u);
      atomicOr(a.status, kStatusTimeout);
    }
    __threadfence();
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// A group of n threads (whole warps) working on one item; named barrier id.
struct Grp {
  int lt, n, id;
  __device__ __forceinline__ void sync() const {
    if (n == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
  }
};

// Minimum over a group, broadcast to its threads (red: >= n/32 + 1 slots).
__device__ __forceinline__ uint64_t grp_min_u64(uint64_t v, const Grp& g, uint64_t* red) {
  v = warp_min_u64(v);
  if (g.n == 32) return v;
  const int w = g.lt >> 5, nw = g.n >> 5;
  if ((g.lt & 31) == 0) red[w] = v;
  g.sync();
  uint64_t r = kNoKey;
  for (int i = 0; i < nw; ++i) r = red[i] < r ? red[i] : r;
  g.sync();   // red is reused by the next call
  return r;
}

// ---------------------------------------------------------------------------
// Phase A: the data event of one item (2D, simulation)
// ---------------------------------------------------------------------------
template <bool BF16>
__device__ void p_event(const WaveArgs& a, int64_t gidx, int wi, const Grp& g, int* cnt) {
  const TiDev& t = a.ti;
  const int T = t.T, Tj = t.Tj, s = t.s;
  const int ncells = Tj * Tj;
  int* counts = cnt + kPCntInts;   // [F][Tj^2]
  unsigned char* rec = a.ev.base + (int64_t)wi * a.ev.stride;
  int* meta = reinterpret_cast<int*>(rec);
  int2* hdl = reinterpret_cast<int2*>(rec + a.ev.hd_off);
  const ItemPos it = decode_sim_item<2>(a, (int)gidx);
  const uint8_t* sg = it.sg;
  g.sync();   // the group's previous item is done with the scratch
  if (g.lt < kPCntInts) cnt[g.lt] = 0;
  g.sync();
  int my_known = 0, my_const = 0, my_mask = 0, bad = 0;
  const bool words = s == 4 && ((it.o[0] | it.Gp[0]) & 3) == 0;
  // facies counts of block u -> shared memory and this thread's sums
  // (indices into cf stay compile-time constants: cf lives in registers)
  auto account = [&](int u, const int (&cf)[8]) {
    int c = 0, last = 0;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      if (f >= t.F) break;
      counts[f * ncells + u] = cf[f];
      c += cf[f];
      last = cf[f];
    }
    if (!c) return;
    my_known += c;
    ++my_mask;
    if (t.score_mode == 0) my_const += t.sd * last;
  };
  if (words) {
    // one 32-bit word of 4 codes per block row (SWAR facies counts); the
    // rows of kNb blocks are loaded before any is counted; hard data replace
    // their bytes first
    constexpr int kNb = 4;
    for (int u0 = g.lt; u0 < ncells; u0 += kNb * g.n) {
      uint32_t vw[kNb][4];
#pragma unroll
      for (int b = 0; b < kNb; ++b) {
        const int u = u0 + b * g.n;
        if (u < ncells) {
          const int ux = u % Tj, uy = u / Tj;
          const uint8_t* r0 = sg + (it.o[0] + ux * 4) + (int64_t)it.Gp[0] * (it.o[1] + uy * 4);
#pragma unroll
          for (int cy = 0; cy < 4; ++cy)
            vw[b][cy] = *reinterpret_cast<const uint32_t*>(r0 + (int64_t)it.Gp[0] * cy);
        }
      }
#pragma unroll
      for (int b = 0; b < kNb; ++b) {
        const int u = u0 + b * g.n;
        if (u >= ncells) break;
        const int ux = u % Tj, uy = u / Tj;
        int cf[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int cy = 0; cy < 4; ++cy) {
          const int qy = uy * 4 + cy;
          const int gx0 = it.o[0] + ux * 4, gy = it.o[1] + qy;
          uint32_t v = vw[b][cy];
          if (it.overlay) {
            const int hy = gy - it.off[1];
            uint32_t hw = 0xFFFFFFFFu;
            if (hy >= 0 && hy < it.G[1]) {
              const uint8_t* orow = it.overlay + (int64_t)it.G[0] * hy;
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
                  hdl[k] = make_int2(qx + t.tp[0] * qy, ((qx + T * qy) << 8) | (int)h);
                if (h >= (uint32_t)t.F) bad |= kStatusBadCode;
              }
              const uint32_t keep = __vcmpeq4(hw, 0xFFFFFFFFu);
              v = (v & keep) | (hw & ~keep);
            }
          }
          int seen = __popc(__vcmpeq4(v, 0xFFFFFFFFu)) >> 3;
#pragma unroll
          for (int f = 0; f < 8; ++f) {
            if (f >= t.F) break;
            const int n = __popc(__vcmpeq4(v, 0x01010101u * (uint32_t)f)) >> 3;
            cf[f] += n;
            seen += n;
          }
          if (seen != 4) bad |= kStatusBadCode;
        }
        account(u, cf);
      }
    }
  } else {
    for (int u = g.lt; u < ncells; u += g.n) {
      const int ux = u % Tj, uy = u / Tj;
      int cf[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int cy = 0; cy < s; ++cy) {
        const int qy = uy * s + cy;
        for (int cx = 0; cx < s; ++cx) {
          const int qx = ux * s + cx;
          const int gx = it.o[0] + qx, gy = it.o[1] + qy;
          uint8_t h = CCW_UNKNOWN;
          if (it.overlay) {
            const int hx = gx - it.off[0], hy = gy - it.off[1];
            if (hx >= 0 && hy >= 0 && hx < it.G[0] && hy < it.G[1])
              h = __ldg(it.overlay + hx + (int64_t)it.G[0] * hy);
          }
          uint8_t v = sg[gx + (int64_t)it.Gp[0] * gy];
          if (h != CCW_UNKNOWN) {
            v = h;
            const int k = atomicAdd(&cnt[3], 1);
            if (k < a.ev.hd_cap)
              hdl[k] = make_int2(qx + t.tp[0] * qy, ((qx + T * qy) << 8) | (int)h);
            if (h >= t.F) bad |= kStatusBadCode;
          }
          if (v != CCW_UNKNOWN) {
            if (v >= t.F) bad |= kStatusBadCode;
#pragma unroll
            for (int f = 0; f < 8; ++f) cf[f] += (v == f);
          }
        }
      }
      account(u, cf);
    }
  }
  my_known = __reduce_add_sync(0xffffffffu, my_known);
  my_const = __reduce_add_sync(0xffffffffu, my_const);
  my_mask = __reduce_add_sync(0xffffffffu, my_mask);
  bad = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
  if ((g.lt & 31) == 0) {
    if (my_known) atomicAdd(&cnt[0], my_known);
    if (my_const) atomicAdd(&cnt[1], my_const);
    if (my_mask) atomicAdd(&cnt[2], my_mask);
    if (bad) atomicOr(&cnt[4], bad);
  }
  g.sync();
  if (it.counts)
    for (int i = g.lt; i < t.F * ncells; i += g.n) it.counts[i] = (uint8_t)counts[i];
  // the weights of Eq. CCW as the B operand: item wi is row wi % nt of
  // N-tile wi / nt; K step k = (ch * Tj + row) * ks/16 + k16 holds taps
  // 16 k16 .. 16 k16 + 15 of template row `row`, two 8 x 8 core matrices
  // (kc = 0, 1) in the canonical K-major layout. One-hot weights are
  // w_f = b_f - b_{F-1}; literal ones the block's code sum.
  {
    const int nt = a.nt, k16n = a.ks / 16;
    const int ntile = wi / nt, ni = wi % nt;
    unsigned char* base = reinterpret_cast<unsigned char*>(a.bmat) +
                          (int64_t)ntile * a.ksteps * 32 * nt + (ni / 8) * 256 + (ni % 8) * 16;
    const int* last = counts + (t.F - 1) * ncells;
    for (int i = g.lt; i < a.ksteps * 2; i += g.n) {
      const int k = i >> 1, kc = i & 1;
      const int k16 = k % k16n, rc = k / k16n;
      const int ch = rc / Tj, row = rc % Tj;
      uint32_t packed[4];
#pragma unroll
      for (int e2 = 0; e2 < 4; ++e2) {
        uint32_t hv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int kx = 16 * k16 + 8 * kc + 2 * e2 + h;
          float w = 0.f;
          if (kx < Tj) {
            const int u = row * Tj + kx;
            if (t.score_mode == 0) {
              w = (float)(counts[ch * ncells + u] - last[u]);
            } else {
              int cs = 0;
              for (int f = 1; f < t.F; ++f) cs += f * counts[f * ncells + u];
              w = (float)cs;
            }
          }
          hv[h] = BF16 ? (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(w))
                       : (uint32_t)__half_as_ushort(__float2half_rn(w));
        }
        packed[e2] = hv[0] | (hv[1] << 16);
      }
      *reinterpret_cast<uint4*>(base + (int64_t)k * 32 * nt + kc * 128) =
          make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
  }
  fence_proxy_async_global();   // the B operand is read by bulk copies in phase B
  const int known = cnt[0];
  if (g.lt == 0) {
    meta[kEvKnown] = known;
    meta[kEvConst] = cnt[1];
    meta[kEvMaskCells] = cnt[2];
    meta[kEvNHd] = min(cnt[3], a.ev.hd_cap);
    meta[kEvMaskType] = 0;
    meta[kEvResolved] = 0;
    const int b = cnt[4] | (cnt[3] > a.ev.hd_cap ? kStatusHdOverflow : 0);
    if (b) atomicOr(a.status, b);
  }
  if (known != 0) return;
  // empty data event: uniform draw (Algorithm 1, lines 5-6) and paste
  const CallDev* c = a.call;
  const int pk = (int)mul_shift(draw_word(c->seed, it.r, it.p, 0u), t.P);
  if (it.log && g.lt < c->log_stride) {
    const int l = g.lt;
    it.log[l] = (l == 0) ? pk
                         : (l == 3 ? (CCW_LOG_FLAG_UNIFORM | CCW_LOG_FLAG_DONE)
                                   : (l < 3 ? 0 : -1));
  }
  const PasteGeom pg = sim_paste_geom<2>(a, it);
  paste_pixels<2>(pg, pk, t.J, g.n, g.lt);
  g.sync();
  paste_hard_data<2>(pg, hdl, min(cnt[3], a.ev.hd_cap), T, g.n, g.lt);
}

// ---------------------------------------------------------------------------
// Phase C: merge, draw and paste of one item (2D, simulation)
// ---------------------------------------------------------------------------
__device__ void p_finish(const WaveArgs& a, int64_t gidx, int wi, const Grp& g,
                         unsigned char* scratch) {
  const TiDev& t = a.ti;
  const int* em = reinterpret_cast<const int*>(a.ev.base + (int64_t)wi * a.ev.stride);
  if (em[kEvKnown] == 0) return;   // finished in phase A
  int16_t* staged = reinterpret_cast<int16_t*>(scratch);
  uint64_t* topk = reinterpret_cast<uint64_t*>(scratch + p_align(t.T * t.T * 2, 16));
  uint64_t* sel_sh = topk + CCW_MAX_TOPK;
  uint64_t* red = sel_sh + 1;
  const int K = a.K;
  const int Kp = (int)((int64_t)K < t.P ? K : t.P);
  const unsigned long long* all = a.part + (int64_t)wi * a.n_parts * K;
  g.sync();   // the group's previous item is done with the scratch
  const int M = a.n_parts * K;
  // the CTAs' keys of this item: loaded once (all loads in flight together)
  // when each thread holds at most kMine of them, else read per round
  constexpr int kMine = 12;
  const bool in_regs = M <= kMine * g.n;
  uint64_t mine[kMine];
#pragma unroll
  for (int i = 0; i < kMine; ++i) {
    const int j = g.lt + i * g.n;
    mine[i] = (in_regs && j < M && (j % K) < Kp) ? all[j] : kNoKey;
  }
  uint64_t prev = 0;
  for (int r = 0; r < Kp; ++r) {
    uint64_t m = kNoKey;
    if (in_regs) {
#pragma unroll
      for (int i = 0; i < kMine; ++i)
        if ((r == 0 || mine[i] > prev) && mine[i] < m) m = mine[i];
    } else {
      for (int j = g.lt; j < M; j += g.n) {
        if ((j % K) >= Kp) continue;
        const uint64_t v = all[j];
        if ((r == 0 || v > prev) && v < m) m = v;
      }
    }
    m = grp_min_u64(m, g, red);
    if (g.lt == 0) topk[r] = m;
    prev = m;
  }
  const ItemPos it = decode_sim_item<2>(a, (int)gidx);
  const CallDev* c = a.call;
  g.sync();
  if (g.lt == 0) *sel_sh = topk[(int)mul_shift(draw_word(c->seed, it.r, it.p, 0u), Kp)];
  g.sync();
  const uint64_t sel = *sel_sh;
  const int pk = key_index(sel);
  if (it.log && g.lt < c->log_stride) {
    const int l = g.lt;
    int val;
    if (l == 0) val = pk;
    else if (l == 1) val = key_score(sel);
    else if (l == 2) val = key_mis(sel);
    else if (l == 3) val = CCW_LOG_FLAG_DONE;
    else val = (l - 4 < Kp) ? key_index(topk[l - 4]) : -1;
    it.log[l] = val;
  }
  const PasteGeom pg = sim_paste_geom<2>(a, it);
  stage_blocks<2>(pg, pk, t.J, staged, g.n, g.lt);
  g.sync();
  const bool aligned = (pg.o[0] % t.s) == 0 && (pg.g[0] % t.s) == 0;
  if (t.J == 2)
    paste_blocks<2, 4>(pg, staged, g.n, g.lt, aligned);
  else if (t.J == 1)
    paste_blocks<2, 2>(pg, staged, g.n, g.lt, aligned);
  else
    paste_pixels<2>(pg, pk, t.J, g.n, g.lt, staged);
  g.sync();
  paste_hard_data<2>(pg, reinterpret_cast<const int2*>(a.ev.base + (int64_t)wi * a.ev.stride +
                                                       a.ev.hd_off),
                     em[kEvNHd], t.T, g.n, g.lt);
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
template <bool BF16>
__global__ void __launch_bounds__(kPThreads, 1) k_persist(const __grid_constant__ WaveArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const TiDev& t = a.ti;
  const int nt = a.nt, K = a.K, nch = t.nch, mt = a.mt;
  const int ncells = t.Tj * t.Tj;
  const PLayout L = p_layout(nch, a.a_nq, mt, nt, a.ksteps, t.F, ncells, t.T, a.gw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar);
  uint64_t* a_full = bars;
  uint64_t* b_full = bars + 1;
  uint64_t* mma_done = bars + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  volatile int* flag = reinterpret_cast<volatile int*>(bars + 4);    // a wait gave up
  volatile int* sflag = reinterpret_cast<volatile int*>(bars + 5);   // grid_sync result
  int4* meta = reinterpret_cast<int4*>(smem + L.meta);
  int2* cand = reinterpret_cast<int2*>(smem + L.cand);
  unsigned char* As = smem + L.a;
  unsigned char* U = smem + L.u;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quarter = warp & 3, parity = warp >> 2;
  const int G = gridDim.x;
  const int n_mg = a.n_mgroups;
  const int my_mg = blockIdx.x % n_mg;
  const int my_rep = blockIdx.x / n_mg;
  const int reps = G / n_mg + ((my_mg < G % n_mg) ? 1 : 0);
  const int64_t L_start = (int64_t)my_mg * mt * 128;
  const int n_mt = min(mt, a.mtiles - my_mg * mt);
  const uint32_t a_bytes = (uint32_t)a.a_nq * 128u;
  const uint32_t b_bytes = (uint32_t)a.ksteps * 32u * (uint32_t)nt;
  const int Kp = (int)((int64_t)K < t.P ? K : t.P);
  const Grp grp{tid % a.gw, a.gw, 1 + tid / a.gw};
  const int n_groups = kPThreads / a.gw;
  const int ggroup = blockIdx.x * n_groups + tid / a.gw;   // this group's global index
  const int n_ggroups = G * n_groups;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
    flag[0] = 0;
    // the CTA's part of the A operand: the TI's 8-shift copy, once per call
    mbar_arrive_expect_tx(a_full, (uint32_t)nch * a_bytes);
    const unsigned char* z8 = reinterpret_cast<const unsigned char*>(a.z8);
    for (int ch = 0; ch < nch; ++ch)
      bulk_g2s(As + (int64_t)ch * a_bytes,
               z8 + ((int64_t)(t.plane0 + ch) * a.z8_nq + L_start / 8) * 128, a_bytes, a_full);
  }
  // (candidate index or -1, offset of its first fine cell in the padded TI)
  // of every row of the CTA's M-tiles: the same for every wavefront
  for (int i = tid; i < mt * 128; i += kPThreads) {
    const int64_t Lpos = L_start + i;
    const int cx = (int)(Lpos % a.px8), cy = (int)(Lpos / a.px8);
    const bool valid = i < n_mt * 128 && cx < t.cd[0] && cy < t.cd[1];
    cand[i] = make_int2(valid ? cx + t.cd[0] * cy : -1, t.s * cx + t.tp[0] * (t.s * cy));
  }
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(mt * nt)) ncols <<= 1;
  if (warp == 0) tmem_alloc(tmem_slot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  bool alive = true;
  bool a_waited = false;
  uint32_t b_uses = 0, m_uses = 0;
  int b_pending = 0, m_pending = 0;   // thread 0: a copy / MMAs not yet seen complete
  unsigned target = 0;
  unsigned long long t0 = 0, tA = 0, tB = 0, tC = 0;
  const bool timing = a.phase_ns != nullptr && blockIdx.x == 0 && tid == 0;
  unsigned long long* work = a.call->work;

  for (int w = 0; w < a.n_waves && alive; ++w) {
    const int64_t off = a.wave_off[w];
    const int n_items = (int)(a.wave_off[w + 1] - off);
    if (timing) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    // ---- phase A: data events -----------------------------------------------
    for (int wi = ggroup; wi < n_items; wi += n_ggroups)
      p_event<BF16>(a, off + wi, wi, grp, reinterpret_cast<int*>(U + (tid / a.gw) * L.grp_a));
    target += G;
    if (!grid_sync(a, target, sflag)) {
      alive = false;
      break;
    }
    if (timing) {
      unsigned long long x;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(x));
      tA += x - t0;
      t0 = x;
    }
    // ---- phase B: contraction and per-CTA K best -----------------------------
    const int n_ntiles = (n_items + nt - 1) / nt;
    unsigned char* Bs = U + L.b;
    for (int nti = my_rep; nti < n_ntiles; nti += reps) {
      for (int i = tid; i < nt; i += kPThreads) {
        const int item = nti * nt + i;
        int4 m = make_int4(0, 0, 0, 0);
        if (item < n_items) {
          const int* emr = reinterpret_cast<const int*>(a.ev.base + (int64_t)item * a.ev.stride);
          m.x = emr[kEvKnown];
          m.y = emr[kEvConst];
          m.z = emr[kEvNHd];
          m.w = m.x > 0;
          if (work && my_mg == 0 && m.w) {
            atomicAdd(&work[0], (unsigned long long)t.P);
            atomicAdd(&work[1], (unsigned long long)t.P * emr[kEvMaskCells] * nch);
          }
        }
        meta[i] = m;
      }
      const int any = __syncthreads_or(tid < nt ? meta[tid].w : 0);
      if (!any) continue;
      if (tid == 0) {
        bool ok = true;
        if (!a_waited) {
          ok = mbar_wait_bounded(a_full, 0u);
          a_waited = ok;
        }
        if (ok) {
          fence_proxy_async_global();
          mbar_arrive_expect_tx(b_full, b_bytes);
          bulk_g2s(Bs, reinterpret_cast<const unsigned char*>(a.bmat) + (int64_t)nti * b_bytes,
                   b_bytes, b_full);
          b_pending = 1;
          ok = mbar_wait_bounded(b_full, b_uses & 1u);
          if (ok) {
            b_pending = 0;
            ++b_uses;
          }
        }
        if (ok) {
          tc_fence_after();
          // K steps (channel, template row, 16 taps) in order; the M-tiles'
          // independent accumulators take turns, so consecutive MMAs never
          // wait on each other's accumulation
          const uint32_t idesc = instr_desc(BF16, 128, nt);
          const int k16n = a.ks / 16;
          const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
          const uint32_t b_step = 32u * (uint32_t)nt, row_bytes = (uint32_t)a.px8 * 16u;
          uint32_t kidx = 0, b_addr = b_base;
          for (int ch = 0; ch < nch; ++ch) {
            uint32_t a_row = a_base + (uint32_t)ch * a_bytes;
            for (int row = 0; row < t.rows; ++row, a_row += row_bytes) {
              for (int k16 = 0; k16 < k16n; ++k16, ++kidx, b_addr += b_step) {
                const uint64_t bd = smem_desc(b_addr, 128u, 256u);
                const uint32_t acc = kidx > 0 ? 1u : 0u;
                for (int j = 0; j < n_mt; ++j) {
                  const uint64_t ad =
                      smem_desc(a_row + (uint32_t)(16 * j + 2 * k16) * 128u, 128u, 128u);
                  mma_f16(tmem + (uint32_t)(j * nt), ad, bd, idesc, acc);
                }
              }
            }
          }
          mma_commit(mma_done);
          m_pending = 1;
          ok = mbar_wait_bounded(mma_done, m_uses & 1u);
          if (ok) {
            m_pending = 0;
            ++m_uses;
          }
        }
        if (!ok) {
          flag[0] = 1;
          atomicExch(&a.gbar[1], 1u);   // the other CTAs stop at their next barrier
        }
      }
      __syncthreads();
      if (flag[0]) {
        alive = false;
        break;
      }
      tc_fence_after();
      // epilogue: scores of one M-tile through shared memory, items in chunks
      // of ntc columns; thread (item n, segment) keeps its item's K best
      float* S = reinterpret_cast<float*>(U + L.s);
      uint16_t* Mt = reinterpret_cast<uint16_t*>(U + L.m);
      uint64_t* worsts = reinterpret_cast<uint64_t*>(U + L.w);
      uint64_t* seglists = reinterpret_cast<uint64_t*>(S);
      const int ntc = nt < 32 ? nt : 32;
      const int spc = ntc + 4;
      const int n = tid % ntc, nseg = kPThreads / ntc, seg = tid / ntc;
      const int seg_len = 128 / nseg;
      const int m = quarter * 32 + lane;
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
      const int half = ntc / 2;
#pragma unroll 1
      for (int cc = 0; cc < nt / ntc; ++cc) {
        const int col = cc * ntc + n;
        const int4 mt4 = meta[col];
        const int item = nti * nt + col;
        const int2* hdl = reinterpret_cast<const int2*>(
            a.ev.base + (int64_t)(item < n_items ? item : 0) * a.ev.stride + a.ev.hd_off);
        uint64_t lst[kPRegK];
#pragma unroll
        for (int i = 0; i < kPRegK; ++i) lst[i] = kNoKey;
        uint64_t worst = kNoKey;
        int hd_sum = 0, act = 0;
        for (int i = 0; i < ntc; ++i) {
          hd_sum += meta[cc * ntc + i].z;
          act |= meta[cc * ntc + i].w;
        }
        if (!act) continue;   // the same decision in every thread
        // hard-data mismatches in a separate pass per M-tile, from lists
        // staged in shared memory (or, for very many, read from the records)
        int* hoff = reinterpret_cast<int*>(U + L.h);
        int2* hs = reinterpret_cast<int2*>(U + L.h + 128);
        const bool staged = hd_sum > 0 &&
                            stage_hard_data(a, meta, nti, nt, cc * ntc, ntc, hoff, hs, kPHdStage);
        const bool hd_tile = staged || hd_sum >= 2 * ntc;
        if (staged) __syncthreads();
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
          if (staged)
            mismatch_tile_staged(t, meta + cc * ntc, ntc, hoff, hs, cand + j * 128, Mt, ntc + 2);
          else if (hd_tile)
            mismatch_tile(a, meta, nti, nt, cc * ntc, ntc, cand + j * 128, Mt, ntc + 2);
          __syncthreads();
          uint64_t bound = kNoKey;
          if (K > 1 && j > 0)
            for (int gq = 0; gq < nseg; ++gq) {
              const uint64_t w2 = worsts[gq * ntc + n];
              bound = w2 < bound ? w2 : bound;
            }
          if (mt4.w)
            scan_segment<kModeSim, kPRegK>(a, S, spc, n, cand + j * 128, seg * seg_len, seg_len,
                                           mt4, hdl, item, K, lst, worst,
                                           hd_tile ? Mt : nullptr, ntc + 2, bound);
          if (K > 1) worsts[seg * ntc + n] = worst;
          __syncthreads();   // S is rewritten next
        }
        // segment lists of the chunk's items (over S), one warp per item merges
#pragma unroll
        for (int i = 0; i < kPRegK; ++i)
          if (i < K) seglists[(seg * ntc + n) * kPRegK + i] = lst[i];
        __syncthreads();
        for (int nn = warp; nn < ntc; nn += kPThreads / 32) {
          if (!meta[cc * ntc + nn].w) continue;
          const int item2 = nti * nt + cc * ntc + nn;
          unsigned long long* part = a.part + ((int64_t)item2 * a.n_parts + my_mg) * K;
          int head = 0;
          const bool has = lane < nseg;
          for (int r = 0; r < Kp; ++r) {
            const uint64_t mine =
                (has && head < Kp) ? seglists[(lane * ntc + nn) * kPRegK + head] : kNoKey;
            const uint64_t best = warp_min_u64(mine);
            if (has && best != kNoKey && mine == best) ++head;
            if (lane == 0) part[r] = best;
          }
        }
        __syncthreads();   // the lists' space is the next chunk's score tile
      }
      tc_fence_before();   // TMEM reads done before the next tile's MMAs
    }
    if (!alive) break;
    target += G;
    if (!grid_sync(a, target, sflag)) {
      alive = false;
      break;
    }
    if (timing) {
      unsigned long long x;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(x));
      tB += x - t0;
      t0 = x;
    }
    // ---- phase C: merge, draw, paste ----------------------------------------
    for (int wi = ggroup; wi < n_items; wi += n_ggroups)
      p_finish(a, off + wi, wi, grp, U + (tid / a.gw) * L.grp_c);
    if (w + 1 < a.n_waves) {
      target += G;
      if (!grid_sync(a, target, sflag)) {
        alive = false;
        break;
      }
    }
    if (timing) {
      unsigned long long x;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(x));
      tC += x - t0;
    }
  }
  if (timing) {
    atomicAdd(&a.phase_ns[0], tA);
    atomicAdd(&a.phase_ns[1], tB);
    atomicAdd(&a.phase_ns[2], tC);
  }
  if (tid == 0) {
    if (flag[0]) atomicOr(a.status, kStatusTimeout);
    // nothing of this CTA may still be in flight when it exits
    if (!a_waited) mbar_wait_bounded(a_full, 0u);
    if (b_pending) mbar_wait_bounded(b_full, b_uses & 1u);
    if (m_pending) mbar_wait_bounded(mma_done, m_uses & 1u);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

template <bool BF16>
static cudaError_t launch_p(const WaveArgs& a, int smem, int grid, cudaStream_t st) {
  auto fn = k_persist<BF16>;
  static int configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, fn, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// CTAs of the cooperative grid: one per SM when the kernel fits one per SM.
int persist_grid(int smem, bool bf16) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  auto fn = bf16 ? k_persist<true> : k_persist<false>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPThreads, smem) != cudaSuccess)
    return 0;
  return per_sm >= 1 ? sms : 0;
}

cudaError_t launch_persist(const WaveArgs& a, int smem, int grid, cudaStream_t st) {
  return a.precision == 2 ? launch_p<true>(a, smem, grid, st) : launch_p<false>(a, smem, grid, st);
}

}  // namespace ccw
