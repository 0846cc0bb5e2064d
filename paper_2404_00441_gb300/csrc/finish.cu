// finish.cu -- phase C of a search step: for every item, merge the per-tile
// top-K keys into the item's K best candidates (Algorithm 1, line 11), draw
// one with Philox (line 12), write the outputs or the patch log and, when
// simulating, paste the Inverse-DWT of the drawn candidate (lines 13-14).
// One CTA per item; items whose data event was empty were finished by the
// event kernel.
#include "device_util.cuh"

namespace ccw {

// Minimum over the CTA, broadcast to every thread.
__device__ __forceinline__ uint64_t block_min_u64(uint64_t v, uint64_t* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_min_u64(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = (lane < nw) ? red[lane] : kNoKey;
    w = warp_min_u64(w);
    if (lane == 0) red[kWarps] = w;
  }
  __syncthreads();
  const uint64_t r = red[kWarps];
  return r;
}

constexpr int kKeysPerThread = 8;

// Shared-memory bytes of the boundary-cut paste behind the staged
// coefficients: the pattern (T^2 bytes), the 0/1 costs and the predecessor
// columns of the two strips (2 x T x O bytes each) and the two cuts (2 x T
// int16).
__host__ __device__ inline int cut_smem_bytes(int T, int O) {
  return ((T * T + 15) & ~15) + 4 * T * O + 4 * T;
}

// Minimum-error cut of one strip (rows i = 0..T-1, columns j < O <= 64; the
// 0/1 cost of a cell in bit 0 of err) by one warp: lane l holds the
// cumulative costs of columns l and l + 32 in registers,
//   E(0, j) = err(0, j),  E(i, j) = err(i, j) + min_{|j' - j| <= 1} E(i - 1, j'),
// and records for every cell the predecessor column that attains the min
// (the lowest on ties). Lane 0 then starts at the cheapest column of the
// last row (the lowest on ties) and follows the predecessors up; the result
// is the same path as tracing back through E itself.
__device__ void strip_cut(const uint8_t* err, uint8_t* pred, int T, int O, int16_t* cut) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  constexpr int kBig = 1 << 20;
  const int j0 = lane, j1 = lane + 32;
  int e0 = kBig, e1 = kBig;   // E of the previous row (kBig beyond the strip)
  for (int i = 0; i < T; ++i) {
    const int up0 = __shfl_up_sync(full, e0, 1), up1 = __shfl_up_sync(full, e1, 1);
    const int dn0 = __shfl_down_sync(full, e0, 1), dn1 = __shfl_down_sync(full, e1, 1);
    const int last0 = __shfl_sync(full, e0, 31), first1 = __shfl_sync(full, e1, 0);
    if (i == 0) {
      if (j0 < O) e0 = err[j0] & 1;
      if (j1 < O) e1 = err[j1] & 1;
      continue;
    }
    // neighbours in column order: left (j - 1), self, right (j + 1)
    const int l0 = lane > 0 ? up0 : kBig, r0 = lane < 31 ? dn0 : first1;
    const int l1 = lane > 0 ? up1 : last0, r1 = lane < 31 ? dn1 : kBig;
    int m0 = l0, p0 = j0 - 1;
    if (e0 < m0) { m0 = e0; p0 = j0; }
    if (r0 < m0) { m0 = r0; p0 = j0 + 1; }
    int m1 = l1, p1 = j1 - 1;
    if (e1 < m1) { m1 = e1; p1 = j1; }
    if (r1 < m1) { m1 = r1; p1 = j1 + 1; }
    if (j0 < O) {
      e0 = (err[i * O + j0] & 1) + m0;
      pred[i * O + j0] = (uint8_t)p0;
    }
    if (j1 < O) {
      e1 = (err[i * O + j1] & 1) + m1;
      pred[i * O + j1] = (uint8_t)p1;
    }
  }
  // cheapest column of the last row, lowest on ties: (E, column) minimum
  int bv = j0 < O ? e0 : kBig, bj = j0;
  if (j1 < O && e1 < bv) { bv = e1; bj = j1; }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const int ov = __shfl_xor_sync(full, bv, d), oj = __shfl_xor_sync(full, bj, d);
    if (ov < bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
  }
  __syncwarp();
  if (lane == 0) {
    int c = bj;
    cut[T - 1] = (int16_t)c;
    for (int i = T - 1; i > 0; --i) {
      c = pred[i * O + c];
      cut[i - 1] = (int16_t)c;
    }
  }
}

// Paste of a 2D pattern through the minimum-error boundary cuts of image
// quilting (Efros and Freeman; the IQ method reviewed in Sec. 2). `pat` holds
// the pattern (T x T, x fastest) in shared memory. In the path frame (x', y')
// = window offsets mirrored along the axes the path runs backwards, the cost
// of a cell is 1 where the grid already holds a value that differs from the
// pattern. The column cut runs through the left strip (rows y', columns
// x' < O; warp 0), the row cut through the top strip (rows x', columns
// y' < O; warp 1). A simulated cell then takes the pattern only on the far
// side of both cuts; cells never simulated always take it.
__device__ void quilt_paste(const PasteGeom& g, const uint8_t* pat, int T, int O, uint32_t flips,
                            unsigned char* work, int nth) {
  uint8_t* errv = work;
  uint8_t* errh = errv + T * O;
  uint8_t* predv = errh + T * O;
  uint8_t* predh = predv + T * O;
  int16_t* cv = reinterpret_cast<int16_t*>(predh + T * O);   // 4 T O bytes: even
  int16_t* ch = cv + T;
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool fx = flips & 1u, fy = flips & 2u;
  // costs of both strips, every thread (row i runs along the strip): bit 0
  // = the grid holds a value that differs from the pattern, bit 1 = the
  // grid holds a value
#pragma unroll 4
  for (int k = tid; k < 2 * T * O; k += nth) {
    const int strip = k / (T * O), r = k - strip * T * O;
    const int i = r / O, j = r - i * O;
    const int xp = strip == 0 ? j : i, yp = strip == 0 ? i : j;
    const int qx = fx ? T - 1 - xp : xp, qy = fy ? T - 1 - yp : yp;
    const uint8_t old = g.grid[(g.o[0] + qx) + (int64_t)g.g[0] * (g.o[1] + qy)];
    (strip == 0 ? errv : errh)[r] =
        old == CCW_UNKNOWN ? 0 : (old != pat[qx + T * qy] ? 3 : 2);
  }
  __syncthreads();
  if (warp == 0) strip_cut(errv, predv, T, O, cv);
  else if (warp == 1) strip_cut(errh, predh, T, O, ch);
  __syncthreads();
  // the paste, 4 cells per thread: a cell keeps the grid's value when it
  // lies in a strip, holds a value and is on the near side of a cut (the
  // strips' flags say which cells hold a value, so the grid is not read)
  const bool aligned = (T & 3) == 0 && (g.o[0] & 3) == 0 && (g.g[0] & 3) == 0;
  const int T4 = (T + 3) >> 2;
  for (int w = tid; w < T * T4; w += nth) {
    const int qy = w / T4, qx0 = (w - qy * T4) * 4;
    const int yp = fy ? T - 1 - qy : qy;
    unsigned keep = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int qx = qx0 + c;
      if (qx >= T) {
        keep |= 1u << c;   // beyond the window (T not a multiple of 4)
        continue;
      }
      const int xp = fx ? T - 1 - qx : qx;
      if (xp >= O && yp >= O) continue;
      const uint8_t f = xp < O ? errv[yp * O + xp] : errh[xp * O + yp];
      if ((f & 2) && !(xp >= cv[yp] && yp >= ch[xp])) keep |= 1u << c;
    }
    uint8_t* row = g.grid + (g.o[0] + qx0) + (int64_t)g.g[0] * (g.o[1] + qy);
    if (aligned && keep == 0) {
      *reinterpret_cast<uint32_t*>(row) = *reinterpret_cast<const uint32_t*>(pat + qx0 + T * qy);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (!((keep >> c) & 1u)) row[c] = pat[qx0 + c + T * qy];
    }
  }
}

// Paste variants, each its own instantiation so that the common one carries
// no code of the others (the kernel is bound by instruction fetch).
enum : int { kPasteBlocks = 0, kPasteCut = 1, kPasteCrop = 2 };

template <int D, int MODE, int PV>
__global__ void __launch_bounds__(kThreads) k_finish(const __grid_constant__ WaveArgs a,
                                                     int staged_bytes) {
  __shared__ uint64_t red[2][kWarps + 1];
  __shared__ uint64_t topk[CCW_MAX_TOPK];
  __shared__ uint64_t sel_sh;
  extern __shared__ __align__(16) int16_t staged[];
  const TiDev& t = a.ti;
  const int tid = threadIdx.x;
  const int nth = blockDim.x;   // a multiple of 32, at most kThreads
  const int item = blockIdx.x;
  pdl_trigger();
  pdl_wait();   // the per-tile keys of this step are complete
  const int* em = reinterpret_cast<const int*>(a.ev.base + (int64_t)item * a.ev.stride);
  if (em[kEvKnown] == 0) return;
  const int K = a.K;
  const int Kp = (int)((int64_t)K < t.P ? K : t.P);
  const unsigned long long* all = a.part + (int64_t)item * a.n_parts * K;
  const int M = a.n_parts * K;
  // keys of this thread (slots >= Kp of a tile are unused)
  uint64_t mine[kKeysPerThread];
  const bool in_regs = M <= kKeysPerThread * nth;
#pragma unroll
  for (int i = 0; i < kKeysPerThread; ++i) {
    const int j = tid + i * nth;
    mine[i] = (in_regs && j < M && (j % K) < Kp) ? all[j] : kNoKey;
  }
  uint64_t prev = 0;
  for (int r = 0; r < Kp; ++r) {
    uint64_t m = kNoKey;
    if (in_regs) {
#pragma unroll
      for (int i = 0; i < kKeysPerThread; ++i)
        if ((r == 0 || mine[i] > prev) && mine[i] < m) m = mine[i];
    } else {
      for (int j = tid; j < M; j += nth) {
        if ((j % K) >= Kp) continue;
        const uint64_t v = all[j];
        if ((r == 0 || v > prev) && v < m) m = v;
      }
    }
    m = block_min_u64(m, red[r & 1]);   // alternate buffers: no reuse race
    if (tid == 0) topk[r] = m;
    prev = m;
  }
  __syncthreads();
  uint64_t seed;
  uint32_t cr, cp;
  ItemPos it;
  if (MODE == kModeSim) {
    it = decode_sim_item<D>(a, item);
    seed = a.call->seed;
    cr = it.r;
    cp = it.p;
  } else {
    seed = a.seed;
    cr = a.ctr[2 * item];
    cp = a.ctr[2 * item + 1];
  }
  // the Philox draw of Algorithm 1 line 12, once per item
  if (tid == 0) sel_sh = topk[(int)mul_shift(draw_word(seed, cr, cp, 0u), Kp)];
  __syncthreads();
  const uint64_t sel = sel_sh;
  const int pk = key_index(sel);
  if (MODE == kModeSearch) {
    if (tid < K) {
      const bool v = tid < Kp;
      a.topk_idx[item * K + tid] = v ? key_index(topk[tid]) : -1;
      a.topk_score[item * K + tid] = v ? key_score(topk[tid]) : 0;
      a.topk_mis[item * K + tid] = v ? key_mis(topk[tid]) : 0;
    }
    if (tid == 0) a.pick[item] = pk;
    return;
  }
  const CallDev* c = a.call;
  if (it.log && tid < c->log_stride) {
    int32_t* e = it.log;
    int val;
    if (tid == 0) val = pk;
    else if (tid == 1) val = key_score(sel);
    else if (tid == 2) val = key_mis(sel);
    else if (tid == 3) val = CCW_LOG_FLAG_DONE | (em[kEvResolved] ? CCW_LOG_FLAG_PROPOSAL : 0);
    else val = (tid - 4 < Kp) ? key_index(topk[tid - 4]) : -1;
    e[tid] = val;
  }
  const PasteGeom g = sim_paste_geom<D>(a, it);
  if (D == 2 && PV == kPasteCrop) {
    // an all-shift candidate: the TI crop at its fine origin
    paste_crop2(g, t.ti, t.tp[0], a.fd0, pk, t.T, nth, tid);
  } else if (D == 2 && PV == kPasteCut) {
    // the pattern into shared memory, then the boundary-cut paste (the
    // launch guarantees staged_bytes > 0 and the cut buffers behind it)
    unsigned char* pat = reinterpret_cast<unsigned char*>(staged) + ((staged_bytes + 15) & ~15);
    stage_blocks<D>(g, pk, t.J, staged, nth, tid);
    __syncthreads();
    PasteGeom gl = g;
    gl.grid = pat;
    gl.g[0] = t.T;
    gl.g[1] = t.T;
    gl.g[2] = 1;
    gl.o[0] = gl.o[1] = gl.o[2] = 0;
    if (t.J == 2)
      paste_blocks<D, 4>(gl, staged, nth, tid, true);
    else if (t.J == 1)
      paste_blocks<D, 2>(gl, staged, nth, tid, true);
    else
      paste_pixels<D>(gl, pk, t.J, nth, tid, staged);
    __syncthreads();
    quilt_paste(g, pat, t.T, a.Oj * t.s, it.flips, pat + ((t.T * t.T + 15) & ~15), nth);
  } else if (staged_bytes > 0) {
    stage_blocks<D>(g, pk, t.J, staged, nth, tid);
    __syncthreads();
    // block-wise inverse in registers for the common levels, else per cell
    const bool aligned = (g.o[0] % t.s) == 0 && (g.g[0] % t.s) == 0;
    if (D == 2 && t.J == 2)
      paste_blocks<D, 4>(g, staged, nth, tid, aligned);
    else if (t.J == 1)
      paste_blocks<D, 2>(g, staged, nth, tid, aligned);
    else
      paste_pixels<D>(g, pk, t.J, nth, tid, staged);
  } else {
    paste_pixels<D>(g, pk, t.J, nth, tid);
  }
  __syncthreads();
  paste_hard_data<D>(g, reinterpret_cast<const int2*>(a.ev.base + (int64_t)item * a.ev.stride +
                                                      a.ev.hd_off),
                     em[kEvNHd], t.T, nth, tid);
}

template <int D, int MODE>
static cudaError_t launch_t(const WaveArgs& a, bool pdl, cudaStream_t st) {
  // the pattern's coefficients (T^d int16) are staged in shared memory when
  // simulating, if they fit
  const int64_t tv = (D == 3) ? (int64_t)a.ti.T * a.ti.T * a.ti.T : (int64_t)a.ti.T * a.ti.T;
  const int staged = (MODE == kModeSim && tv * 2 <= 160 * 1024) ? (int)(tv * 2) : 0;
  // the boundary-cut paste (2D, T <= kMaxCutTempl, so staged > 0) keeps the
  // pattern and the cut buffers behind the coefficients
  const bool cut = D == 2 && MODE == kModeSim && a.cut && a.Oj > 0;
  const int smem =
      cut ? ((staged + 15) & ~15) + cut_smem_bytes(a.ti.T, a.Oj * a.ti.s) : staged;
  auto fn = cut ? k_finish<D, MODE, kPasteCut>
                : (D == 2 && MODE == kModeSim && a.allshift) ? k_finish<D, MODE, kPasteCrop>
                                                             : k_finish<D, MODE, kPasteBlocks>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  // one thread per level-J block of the pattern, up to kThreads
  const int nblk = (D == 3) ? a.ti.Tj * a.ti.Tj * a.ti.Tj : a.ti.Tj * a.ti.Tj;
  const int nth = std::min(kThreads, std::max(96, (nblk + 31) / 32 * 32));   // >= 4 + K log words
  return launch_pdl(fn, dim3(a.n_items), dim3(nth), smem, st, pdl, a, staged);
}

cudaError_t launch_finish(int mode, const WaveArgs& a, bool pdl, cudaStream_t st) {
  if (a.ti.d == 2)
    return mode == kModeSim ? launch_t<2, kModeSim>(a, pdl, st)
                            : launch_t<2, kModeSearch>(a, pdl, st);
  return mode == kModeSim ? launch_t<3, kModeSim>(a, pdl, st)
                          : launch_t<3, kModeSearch>(a, pdl, st);
}

}  // namespace ccw
