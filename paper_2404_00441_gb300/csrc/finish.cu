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

template <int D, int MODE>
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
  if (staged_bytes > 0) {
    stage_blocks<D>(g, pk, t.J, staged, nth);
    __syncthreads();
    // block-wise inverse in registers for the common levels, else per cell
    const bool aligned = (g.o[0] % t.s) == 0 && (g.g[0] % t.s) == 0;
    if (D == 2 && t.J == 2)
      paste_blocks<D, 4>(g, staged, nth, aligned);
    else if (t.J == 1)
      paste_blocks<D, 2>(g, staged, nth, aligned);
    else
      paste_pixels<D>(g, pk, t.J, nth, staged);
  } else {
    paste_pixels<D>(g, pk, t.J, nth);
  }
  __syncthreads();
  paste_hard_data<D>(g, reinterpret_cast<const int2*>(a.ev.base + (int64_t)item * a.ev.stride +
                                                      a.ev.hd_off),
                     em[kEvNHd], t.T, nth);
}

template <int D, int MODE>
static cudaError_t launch_t(const WaveArgs& a, bool pdl, cudaStream_t st) {
  // the pattern's coefficients (T^d int16) are staged in shared memory when
  // simulating, if they fit
  const int64_t tv = (D == 3) ? (int64_t)a.ti.T * a.ti.T * a.ti.T : (int64_t)a.ti.T * a.ti.T;
  const int staged = (MODE == kModeSim && tv * 2 <= 160 * 1024) ? (int)(tv * 2) : 0;
  auto fn = k_finish<D, MODE>;
  if (staged > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, staged);
    if (e != cudaSuccess) return e;
  }
  // one thread per level-J block of the pattern, up to kThreads
  const int nblk = (D == 3) ? a.ti.Tj * a.ti.Tj * a.ti.Tj : a.ti.Tj * a.ti.Tj;
  const int nth = std::min(kThreads, std::max(96, (nblk + 31) / 32 * 32));   // >= 4 + K log words
  return launch_pdl(fn, dim3(a.n_items), dim3(nth), staged, st, pdl, a, staged);
}

cudaError_t launch_finish(int mode, const WaveArgs& a, bool pdl, cudaStream_t st) {
  if (a.ti.d == 2)
    return mode == kModeSim ? launch_t<2, kModeSim>(a, pdl, st)
                            : launch_t<2, kModeSearch>(a, pdl, st);
  return mode == kModeSim ? launch_t<3, kModeSim>(a, pdl, st)
                          : launch_t<3, kModeSearch>(a, pdl, st);
}

}  // namespace ccw
