// ccf_simt.cu -- phase B of a search step on the FP32 lanes: the masked
// cross-correlation of Eq. CCW (Algorithm 1, line 10), hard-data mismatches
// (Sec. 4.4) and the per-tile top-K of every item (Algorithm 1, line 11).
//
// A CTA owns one tile of candidates and a group of NB items. The TI's
// level-J plane of each scored channel arrives in shared memory by one TMA
// bulk-tensor copy per channel (double-buffered when it fits; zero fill past
// the TI). Each thread scores 4 x-consecutive candidates for all NB items:
// a 4-wide chunk of template taps costs two 16-byte tile loads, NB 16-byte
// weight loads (broadcast) and 16 NB multiply-adds. Only template rows that
// hold data in some item are visited, from the first to the last 4-wide
// chunk holding data. FP32 is exact: every partial sum is an integer below
// 2^24 (checked on the host).
//
// Selection: each warp reduces its candidates to the K best keys per item,
// then one warp per item merges the 8 warp lists into the tile's K keys in
// global scratch; the finish kernel merges the tiles of every item.
#include "device_util.cuh"

namespace ccw {

template <int D>
struct SimtTile;
template <>
struct SimtTile<2> {
  static constexpr int TXT = 16, TX = TXT * kRx, TY = 16, TZ = 1;
};
template <>
struct SimtTile<3> {
  static constexpr int TXT = 8, TX = TXT * kRx, TY = 8, TZ = 4;
};

struct SimtSmem {
  int bar_off, meta_off, spans_off, wi_off, wres_off, tile_off;
  int tile_floats, nbuf, bytes;
};

__host__ __device__ inline int al(int v, int a) { return (v + a - 1) / a * a; }

__host__ __device__ inline SimtSmem simt_smem(int d, int nch, int rows, int chunks, int Tj,
                                              int TjP, int NB, int K, int nbuf) {
  const int TX = d == 3 ? SimtTile<3>::TX : SimtTile<2>::TX;
  const int TY = d == 3 ? SimtTile<3>::TY : SimtTile<2>::TY;
  const int TZ = d == 3 ? SimtTile<3>::TZ : SimtTile<2>::TZ;
  SimtSmem L;
  const int SX = TX + TjP, SY = TY + Tj - 1, SZ = (d == 3) ? TZ + Tj - 1 : 1;
  L.tile_floats = SX * SY * SZ;
  L.nbuf = nbuf;
  int off = 0;
  L.bar_off = off;
  off += 64;
  L.meta_off = off;  // per item: known, const, n_hd, active, last, mask cells
  off = al(off + NB * 8 * 4, 16);
  L.spans_off = off;
  off = al(off + rows * 4, 16);
  L.wi_off = off;
  off = al(off + nch * rows * chunks * NB * 16, 16);
  L.wres_off = off;
  off = al(off + kWarps * NB * K * 8, 128);
  L.tile_off = off;
  off = al(off + nbuf * al(L.tile_floats * 4, 128), 128);
  L.bytes = off + 128;  // slack to align the dynamic shared memory base
  return L;
}

enum { kMKnown = 0, kMConst, kMNHd, kMActive, kMMask };

template <int D, int NB, int MODE>
__global__ void __launch_bounds__(kThreads)
    k_ccf_simt(const __grid_constant__ WaveArgs a, const __grid_constant__ CUtensorMap tmap,
               int nbuf) {
  using TS = SimtTile<D>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const TiDev& t = a.ti;
  const int rows = t.rows, chunks = t.chunks, Tj = t.Tj, T = t.T, s = t.s;
  const int K = a.K;
  const SimtSmem L = simt_smem(D, t.nch, rows, chunks, Tj, t.TjP, NB, K, nbuf);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar_off);
  int* flag = reinterpret_cast<int*>(smem + L.bar_off + 32);
  int* meta = reinterpret_cast<int*>(smem + L.meta_off);
  int* spans = reinterpret_cast<int*>(smem + L.spans_off);
  float4* Wi = reinterpret_cast<float4*>(smem + L.wi_off);
  uint64_t* wres = reinterpret_cast<uint64_t*>(smem + L.wres_off);
  const int tile_stride = al(L.tile_floats * 4, 128) / 4;
  float* tiles = reinterpret_cast<float*>(smem + L.tile_off);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile_id = blockIdx.x;
  const int item0 = blockIdx.y * NB;
  const int SX = TS::TX + t.TjP, SY = TS::TY + Tj - 1;
  const int cx0 = (tile_id % t.tiles[0]) * TS::TX;
  const int cy0 = ((tile_id / t.tiles[0]) % t.tiles[1]) * TS::TY;
  const int cz0 = (tile_id / (t.tiles[0] * t.tiles[1])) * TS::TZ;
  const uint32_t tile_bytes = (uint32_t)(L.tile_floats * 4);

  // ---- start the TMA copies of the first channel planes -------------------
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    flag[0] = 0;
    for (int b = 0; b < nbuf && b < t.nch; ++b) {
      mbar_arrive_expect_tx(&bar[b], tile_bytes);
      tma_load_4d(tiles + b * tile_stride, &tmap, &bar[b], cx0, cy0, cz0, t.plane0 + b);
    }
  }

  // ---- per-item event records --------------------------------------------
  pdl_trigger();
  pdl_wait();   // the event records of this step are complete
  if (tid < NB) {
    const int item = item0 + tid;
    int* m = meta + tid * 8;
    if (item < a.n_items) {
      const int* em = reinterpret_cast<const int*>(a.ev.base + (int64_t)item * a.ev.stride);
      m[kMKnown] = em[kEvKnown];
      m[kMConst] = em[kEvConst];
      m[kMNHd] = em[kEvNHd];
      m[kMMask] = em[kEvMaskCells];
      // items settled by the learned proposal need no full search
      m[kMActive] = (MODE == kModeMap) ? 1 : (em[kEvKnown] > 0 && !em[kEvResolved]);
    } else {
      m[kMKnown] = 0;
      m[kMConst] = 0;
      m[kMNHd] = 0;
      m[kMMask] = 0;
      m[kMActive] = 0;
    }
  }
  if (tid == 0) flag[1] = 0;  // number of spans
  __syncthreads();
  // weights of the group, interleaved [ch][row][chunk][nb]
  {
    const int total = t.nch * rows * chunks * NB;
    for (int i = tid; i < total; i += kThreads) {
      const int nb = i % NB;
      const int rest = i / NB;   // (ch * rows + row) * chunks + g
      float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
      if (meta[nb * 8 + kMActive]) {
        const float4* src = reinterpret_cast<const float4*>(
            a.ev.base + (int64_t)(item0 + nb) * a.ev.stride + a.ev.w_off);
        w = src[rest];
      }
      Wi[i] = w;
    }
  }
  // rows holding data in some item of the group: one span of chunks each
  for (int row = tid; row < rows; row += kThreads) {
    uint32_t m = 0;
#pragma unroll
    for (int nb = 0; nb < NB; ++nb)
      if (meta[nb * 8 + kMActive])
        m |= reinterpret_cast<const uint32_t*>(a.ev.base + (int64_t)(item0 + nb) * a.ev.stride +
                                               a.ev.mask_off)[row];
    if (m) {
      const int g0 = __ffs(m) - 1, g1 = 31 - __clz(m);
      const int k = atomicAdd(&flag[1], 1);
      spans[k] = (row << 16) | (g0 << 8) | g1;
    }
  }
  __syncthreads();
  const int n_spans = flag[1];
  bool any_known = false;
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) any_known |= meta[nb * 8 + kMActive] != 0;

  // ---- masked CCF -----------------------------------------------------------
  const int ltx = tid % TS::TXT;
  const int lty = (tid / TS::TXT) % TS::TY;
  const int ltz = tid / (TS::TXT * TS::TY);
  float acc[kRx][NB];
#pragma unroll
  for (int i = 0; i < kRx; ++i)
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) acc[i][nb] = 0.f;
  int timed_out_ch = -1;
  for (int ch = 0; ch < t.nch; ++ch) {
    const int b = ch % nbuf;
    const uint32_t parity = (uint32_t)((ch / nbuf) & 1);
    if (tid == 0 && !mbar_wait_bounded(&bar[b], parity)) flag[0] = 1;
    __syncthreads();
    if (flag[0]) {
      timed_out_ch = ch;
      break;
    }
    mbar_try_wait(&bar[b], parity);   // acquire the copy for every thread
    if (any_known) {
      const float* tile = tiles + b * tile_stride;
      const float4* wch = Wi + (int64_t)ch * rows * chunks * NB;
      for (int sp = 0; sp < n_spans; ++sp) {
        const int e = spans[sp];
        const int row = e >> 16, g0 = (e >> 8) & 0xFF, g1 = e & 0xFF;
        const int uy = row % Tj, uz = row / Tj;
        const float4* trow = reinterpret_cast<const float4*>(
            tile + ((ltz + uz) * SY + (lty + uy)) * SX + kRx * ltx);
        const float4* wrow = wch + (int64_t)row * chunks * NB;
        float4 cur = trow[g0];
        for (int g = g0; g <= g1; ++g) {
          const float4 nxt = trow[g + 1];
#pragma unroll
          for (int nb = 0; nb < NB; ++nb) {
            const float4 w = wrow[g * NB + nb];
            acc[0][nb] = fmaf(w.x, cur.x, acc[0][nb]);
            acc[0][nb] = fmaf(w.y, cur.y, acc[0][nb]);
            acc[0][nb] = fmaf(w.z, cur.z, acc[0][nb]);
            acc[0][nb] = fmaf(w.w, cur.w, acc[0][nb]);
            acc[1][nb] = fmaf(w.x, cur.y, acc[1][nb]);
            acc[1][nb] = fmaf(w.y, cur.z, acc[1][nb]);
            acc[1][nb] = fmaf(w.z, cur.w, acc[1][nb]);
            acc[1][nb] = fmaf(w.w, nxt.x, acc[1][nb]);
            acc[2][nb] = fmaf(w.x, cur.z, acc[2][nb]);
            acc[2][nb] = fmaf(w.y, cur.w, acc[2][nb]);
            acc[2][nb] = fmaf(w.z, nxt.x, acc[2][nb]);
            acc[2][nb] = fmaf(w.w, nxt.y, acc[2][nb]);
            acc[3][nb] = fmaf(w.x, cur.w, acc[3][nb]);
            acc[3][nb] = fmaf(w.y, nxt.x, acc[3][nb]);
            acc[3][nb] = fmaf(w.z, nxt.y, acc[3][nb]);
            acc[3][nb] = fmaf(w.w, nxt.z, acc[3][nb]);
          }
          cur = nxt;
        }
      }
    }
    __syncthreads();   // every thread is done with buffer b
    if (tid == 0 && ch + nbuf < t.nch) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar[b], tile_bytes);
      tma_load_4d(tiles + b * tile_stride, &tmap, &bar[b], cx0, cy0, cz0, t.plane0 + ch + nbuf);
    }
  }
  if (timed_out_ch >= 0) {
    // record the failure, then let the copies that may still be in flight
    // (the one waited for and, double-buffered, the next channel's) land
    // before the CTA exits
    if (tid == 0) {
      atomicOr(a.status, kStatusTimeout);
      for (int ch = timed_out_ch; ch < t.nch && ch < timed_out_ch + nbuf; ++ch)
        mbar_wait_bounded(&bar[ch % nbuf], (uint32_t)((ch / nbuf) & 1));
    }
    return;
  }

  // ---- scores, mismatches, per-item selection -------------------------------
  const int cy = cy0 + lty, cz = cz0 + ltz;
  const int64_t Kp = (int64_t)K < t.P ? K : t.P;
  unsigned long long* work = (MODE == kModeSim) ? a.call->work : a.work;
  if (work && tid == 0 && tile_id == 0) {
#pragma unroll
    for (int nb = 0; nb < NB; ++nb)
      if (meta[nb * 8 + kMActive] && MODE != kModeMap) {
        atomicAdd(&work[0], (unsigned long long)t.P);
        atomicAdd(&work[1], (unsigned long long)t.P * meta[nb * 8 + kMMask] * t.nch);
      }
  }
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    if (!meta[nb * 8 + kMActive]) continue;
    const int item = item0 + nb;
    const int known = meta[nb * 8 + kMKnown];
    const int cons = meta[nb * 8 + kMConst];
    const int nhd = meta[nb * 8 + kMNHd];
    const int2* hdl = reinterpret_cast<const int2*>(a.ev.base + (int64_t)item * a.ev.stride +
                                                    a.ev.hd_off);
    // hard-data mismatches of the thread's candidates, loads overlapped
    const uint8_t* tb0 =
        t.ti + (int64_t)s * (cx0 + kRx * ltx) + (int64_t)t.tp[0] * ((int64_t)s * cy + (int64_t)t.tp[1] * s * cz);
    const bool row_ok = cy < t.cd[1] && cz < t.cd[2];
    int misv[kRx];
#pragma unroll
    for (int i = 0; i < kRx; ++i) misv[i] = 0;
    if (row_ok) {
      for (int k = 0; k < nhd; ++k) {
        const int2 e = __ldg(hdl + k);
#pragma unroll
        for (int i = 0; i < kRx; ++i)
          if (cx0 + kRx * ltx + i < t.cd[0])
            misv[i] += (__ldg(tb0 + (int64_t)s * i + e.x) != (uint8_t)e.y);
      }
    }
    uint64_t keys[kRx];
#pragma unroll
    for (int i = 0; i < kRx; ++i) {
      const int cx = cx0 + kRx * ltx + i;
      keys[i] = kNoKey;
      if (cx >= t.cd[0] || cy >= t.cd[1] || cz >= t.cd[2]) continue;
      const int score = __float2int_rn(acc[i][nb]) + cons;
      const int mis = misv[i];
      const int c = cx + t.cd[0] * (cy + t.cd[1] * cz);
      if (MODE == kModeMap) {
        a.map_score[(int64_t)item * t.P + c] = known ? score : 0;
        if (a.map_mis) a.map_mis[(int64_t)item * t.P + c] = known ? mis : 0;
      } else {
        keys[i] = make_key(mis, score, c);
      }
    }
    if (MODE == kModeMap) continue;
    // warp top-K of this item
    uint64_t prev = 0;
    bool first = true;
    for (int r = 0; r < Kp; ++r) {
      uint64_t m = kNoKey;
#pragma unroll
      for (int i = 0; i < kRx; ++i)
        if ((first || keys[i] > prev) && keys[i] < m) m = keys[i];
      m = warp_min_u64(m);
      if (lane == 0) wres[(warp * NB + nb) * K + r] = m;
      prev = m;
      first = false;
      if (m == kNoKey) {
        if (lane == 0)
          for (int rr = r + 1; rr < Kp; ++rr) wres[(warp * NB + nb) * K + rr] = kNoKey;
        break;
      }
    }
  }
  if (MODE == kModeMap) return;
  __syncthreads();
  // one warp per item merges the warp lists into the tile's K keys
  for (int nb = warp; nb < NB; nb += kWarps) {
    if (!meta[nb * 8 + kMActive]) continue;
    const int item = item0 + nb;
    const int M = kWarps * (int)Kp;
    uint64_t prev = 0;
    bool first = true;
    unsigned long long* part = a.part + ((int64_t)item * t.n_tiles + tile_id) * K;
    for (int r = 0; r < Kp; ++r) {
      uint64_t m = kNoKey;
      for (int j = lane; j < M; j += 32) {
        const uint64_t v = wres[((j / (int)Kp) * NB + nb) * K + (j % (int)Kp)];
        if ((first || v > prev) && v < m) m = v;
      }
      m = warp_min_u64(m);
      if (lane == 0) part[r] = m;
      prev = m;
      first = false;
    }
  }
}

// ---------------------------------------------------------------------------
int simt_smem_bytes(int d, int nch, int rows, int chunks, int Tj, int TjP, int NB, int K,
                    int nbuf) {
  return simt_smem(d, nch, rows, chunks, Tj, TjP, NB, K, nbuf).bytes;
}

void simt_tile_shape(int d, int tile[3]) {
  if (d == 3) {
    tile[0] = SimtTile<3>::TX;
    tile[1] = SimtTile<3>::TY;
    tile[2] = SimtTile<3>::TZ;
  } else {
    tile[0] = SimtTile<2>::TX;
    tile[1] = SimtTile<2>::TY;
    tile[2] = 1;
  }
}

// box of the TMA copy of one channel plane (x, y, z) for the tile shape
void simt_tma_box(int d, int Tj, int TjP, int box[3]) {
  int tile[3];
  simt_tile_shape(d, tile);
  box[0] = tile[0] + TjP;
  box[1] = tile[1] + Tj - 1;
  box[2] = (d == 3) ? tile[2] + Tj - 1 : 1;
}

template <int D, int NB, int MODE>
static cudaError_t launch_t(const WaveArgs& a, const CUtensorMap& tmap, int nbuf, int smem,
                            bool pdl, cudaStream_t st) {
  auto fn = k_ccf_simt<D, NB, MODE>;
  static int configured = 0;   // largest dynamic shared memory size set so far
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  dim3 grid(a.ti.n_tiles, (a.n_items + NB - 1) / NB);
  return launch_pdl(fn, grid, dim3(kThreads), smem, st, pdl, a, tmap, nbuf);
}

template <int D, int NB>
static cudaError_t launch_nb(int mode, const WaveArgs& a, const CUtensorMap& tmap, int nbuf,
                             int smem, bool pdl, cudaStream_t st) {
  if (mode == kModeSim) return launch_t<D, NB, kModeSim>(a, tmap, nbuf, smem, pdl, st);
  if (mode == kModeSearch) return launch_t<D, NB, kModeSearch>(a, tmap, nbuf, smem, pdl, st);
  return launch_t<D, NB, kModeMap>(a, tmap, nbuf, smem, pdl, st);
}

cudaError_t launch_ccf_simt(int mode, const WaveArgs& a, const CUtensorMap& tmap, int nbuf,
                            int smem, bool pdl, cudaStream_t st) {
  if (a.ti.d == 2) {
    switch (a.nb) {
      case 1: return launch_nb<2, 1>(mode, a, tmap, nbuf, smem, pdl, st);
      case 2: return launch_nb<2, 2>(mode, a, tmap, nbuf, smem, pdl, st);
      case 8: return launch_nb<2, 8>(mode, a, tmap, nbuf, smem, pdl, st);
      default: return launch_nb<2, 4>(mode, a, tmap, nbuf, smem, pdl, st);
    }
  }
  switch (a.nb) {
    case 1: return launch_nb<3, 1>(mode, a, tmap, nbuf, smem, pdl, st);
    case 4: return launch_nb<3, 4>(mode, a, tmap, nbuf, smem, pdl, st);
    default: return launch_nb<3, 2>(mode, a, tmap, nbuf, smem, pdl, st);
  }
}

}  // namespace ccw
