// search.cu -- the best-match search kernel of CCWSIM on sm_103a.
//
// One launch processes a set of "items" (a patch of one realization, or one
// explicit data event) against every candidate of the training image. A CTA
// owns one tile of candidates of one item and runs, in order:
//   1. the data event and its level-J Haar approximation (Algorithm 1,
//      lines 8-9): facies counts of every s^d block of the known cells; the
//      one-hot weights w_f = b_f - b_{F-1} (f < F-1) and the constant
//      s^d * sum_u b_{F-1}(u) that restore the full F-channel score;
//   2. the masked cross-correlation of Eq. CCW over the tile (Algorithm 1,
//      line 10): exact FP32 multiply-adds over the TI's level-J planes staged
//      in shared memory, only over rows of the template that hold data;
//   3. the hard-data mismatch count of every candidate (Sec. 4.4);
//   4. the tile's top-K by the 64-bit ranking key, published to global
//      scratch; the last CTA of the item merges all tiles, draws the pick
//      with Philox (Algorithm 1, lines 11-12) and, when simulating, pastes
//      the Inverse-DWT of the pick (Algorithm 1, lines 13-14).
#include "ccw_internal.cuh"

namespace ccw {

template <int D>
struct TileShape;
template <>
struct TileShape<2> {
  static constexpr int TXT = 16, TX = TXT * kRx, TY = 16, TZ = 1;
};
template <>
struct TileShape<3> {
  static constexpr int TXT = 8, TX = TXT * kRx, TY = 8, TZ = 4;
};

struct SmemLayout {
  int w_off, tile_off, spans_off, hd_off, red_off, topk_off, misc_off, bytes;
  int rows, SX, SY, SZ;
};

__host__ __device__ inline int align16(int v) { return (v + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int d, int nch, int Tj, int TjP, int TX, int TY,
                                                  int TZ) {
  SmemLayout L;
  L.rows = (d == 3) ? Tj * Tj : Tj;
  L.SX = TX + TjP;
  L.SY = TY + Tj - 1;
  L.SZ = (d == 3) ? TZ + Tj - 1 : 1;
  int off = 0;
  L.w_off = off;
  off = align16(off + nch * L.rows * TjP * 4);
  L.tile_off = off;
  off = align16(off + L.SZ * L.SY * L.SX * 4);
  L.spans_off = off;
  off = align16(off + L.rows * 4);
  L.hd_off = off;
  off = align16(off + kMaxHd * 4);
  L.red_off = off;
  off = align16(off + 32 * 8);
  L.topk_off = off;
  off = align16(off + CCW_MAX_TOPK * 8);
  L.misc_off = off;
  off = align16(off + 16 * 4);
  L.bytes = off;
  return L;
}

int search_smem_bytes(int d, int nch, int Tj, int TjP) {
  if (d == 3)
    return smem_layout(3, nch, Tj, TjP, TileShape<3>::TX, TileShape<3>::TY, TileShape<3>::TZ).bytes;
  return smem_layout(2, nch, Tj, TjP, TileShape<2>::TX, TileShape<2>::TY, TileShape<2>::TZ).bytes;
}

void search_tiles(int d, const int cd[3], int tiles[3]) {
  if (d == 3) {
    tiles[0] = (cd[0] + TileShape<3>::TX - 1) / TileShape<3>::TX;
    tiles[1] = (cd[1] + TileShape<3>::TY - 1) / TileShape<3>::TY;
    tiles[2] = (cd[2] + TileShape<3>::TZ - 1) / TileShape<3>::TZ;
  } else {
    tiles[0] = (cd[0] + TileShape<2>::TX - 1) / TileShape<2>::TX;
    tiles[1] = (cd[1] + TileShape<2>::TY - 1) / TileShape<2>::TY;
    tiles[2] = 1;
  }
}

// misc ints in shared memory
enum { kMiscNSpans = 0, kMiscNHd, kMiscKnown, kMiscConst, kMiscMaskCells, kMiscLast, kMiscBad };

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (w < v) ? w : v;
  }
  return v;
}

// Minimum over the CTA of one value per thread; result broadcast.
__device__ __forceinline__ uint64_t block_min_u64(uint64_t v, uint64_t* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_min_u64(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = (lane < kThreads / 32) ? red[lane] : kNoKey;
    w = warp_min_u64(w);
    if (lane == 0) red[kThreads / 32] = w;
  }
  __syncthreads();
  const uint64_t r = red[kThreads / 32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Inverse scaled Haar of one s^d block held in place (layout of
// ccw_ti_export what = 2): level j = J..1, axes z, y, x; pairs 2^(j-1) apart:
// low = (lo + hi) / 2 at the lower position, (lo - hi) / 2 at the upper.
// ---------------------------------------------------------------------------
template <int D>
__device__ void haar_block_inverse(int* v, int s, int J) {
  const int sz = (D == 3) ? s : 1;
  for (int j = J; j >= 1; --j) {
    const int h = 1 << (j - 1);
    for (int a = D - 1; a >= 0; --a) {
      const int stride = (a == 0) ? 1 : (a == 1 ? s : s * s);
      const int hx = (a == 0) ? 2 * h : h, hy = (a == 1) ? 2 * h : h,
                hz = (D == 3) ? ((a == 2) ? 2 * h : h) : 1;
      for (int z = 0; z < sz; z += hz)
        for (int y = 0; y < s; y += hy)
          for (int x = 0; x < s; x += hx) {
            const int p = x + s * (y + s * z), q = p + h * stride;
            const int lo = v[p], hi = v[q];
            v[p] = (lo + hi) >> 1;
            v[q] = (lo - hi) >> 1;
          }
    }
  }
}

// Paste the Inverse-DWT of candidate `pick` with its first cell at window
// origin `o` (coordinates of `grid`, dims gdim). Cells outside the grid are
// skipped. When `overlay` is given, a hard datum of the cell (overlay coords =
// grid coords - off) replaces the pattern value.
template <int D>
__device__ void paste_pattern(const SearchArgs& a, int pick, const int o[3], uint8_t* grid,
                              const int gdim[3], const uint8_t* overlay, const int off[3]) {
  const int pcx = pick % a.cd[0];
  const int pcy = (pick / a.cd[0]) % a.cd[1];
  const int pcz = pick / (a.cd[0] * a.cd[1]);
  const int Tj = a.Tj, s = a.s;
  const int nblk = (D == 3) ? Tj * Tj * Tj : Tj * Tj;
  int v[256];
  for (int b = threadIdx.x; b < nblk; b += kThreads) {
    const int ux = b % Tj, uy = (b / Tj) % Tj, uz = (D == 3) ? b / (Tj * Tj) : 0;
    const int64_t gb = (int64_t)(pcx + ux) +
                       (int64_t)a.nc[0] * ((pcy + uy) + (int64_t)a.nc[1] * (pcz + uz));
    const int16_t* src = a.pyr + gb * a.sd;
    for (int c = 0; c < a.sd; ++c) v[c] = src[c];
    haar_block_inverse<D>(v, s, a.J);
    const int sz = (D == 3) ? s : 1;
    for (int cz = 0; cz < sz; ++cz)
      for (int cy = 0; cy < s; ++cy)
        for (int cx = 0; cx < s; ++cx) {
          const int gx = o[0] + s * ux + cx, gy = o[1] + s * uy + cy,
                    gz = (D == 3) ? o[2] + s * uz + cz : 0;
          if (gx < 0 || gy < 0 || gz < 0 || gx >= gdim[0] || gy >= gdim[1] || gz >= gdim[2])
            continue;
          uint8_t val = (uint8_t)v[cx + s * (cy + s * cz)];
          if (overlay) {
            const int hx = gx - off[0], hy = gy - off[1], hz = gz - off[2];
            if (hx >= 0 && hy >= 0 && hz >= 0 && hx < a.G[0] && hy < a.G[1] && hz < a.G[2]) {
              const uint8_t h =
                  overlay[hx + (int64_t)a.G[0] * (hy + (int64_t)a.G[1] * hz)];
              if (h != CCW_UNKNOWN) val = h;
            }
          }
          grid[gx + (int64_t)gdim[0] * (gy + (int64_t)gdim[1] * gz)] = val;
        }
  }
}

template <int D, int MODE>
__global__ void __launch_bounds__(kThreads) k_search(const __grid_constant__ SearchArgs a) {
  using TS = TileShape<D>;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(D, a.nch, a.Tj, a.TjP, TS::TX, TS::TY, TS::TZ);
  float* W = reinterpret_cast<float*>(smem + L.w_off);
  float* tile = reinterpret_cast<float*>(smem + L.tile_off);
  int* spans = reinterpret_cast<int*>(smem + L.spans_off);
  int* hdl = reinterpret_cast<int*>(smem + L.hd_off);
  uint64_t* red = reinterpret_cast<uint64_t*>(smem + L.red_off);
  uint64_t* topk = reinterpret_cast<uint64_t*>(smem + L.topk_off);
  int* misc = reinterpret_cast<int*>(smem + L.misc_off);

  const int tid = threadIdx.x;
  const int item = blockIdx.y;
  const int tile_id = blockIdx.x;
  const int T = a.T, Tj = a.Tj, s = a.s;

  // ---- item decode ---------------------------------------------------------
  int o[3] = {0, 0, 0}, off[3] = {0, 0, 0};
  uint32_t ctr_r = 0, ctr_p = 0;
  int slot = 0, patch = 0;
  uint8_t* sg = nullptr;
  const uint8_t* de = nullptr;
  const uint8_t* hdw = nullptr;
  if (MODE == kModeSim) {
    const int2 it = a.items[item];
    slot = it.x;
    patch = it.y;
    ctr_r = (uint32_t)(a.real_base + slot);
    ctr_p = (uint32_t)patch;
    const uint32_t flips =
        a.path_random ? (draw_word(a.seed, ctr_r, 0u, 1u) & ((1u << D) - 1u)) : 0u;
    const int ip[3] = {patch % a.np[0], (patch / a.np[0]) % a.np[1], patch / (a.np[0] * a.np[1])};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const bool f = (flips >> ax) & 1u;
      const int t = (ax < D) ? T : 1;
      o[ax] = (ax < D) ? (f ? a.Gp[ax] - t - a.S * ip[ax] : a.S * ip[ax]) : 0;
      off[ax] = (ax < D && f) ? a.Gp[ax] - a.G[ax] : 0;
    }
    sg = a.sg + (int64_t)slot * a.gp_vol;
  } else {
    const int64_t tv = (D == 3) ? (int64_t)T * T * T : (int64_t)T * T;
    de = a.de + (int64_t)item * tv;
    hdw = a.hd ? a.hd + (int64_t)item * tv : nullptr;
    if (MODE == kModeSearch) {
      ctr_r = a.ctr[2 * item];
      ctr_p = a.ctr[2 * item + 1];
    }
  }

  // ---- 1. data event and its level-J approximation --------------------------
  const int rows = L.rows;
  for (int i = tid; i < a.nch * rows * a.TjP; i += kThreads) W[i] = 0.f;
  if (tid < 16) misc[tid] = 0;
  __syncthreads();
  {
    const int ncells = (D == 3) ? Tj * Tj * Tj : Tj * Tj;
    const int sz = (D == 3) ? s : 1;
    int my_known = 0, my_const = 0, my_mask = 0;
    for (int u = tid; u < ncells; u += kThreads) {
      const int ux = u % Tj, uy = (u / Tj) % Tj, uz = (D == 3) ? u / (Tj * Tj) : 0;
      int b0 = 0, b1 = 0, b2 = 0, b3 = 0, b4 = 0, b5 = 0, b6 = 0, b7 = 0, csum = 0, cnt = 0;
      for (int cz = 0; cz < sz; ++cz)
        for (int cy = 0; cy < s; ++cy)
          for (int cx = 0; cx < s; ++cx) {
            const int qx = s * ux + cx, qy = s * uy + cy, qz = (D == 3) ? s * uz + cz : 0;
            uint8_t v, h;
            if (MODE == kModeSim) {
              const int gx = o[0] + qx, gy = o[1] + qy, gz = o[2] + qz;
              const int hx = gx - off[0], hy = gy - off[1], hz = gz - off[2];
              h = CCW_UNKNOWN;
              if (hx >= 0 && hy >= 0 && hz >= 0 && hx < a.G[0] && hy < a.G[1] && hz < a.G[2])
                h = a.overlay[hx + (int64_t)a.G[0] * (hy + (int64_t)a.G[1] * hz)];
              const uint8_t sv = sg[gx + (int64_t)a.Gp[0] * (gy + (int64_t)a.Gp[1] * gz)];
              v = (h != CCW_UNKNOWN) ? h : sv;
            } else {
              const int q = qx + T * (qy + T * qz);
              v = de[q];
              h = hdw ? hdw[q] : (uint8_t)CCW_UNKNOWN;
            }
            if (h != CCW_UNKNOWN) {
              const int slot_h = atomicAdd(&misc[kMiscNHd], 1);
              if (slot_h < kMaxHd) hdl[slot_h] = ((qx + T * (qy + T * qz)) << 8) | h;
              if (h >= a.F) atomicOr(&misc[kMiscBad], kStatusBadCode);
            }
            if (v != CCW_UNKNOWN) {
              if (v >= a.F) {
                atomicOr(&misc[kMiscBad], kStatusBadCode);
                continue;
              }
              ++cnt;
              csum += v;
              b0 += (v == 0);
              b1 += (v == 1);
              b2 += (v == 2);
              b3 += (v == 3);
              b4 += (v == 4);
              b5 += (v == 5);
              b6 += (v == 6);
              b7 += (v == 7);
            }
          }
      if (cnt) {
        my_known += cnt;
        ++my_mask;
        const int row = uy + Tj * uz;
        if (a.score_mode == 0) {
          const int bl[8] = {b0, b1, b2, b3, b4, b5, b6, b7};
          const int blast = bl[a.F - 1];
          for (int ch = 0; ch < a.F - 1; ++ch)
            W[(ch * rows + row) * a.TjP + ux] = (float)(bl[ch] - blast);
          my_const += a.sd * blast;
        } else {
          W[row * a.TjP + ux] = (float)csum;
        }
      }
    }
    if (my_known) atomicAdd(&misc[kMiscKnown], my_known);
    if (my_const) atomicAdd(&misc[kMiscConst], my_const);
    if (my_mask) atomicAdd(&misc[kMiscMaskCells], my_mask);
  }
  __syncthreads();
  // row spans (in 4-wide chunks) of the template rows that hold weights
  for (int row = tid; row < rows; row += kThreads) {
    int lo = Tj, hi = -1;
    for (int ch = 0; ch < a.nch; ++ch) {
      const float* wr = W + (ch * rows + row) * a.TjP;
      for (int ux = 0; ux < Tj; ++ux)
        if (wr[ux] != 0.f) {
          lo = min(lo, ux);
          hi = max(hi, ux);
        }
    }
    if (hi >= 0) {
      const int k = atomicAdd(&misc[kMiscNSpans], 1);
      spans[k] = (row << 16) | ((lo >> 2) << 8) | (hi >> 2);
    }
  }
  __syncthreads();
  const int known = misc[kMiscKnown];
  const int cons = misc[kMiscConst];
  const int n_spans = misc[kMiscNSpans];
  const int n_hd = min(misc[kMiscNHd], kMaxHd);
  if (tid == 0 && tile_id == 0) {
    const int bad = misc[kMiscBad] | (misc[kMiscNHd] > kMaxHd ? kStatusHdOverflow : 0);
    if (bad) atomicOr(a.status, bad);
  }

  // ---- empty data event: one uniform draw (Algorithm 1, lines 5-6) --------
  if (known == 0) {
    if (MODE == kModeMap) {
      // all-zero maps
    } else if (tile_id != 0) {
      return;
    } else {
      const uint32_t u = draw_word(a.seed, ctr_r, ctr_p, 0u);
      const int pk = (int)mul_shift(u, a.P);
      if (MODE == kModeSearch) {
        if (tid < a.K) {
          a.topk_idx[item * a.K + tid] = -1;
          a.topk_score[item * a.K + tid] = 0;
          a.topk_mis[item * a.K + tid] = 0;
        }
        if (tid == 0) a.pick[item] = pk;
      } else {
        if (a.log && tid < a.log_stride) {
          int32_t* e = a.log + ((int64_t)slot * a.n_patches + patch) * a.log_stride;
          e[tid] = (tid == 0) ? pk : (tid == 3 ? (CCW_LOG_FLAG_UNIFORM | CCW_LOG_FLAG_DONE)
                                              : (tid < 3 ? 0 : -1));
        }
        const int gdim[3] = {a.Gp[0], a.Gp[1], a.Gp[2]};
        paste_pattern<D>(a, pk, o, sg, gdim, a.overlay, off);
      }
      return;
    }
  }
  if (a.work && tid == 0 && tile_id == 0 && known) {
    atomicAdd(&a.work[0], (unsigned long long)a.P);
    atomicAdd(&a.work[1], (unsigned long long)a.P * (unsigned long long)misc[kMiscMaskCells] *
                              (unsigned long long)a.nch);
  }

  // ---- 2. masked CCF over this tile ---------------------------------------
  const int tx_t = tile_id % a.tiles[0];
  const int ty_t = (tile_id / a.tiles[0]) % a.tiles[1];
  const int tz_t = tile_id / (a.tiles[0] * a.tiles[1]);
  const int cx0 = tx_t * TS::TX, cy0 = ty_t * TS::TY, cz0 = tz_t * TS::TZ;
  const int ltx = tid % TS::TXT;
  const int lty = (tid / TS::TXT) % TS::TY;
  const int ltz = tid / (TS::TXT * TS::TY);
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
  if (known) {
    const int SX = L.SX, SY = L.SY, SZ = L.SZ;
    const int tile_n = SX * SY * SZ;
    for (int ch = 0; ch < a.nch; ++ch) {
      const float* plane = a.planes + (int64_t)ch * a.ncv;
      for (int i = tid; i < tile_n; i += kThreads) {
        const int lx = i % SX, ly = (i / SX) % SY, lz = i / (SX * SY);
        const int gx = cx0 + lx, gy = cy0 + ly, gz = cz0 + lz;
        float val = 0.f;
        if (gx < a.nc[0] && gy < a.nc[1] && gz < a.nc[2])
          val = __ldg(plane + gx + (int64_t)a.nc[0] * (gy + (int64_t)a.nc[1] * gz));
        tile[i] = val;
      }
      __syncthreads();
      const float* wch = W + ch * rows * a.TjP;
      for (int sp = 0; sp < n_spans; ++sp) {
        const int e = spans[sp];
        const int row = e >> 16, g0 = (e >> 8) & 0xFF, g1 = e & 0xFF;
        const int uy = row % Tj, uz = row / Tj;
        const float4* trow = reinterpret_cast<const float4*>(
            tile + ((ltz + uz) * SY + (lty + uy)) * SX + kRx * ltx);
        const float4* wrow = reinterpret_cast<const float4*>(wch + row * a.TjP);
        float4 cur = trow[g0];
        for (int g = g0; g <= g1; ++g) {
          const float4 nxt = trow[g + 1];
          const float4 w = wrow[g];
          acc0 = fmaf(w.x, cur.x, acc0);
          acc0 = fmaf(w.y, cur.y, acc0);
          acc0 = fmaf(w.z, cur.z, acc0);
          acc0 = fmaf(w.w, cur.w, acc0);
          acc1 = fmaf(w.x, cur.y, acc1);
          acc1 = fmaf(w.y, cur.z, acc1);
          acc1 = fmaf(w.z, cur.w, acc1);
          acc1 = fmaf(w.w, nxt.x, acc1);
          acc2 = fmaf(w.x, cur.z, acc2);
          acc2 = fmaf(w.y, cur.w, acc2);
          acc2 = fmaf(w.z, nxt.x, acc2);
          acc2 = fmaf(w.w, nxt.y, acc2);
          acc3 = fmaf(w.x, cur.w, acc3);
          acc3 = fmaf(w.y, nxt.x, acc3);
          acc3 = fmaf(w.z, nxt.y, acc3);
          acc3 = fmaf(w.w, nxt.z, acc3);
          cur = nxt;
        }
      }
      __syncthreads();
    }
  }

  // ---- 3. scores, mismatches ------------------------------------------------
  const int cy = cy0 + lty, cz = cz0 + ltz;
  const float accs[4] = {acc0, acc1, acc2, acc3};
  uint64_t keys[4];
#pragma unroll
  for (int i = 0; i < kRx; ++i) {
    const int cx = cx0 + kRx * ltx + i;
    keys[i] = kNoKey;
    if (cx >= a.cd[0] || cy >= a.cd[1] || cz >= a.cd[2]) continue;
    const int score = __float2int_rn(accs[i]) + cons;
    int mis = 0;
    for (int k = 0; k < n_hd; ++k) {
      const int e = hdl[k];
      const int q = e >> 8;
      const int qx = q % T, qy = (q / T) % T, qz = (D == 3) ? q / (T * T) : 0;
      const int fx = s * cx + qx, fy = s * cy + qy, fz = (D == 3) ? s * cz + qz : 0;
      mis += (a.ti[fx + (int64_t)a.n[0] * (fy + (int64_t)a.n[1] * fz)] != (uint8_t)(e & 0xFF));
    }
    const int c = cx + a.cd[0] * (cy + a.cd[1] * cz);
    if (MODE == kModeMap) {
      a.map_score[(int64_t)item * a.P + c] = known ? score : 0;
      if (a.map_mis) a.map_mis[(int64_t)item * a.P + c] = known ? mis : 0;
    } else {
      keys[i] = make_key(mis, score, c);
    }
  }
  if (MODE == kModeMap) return;

  // ---- 4. tile top-K, cross-tile merge, draw, paste -------------------------
  const int K = a.K;
  const int Kp = (int)((int64_t)K < a.P ? K : a.P);
  {
    uint64_t prev = 0;
    bool first = true;
    for (int r = 0; r < Kp; ++r) {
      uint64_t m = kNoKey;
#pragma unroll
      for (int i = 0; i < kRx; ++i)
        if ((first || keys[i] > prev) && keys[i] < m) m = keys[i];
      m = block_min_u64(m, red);
      if (tid == 0) topk[r] = m;
      prev = m;
      first = false;
      if (m == kNoKey) {
        if (tid == 0)
          for (int rr = r + 1; rr < Kp; ++rr) topk[rr] = kNoKey;
        break;
      }
    }
  }
  __syncthreads();
  unsigned long long* part = a.part + ((int64_t)item * a.n_tiles + tile_id) * K;
  if (tid < Kp) part[tid] = topk[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned int prev = atomicAdd(&a.counters[item], 1u);
    misc[kMiscLast] = (prev == (unsigned int)(a.n_tiles - 1));
  }
  __syncthreads();
  if (!misc[kMiscLast]) return;
  __threadfence();

  // last CTA of this item: merge n_tiles * Kp keys
  {
    const unsigned long long* all = a.part + (int64_t)item * a.n_tiles * K;
    const int M = a.n_tiles * K;
    uint64_t prev = 0;
    bool first = true;
    for (int r = 0; r < Kp; ++r) {
      uint64_t m = kNoKey;
      for (int j = tid; j < M; j += kThreads) {
        if ((j % K) >= Kp) continue;
        const uint64_t v = __ldcg(all + j);
        if ((first || v > prev) && v < m) m = v;
      }
      m = block_min_u64(m, red);
      if (tid == 0) topk[r] = m;
      prev = m;
      first = false;
    }
  }
  if (tid == 0) a.counters[item] = 0u;
  __syncthreads();
  const uint32_t u = draw_word(a.seed, ctr_r, ctr_p, 0u);
  const int jsel = (int)mul_shift(u, Kp);
  const uint64_t sel = topk[jsel];
  const int pk = key_index(sel);
  if (MODE == kModeSearch) {
    if (tid < K) {
      const bool v = tid < Kp;
      a.topk_idx[item * K + tid] = v ? key_index(topk[tid]) : -1;
      a.topk_score[item * K + tid] = v ? key_score(topk[tid]) : 0;
      a.topk_mis[item * K + tid] = v ? key_mis(topk[tid]) : 0;
    }
    if (tid == 0) a.pick[item] = pk;
  } else {
    if (a.log && tid < a.log_stride) {
      int32_t* e = a.log + ((int64_t)slot * a.n_patches + patch) * a.log_stride;
      int val;
      if (tid == 0) val = pk;
      else if (tid == 1) val = key_score(sel);
      else if (tid == 2) val = key_mis(sel);
      else if (tid == 3) val = CCW_LOG_FLAG_DONE;
      else val = (tid - 4 < Kp) ? key_index(topk[tid - 4]) : -1;
      e[tid] = val;
    }
    const int gdim[3] = {a.Gp[0], a.Gp[1], a.Gp[2]};
    paste_pattern<D>(a, pk, o, sg, gdim, a.overlay, off);
  }
}

// Standalone Inverse-DWT paste (ccw_idwt_paste): one CTA per batch element.
template <int D>
__global__ void __launch_bounds__(kThreads)
    k_idwt_paste(const __grid_constant__ SearchArgs a, const int32_t* picks,
                 const int32_t* origins, uint8_t* grid, int gx, int gy, int gz) {
  const int b = blockIdx.x;
  const int pk = picks[b];
  if (pk < 0 || pk >= a.P) {
    if (threadIdx.x == 0) atomicOr(a.status, kStatusBadCode);
    return;
  }
  const int o[3] = {origins[3 * b], origins[3 * b + 1], (D == 3) ? origins[3 * b + 2] : 0};
  const int gdim[3] = {gx, gy, gz};
  const int off[3] = {0, 0, 0};
  paste_pattern<D>(a, pk, o, grid, gdim, nullptr, off);
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
template <int D, int MODE>
static cudaError_t launch_search_t(const SearchArgs& a, int smem, cudaStream_t st) {
  auto fn = k_search<D, MODE>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.n_tiles, a.n_items);
  fn<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_search(int d, int mode, const SearchArgs& a, int smem, cudaStream_t st) {
  if (d == 2) {
    if (mode == kModeSim) return launch_search_t<2, kModeSim>(a, smem, st);
    if (mode == kModeSearch) return launch_search_t<2, kModeSearch>(a, smem, st);
    return launch_search_t<2, kModeMap>(a, smem, st);
  }
  if (mode == kModeSim) return launch_search_t<3, kModeSim>(a, smem, st);
  if (mode == kModeSearch) return launch_search_t<3, kModeSearch>(a, smem, st);
  return launch_search_t<3, kModeMap>(a, smem, st);
}

cudaError_t launch_idwt_paste(int d, const SearchArgs& a, int B, const int32_t* picks,
                              const int32_t* origins, uint8_t* grid, const int gdim[3],
                              cudaStream_t st) {
  if (d == 2)
    k_idwt_paste<2><<<B, kThreads, 0, st>>>(a, picks, origins, grid, gdim[0], gdim[1], gdim[2]);
  else
    k_idwt_paste<3><<<B, kThreads, 0, st>>>(a, picks, origins, grid, gdim[0], gdim[1], gdim[2]);
  return cudaGetLastError();
}

}  // namespace ccw
