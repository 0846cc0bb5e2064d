// device_util.cuh -- device helpers shared by the kernels: reductions,
// mbarrier / TMA wrappers with bounded waits, the Inverse-DWT paste and the
// decoding of simulation items.
#pragma once

#include <cuda.h>

#include <utility>

#include "ccw_internal.cuh"

namespace ccw {

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (w < v) ? w : v;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while its predecessor in the
// stream runs; pdl_wait() blocks until the predecessor has completed and its
// memory is visible, pdl_trigger() lets the successor start launching.
// Both are no-ops for kernels launched without the attribute.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch `kernel` on `st`, with the programmatic stream-serialization
// attribute when `pdl` is set.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, int smem,
                              cudaStream_t st, bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// mbarrier and bulk-tensor copies (PTX ISA: mbarrier.*, cp.async.bulk.tensor)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity` of an mbarrier. Returns false when the
// iteration limit is reached (the caller records kStatusTimeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t max_iters = (1u << 22)) {
  for (uint32_t i = 0; i < max_iters; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 4D tiled bulk-tensor load (global -> shared), completion on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
      "r"(smem_u32(bar))
      : "memory");
}

struct PasteGeom {
  const int16_t* pyr;
  int nc0, nc1;      // level-J TI dims (x, y)
  int cd0, cd1;      // candidate grid dims (x, y)
  int Tj;
  uint8_t* grid;
  int g[3];          // grid dims
  int o[3];          // window origin in grid coordinates
};

// Visit the cells (qx, qy, qz) of a T^d window with consecutive threads on
// consecutive x (coalesced rows); indices advance without divisions.
// `lt` is the calling thread's index among the nthreads that share the work
// (threadIdx.x when the whole CTA does).
template <int D, typename Fn>
__device__ __forceinline__ void for_window(int T, int nthreads, int lt, Fn&& fn) {
  const int nrows = (D == 3) ? T * T : T;
  if (T <= nthreads) {
    const int rpi = nthreads / T;
    const int qx = lt % T, r0 = lt / T;
    if (r0 >= rpi) return;
    int qy = r0, qz = 0;
    while (qy >= T) {
      qy -= T;
      ++qz;
    }
    for (int row = r0; row < nrows; row += rpi) {
      fn(qx, qy, qz);
      qy += rpi;
      while (qy >= T) {
        qy -= T;
        ++qz;
      }
    }
  } else {
    for (int row = 0; row < nrows; ++row)
      for (int qx = lt; qx < T; qx += nthreads) fn(qx, row % T, row / T);
  }
}

// Copy the level-J blocks covered by candidate `pick` (Tj^d blocks of s^d
// coefficients, one contiguous run of Tj blocks per coarse row) into shared
// memory, ordered (ux fastest, then uy, uz). Needs a following barrier.
template <int D>
__device__ void stage_blocks(const PasteGeom& p, int pick, int J, int16_t* sm, int nthreads,
                             int lt) {
  const int s = 1 << J;
  const int sd = (D == 3) ? s * s * s : s * s;
  const int pcx = pick % p.cd0;
  const int pcy = (pick / p.cd0) % p.cd1;
  const int pcz = pick / (p.cd0 * p.cd1);
  const int Tj = p.Tj;
  const int nrows = (D == 3) ? Tj * Tj : Tj;
  const int run = Tj * sd;   // coefficients per coarse row
  if (sd % 4 == 0 && run / 4 <= nthreads) {
    // rows in parallel: thread (r0, k) copies 8-byte word k of rows r0,
    // r0 + rpp, ... (one division per thread)
    const int run4 = run / 4;
    const int rpp = nthreads / run4;
    const int r0 = lt / run4, k = lt % run4;
    if (r0 < rpp) {
      // up to 4 rows' words loaded before any is stored (latencies overlap)
      int uy = r0 % Tj, uz = r0 / Tj;
      for (int row = r0; row < nrows; row += 4 * rpp) {
        uint2 v[4];
        int rows_done = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (row + b * rpp < nrows) {
            const int16_t* src =
                p.pyr +
                ((int64_t)pcx + (int64_t)p.nc0 * ((pcy + uy) + (int64_t)p.nc1 * (pcz + uz))) * sd;
            v[b] = __ldg(reinterpret_cast<const uint2*>(src) + k);
            rows_done = b + 1;
          }
          uy += rpp;
          while (uy >= Tj) {
            uy -= Tj;
            ++uz;
          }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (b < rows_done)
            reinterpret_cast<uint2*>(sm + (int64_t)(row + b * rpp) * run)[k] = v[b];
      }
    }
  } else if (sd % 4 == 0) {
    const int run4 = run / 4;
    // fewer threads than 8-byte words per row: kBatch words per thread are
    // loaded before any is stored, so their latencies overlap
    constexpr int kBatch = 8;
    const int total = nrows * run4;
    for (int i0 = lt; i0 < total; i0 += kBatch * nthreads) {
      uint2 v[kBatch];
      int dst[kBatch];
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const int i = i0 + b * nthreads;
        dst[b] = -1;
        if (i < total) {
          const int row = i / run4, k = i % run4;
          const int uy = row % Tj, uz = row / Tj;
          const int16_t* src =
              p.pyr +
              ((int64_t)pcx + (int64_t)p.nc0 * ((pcy + uy) + (int64_t)p.nc1 * (pcz + uz))) * sd;
          v[b] = __ldg(reinterpret_cast<const uint2*>(src) + k);
          dst[b] = row * run4 + k;
        }
      }
#pragma unroll
      for (int b = 0; b < kBatch; ++b)
        if (dst[b] >= 0) reinterpret_cast<uint2*>(sm)[dst[b]] = v[b];
    }
  } else {
    for (int i = lt; i < nrows * run; i += nthreads) {
      const int row = i / run, k = i % run;
      const int uy = row % Tj, uz = row / Tj;
      const int16_t* src =
          p.pyr + ((int64_t)pcx + (int64_t)p.nc0 * ((pcy + uy) + (int64_t)p.nc1 * (pcz + uz))) * sd;
      sm[(int64_t)row * run + k] = __ldg(src + k);
    }
  }
}

// CTA-cooperative Inverse-DWT paste of candidate `pick` (Algorithm 1, lines
// 13-14). Each fine cell q of the pattern is the Haar expansion of Sec. 3.1
// evaluated at q: with s = 2^J, the scaled-Haar synthesis gives
//   s^d x(q) = cA_J + sum_{j=1..J} 2^(d (J - j)) sum_{b != 0} sign_{j,b}(q) Z_{j,b}
// where Z_{j,b} is the level-j detail coefficient of band b covering q and
// sign_{j,b}(q) is the product, over the axes of band b, of +1 (q in the
// lower half of its level-j cell along that axis) or -1 (upper half). In the
// per-block in-place layout Z_{j,b} sits at the cell's origin plus 2^(j-1)
// along every axis of b. Coefficients come from `staged` (stage_blocks) when
// given, else from global memory. Cells outside the grid are skipped. The
// caller re-imposes hard data afterwards (after a barrier).
template <int D>
__device__ void paste_pixels(const PasteGeom& p, int pick, int J, int nthreads, int lt,
                             const int16_t* staged = nullptr) {
  const int s = 1 << J;
  const int sd = (D == 3) ? s * s * s : s * s;
  const int pcx = pick % p.cd0;
  const int pcy = (pick / p.cd0) % p.cd1;
  const int pcz = pick / (p.cd0 * p.cd1);
  const int Tj = p.Tj;
  const int T = Tj * s;
  for_window<D>(T, nthreads, lt, [&](int qx, int qy, int qz) {
    const int gx = p.o[0] + qx, gy = p.o[1] + qy, gz = p.o[2] + qz;
    if (gx < 0 || gy < 0 || gz < 0 || gx >= p.g[0] || gy >= p.g[1] || gz >= p.g[2]) return;
    const int ux = qx >> J, uy = qy >> J, uz = qz >> J;
    const int cx = qx & (s - 1), cy = qy & (s - 1), cz = qz & (s - 1);
    const int16_t* blk =
        staged ? staged + (ux + Tj * (uy + Tj * uz)) * sd
               : p.pyr + ((int64_t)(pcx + ux) +
                          (int64_t)p.nc0 * ((pcy + uy) + (int64_t)p.nc1 * (pcz + uz))) * sd;
    int acc = blk[0];
    for (int j = 1; j <= J; ++j) {
      const int h = 1 << (j - 1);
      const int m = ~((1 << j) - 1);
      const int bx = cx & m, by = cy & m, bz = cz & m;
      const int sx = (cx & h) ? -1 : 1, sy = (cy & h) ? -1 : 1, sz = (cz & h) ? -1 : 1;
      const int f = 1 << (D * (J - j));
      for (int b = 1; b < (1 << D); ++b) {
        const int px = bx + ((b & 1) ? h : 0), py = by + ((b & 2) ? h : 0),
                  pz = bz + ((b & 4) ? h : 0);
        const int sign = ((b & 1) ? sx : 1) * ((b & 2) ? sy : 1) * ((b & 4) ? sz : 1);
        acc += f * sign * (int)blk[px + s * (py + s * pz)];
      }
    }
    p.grid[gx + (int64_t)p.g[0] * (gy + (int64_t)p.g[1] * gz)] = (uint8_t)(acc >> (D * J));
  });
}

// Inverse of the per-block scaled Haar analysis (Sec. 3.1) for a block of
// S^D coefficients in registers, in the in-place layout (level j pairs
// samples 2^(j-1) apart, sum at the lower, difference at the upper index,
// axes x, y, z in turn): the levels and axes in reverse order, each pair
// (l, d) back to ((l + d) / 2, (l - d) / 2), exact in integers.
template <int D, int S>
__device__ __forceinline__ void haar_block_inverse(int (&v)[(D == 3) ? S * S * S : S * S]) {
  constexpr int SZ = (D == 3) ? S : 1;
#pragma unroll
  for (int h = S / 2; h >= 1; h /= 2) {
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      const int stride = (a == 0) ? 1 : (a == 1 ? S : S * S);
      const int hx = (a == 0) ? 2 * h : h, hy = (a == 1) ? 2 * h : h,
                hz = (D == 3) ? ((a == 2) ? 2 * h : h) : 1;
#pragma unroll
      for (int z = 0; z < SZ; z += hz)
#pragma unroll
        for (int y = 0; y < S; y += hy)
#pragma unroll
          for (int x = 0; x < S; x += hx) {
            const int p = x + S * (y + S * z), q = p + h * stride;
            const int l = v[p], d = v[q];
            v[p] = (l + d) >> 1;   // l + d and l - d are even
            v[q] = (l - d) >> 1;
          }
    }
  }
}

// CTA-cooperative Inverse-DWT paste with one thread per level-J block of the
// drawn pattern (Algorithm 1, lines 13-14): the block's S^D coefficients
// from `staged` (stage_blocks), inverted in registers, written row by row
// (S-byte words when `aligned`: window origin and grid pitch multiples of S).
// For windows that lie inside the grid (simulation lattice).
template <int D, int S>
__device__ void paste_blocks(const PasteGeom& p, const int16_t* staged, int nthreads, int lt,
                             bool aligned) {
  constexpr int SD = (D == 3) ? S * S * S : S * S;
  constexpr int SZ = (D == 3) ? S : 1;
  const int Tj = p.Tj;
  const int nblk = (D == 3) ? Tj * Tj * Tj : Tj * Tj;
  for (int u = lt; u < nblk; u += nthreads) {
    const int ux = u % Tj, uy = (u / Tj) % Tj, uz = (D == 3) ? u / (Tj * Tj) : 0;
    int v[SD];
    const int16_t* blk = staged + u * SD;
#pragma unroll
    for (int i = 0; i < SD; ++i) v[i] = blk[i];
    haar_block_inverse<D, S>(v);
#pragma unroll
    for (int cz = 0; cz < SZ; ++cz)
#pragma unroll
      for (int cy = 0; cy < S; ++cy) {
        const int gx = p.o[0] + ux * S, gy = p.o[1] + uy * S + cy, gz = p.o[2] + uz * S + cz;
        uint8_t* row = p.grid + gx + (int64_t)p.g[0] * (gy + (int64_t)p.g[1] * gz);
        const int* r = v + S * (cy + S * cz);
        if (S == 4 && aligned) {
          *reinterpret_cast<uint32_t*>(row) = (uint32_t)(r[0] & 0xFF) |
                                              ((uint32_t)(r[1] & 0xFF) << 8) |
                                              ((uint32_t)(r[2] & 0xFF) << 16) |
                                              ((uint32_t)(r[3 % S] & 0xFF) << 24);
        } else if (S == 2 && aligned) {
          *reinterpret_cast<uint16_t*>(row) =
              (uint16_t)((r[0] & 0xFF) | ((r[1 % S] & 0xFF) << 8));
        } else {
#pragma unroll
          for (int cx = 0; cx < S; ++cx) row[cx] = (uint8_t)r[cx];
        }
      }
  }
}

// CTA-cooperative paste of the TI crop at fine origin c (an all-shift
// candidate; its level-J approximation and details reconstruct exactly
// this crop). `ti` is the cropped fine TI with row pitch tp0 (2D).
__device__ __forceinline__ void paste_crop2(const PasteGeom& p, const uint8_t* ti, int tp0,
                                            int fd0, int c, int T, int nthreads, int lt) {
  const int cx = c % fd0, cy = c / fd0;
  for_window<2>(T, nthreads, lt, [&](int qx, int qy, int) {
    const int gx = p.o[0] + qx, gy = p.o[1] + qy;
    if (gx < 0 || gy < 0 || gx >= p.g[0] || gy >= p.g[1]) return;
    p.grid[gx + (int64_t)p.g[0] * gy] = __ldg(ti + (cx + qx) + (int64_t)tp0 * (cy + qy));
  });
}

// Re-impose the hard data of a pasted window (event-record list, int2 .y =
// (window offset << 8) | code; virtual-template entries are skipped). Call
// after a barrier that follows the paste.
template <int D>
__device__ void paste_hard_data(const PasteGeom& p, const int2* hdl, int n_hd, int T,
                                int nthreads, int lt) {
  for (int k = lt; k < n_hd; k += nthreads) {
    const int e = hdl[k].y;
    if (e < 0) continue;   // kHdVirtual: outside the window
    const int q = e >> 8;
    const int qx = q % T, qy = (q / T) % T, qz = (D == 3) ? q / (T * T) : 0;
    const int gx = p.o[0] + qx, gy = p.o[1] + qy, gz = p.o[2] + qz;
    if (gx < 0 || gy < 0 || gz < 0 || gx >= p.g[0] || gy >= p.g[1] || gz >= p.g[2]) continue;
    p.grid[gx + (int64_t)p.g[0] * (gy + (int64_t)p.g[1] * gz)] = (uint8_t)(e & 0xFF);
  }
}

// Position of a simulation item (realization slot, patch) in its padded
// grid, with the path mirroring of its realization (Algorithm 1, line 3).
struct ItemPos {
  int group, slot, patch;
  uint32_t r, p;
  uint32_t flips;           // bit a: the path runs backwards along axis a
  int o[3], off[3];
  uint8_t* sg;              // this realization's padded grid
  const uint8_t* overlay;   // the group's hard data
  int G[3], Gp[3];
  int32_t* log;             // this patch's log record, or NULL
  uint8_t* counts;          // this patch's block-count record, or NULL
};

template <int D>
__device__ __forceinline__ ItemPos decode_sim_item(const WaveArgs& a, int item) {
  ItemPos it;
  const int4 v = a.items[item];
  it.group = v.x;
  it.slot = v.y;
  it.patch = v.z;
  const SimGroup& s = a.groups[it.group];
  const CallDev* c = a.call;
  it.r = (uint32_t)(s.real_base + it.slot);
  it.p = (uint32_t)it.patch;
  const uint32_t flips =
      c->path_random ? (draw_word(c->seed, it.r, 0u, 1u) & ((1u << D) - 1u)) : 0u;
  it.flips = flips;
  const int np0 = s.np[0], np1 = s.np[1];
  const int ip[3] = {it.patch % np0, (it.patch / np0) % np1, it.patch / (np0 * np1)};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    it.G[ax] = s.G[ax];
    it.Gp[ax] = s.Gp[ax];
    const bool f = (flips >> ax) & 1u;
    if (ax < D) {
      it.o[ax] = f ? it.Gp[ax] - a.ti.T - a.S * ip[ax] : a.S * ip[ax];
      it.off[ax] = f ? it.Gp[ax] - it.G[ax] : 0;
    } else {
      it.o[ax] = 0;
      it.off[ax] = 0;
    }
  }
  it.sg = s.sg + (int64_t)it.slot * s.gp_vol;
  it.overlay = s.overlay;
  it.log = s.log ? s.log + ((int64_t)it.slot * s.n_patches + it.patch) * c->log_stride : nullptr;
  it.counts = s.counts ? s.counts + ((int64_t)it.slot * s.n_patches + it.patch) * a.ti.F *
                                        ((D == 3) ? a.ti.Tj * a.ti.Tj * a.ti.Tj : a.ti.Tj * a.ti.Tj)
                       : nullptr;
  return it;
}

template <int D>
__device__ __forceinline__ PasteGeom sim_paste_geom(const WaveArgs& a, const ItemPos& it) {
  PasteGeom g;
  g.pyr = a.ti.pyr;
  g.nc0 = a.ti.nc[0];
  g.nc1 = a.ti.nc[1];
  g.cd0 = a.ti.cd[0];
  g.cd1 = a.ti.cd[1];
  g.Tj = a.ti.Tj;
  g.grid = it.sg;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    g.g[ax] = it.Gp[ax];
    g.o[ax] = it.o[ax];
  }
  return g;
}

}  // namespace ccw
