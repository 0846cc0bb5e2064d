// prepare.cu -- training-image preparation (Algorithm 1, line 2: DWT of the
// TI at level J), the hard-data overlay and the final crop of the simulation
// grid.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include <algorithm>

#include "ccw_internal.cuh"

namespace ccw {

// Copy the TI into its cropped buffer (dims multiples of s) and flag codes
// >= F.
__global__ void k_crop_ti(const uint8_t* __restrict__ src, int sx, int sy, uint8_t* __restrict__ dst,
                          int nx, int ny, int nz, int F, int* status) {
  const int64_t total = (int64_t)nx * ny * nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const int y = (int)((i / nx) % ny);
    const int z = (int)(i / ((int64_t)nx * ny));
    const uint8_t v = src[x + (int64_t)sx * (y + (int64_t)sy * z)];
    if (v >= F) atomicOr(status, kStatusBadCode);
    dst[i] = v;
  }
}

// The cropped TI inside a border of (bx, by, bz) cells of 255: the fine TI
// that the hard-data checks read, so that a datum of the virtual template
// whose position falls outside the TI never matches.
__global__ void k_pad_ti(const uint8_t* __restrict__ ti, int nx, int ny, int nz,
                         uint8_t* __restrict__ dst, int px, int py, int pz, int bx, int by,
                         int bz) {
  const int64_t total = (int64_t)px * py * pz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % px) - bx;
    const int y = (int)((i / px) % py) - by;
    const int z = (int)(i / ((int64_t)px * py)) - bz;
    const bool in = x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz;
    dst[i] = in ? ti[x + (int64_t)nx * (y + (int64_t)ny * z)] : (uint8_t)CCW_UNKNOWN;
  }
}

// Forward scaled Haar of one s^d block in place (the layout inverted by
// haar_block_inverse in search.cu): level j = 1..J, axes x, y, z; samples
// 2^(j-1) apart are replaced by their sum (lower position) and difference
// (upper position).
template <int D>
__device__ void haar_block_forward(int* v, int s, int J) {
  const int sz = (D == 3) ? s : 1;
  for (int j = 1; j <= J; ++j) {
    const int h = 1 << (j - 1);
    for (int a = 0; a < D; ++a) {
      const int stride = (a == 0) ? 1 : (a == 1 ? s : s * s);
      const int hx = (a == 0) ? 2 * h : h, hy = (a == 1) ? 2 * h : h,
                hz = (D == 3) ? ((a == 2) ? 2 * h : h) : 1;
      for (int z = 0; z < sz; z += hz)
        for (int y = 0; y < s; y += hy)
          for (int x = 0; x < s; x += hx) {
            const int p = x + s * (y + s * z), q = p + h * stride;
            const int lo = v[p], hi = v[q];
            v[p] = lo + hi;
            v[q] = lo - hi;
          }
    }
  }
}

// One thread per level-J block: facies counts (the level-J approximation of
// each indicator image, facies 0..F-2), the code sum (approximation of the
// code image) and the block's full J-level Haar coefficients of the codes.
template <int D>
__global__ void k_ti_pyramid(const uint8_t* __restrict__ ti, int nx, int ny, int ncx, int ncy,
                             int ncz, int s, int J, int F, float* __restrict__ planes, int px,
                             int16_t* __restrict__ pyr) {
  const int64_t ncv = (int64_t)ncx * ncy * ncz;
  const int64_t plane_vol = (int64_t)px * ncy * ncz;
  const int sd = (D == 3) ? s * s * s : s * s;
  const int sz = (D == 3) ? s : 1;
  int v[256];
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < ncv;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int bx = (int)(b % ncx);
    const int by = (int)((b / ncx) % ncy);
    const int bz = (int)(b / ((int64_t)ncx * ncy));
    int counts[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int csum = 0;
    for (int cz = 0; cz < sz; ++cz)
      for (int cy = 0; cy < s; ++cy)
        for (int cx = 0; cx < s; ++cx) {
          const int gx = s * bx + cx, gy = s * by + cy, gz = (D == 3) ? s * bz + cz : 0;
          const int c = ti[gx + (int64_t)nx * (gy + (int64_t)ny * gz)];
          v[cx + s * (cy + s * cz)] = c;
          csum += c;
#pragma unroll
          for (int f = 0; f < 8; ++f) counts[f] += (c == f);
        }
    const int64_t pb = bx + (int64_t)px * (by + (int64_t)ncy * bz);
    for (int f = 0; f < F - 1; ++f) planes[f * plane_vol + pb] = (float)counts[f];
    planes[(int64_t)(F - 1) * plane_vol + pb] = (float)csum;
    haar_block_forward<D>(v, s, J);
    int16_t* dst = pyr + b * sd;
    for (int c = 0; c < sd; ++c) dst[c] = (int16_t)v[c];
  }
}

// Hard-data overlay in grid coordinates; a cell with two hard data keeps the
// smaller code (byte-wise atomic minimum by compare-and-swap on the word).
__global__ void k_hd_overlay(const int32_t* __restrict__ cells, const uint8_t* __restrict__ vals,
                             int n, int d, int gx, int gy, int gz, int F, uint8_t* overlay,
                             int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int x = cells[i * d], y = cells[i * d + 1], z = (d == 3) ? cells[i * d + 2] : 0;
  const unsigned v = vals[i];
  if (x < 0 || y < 0 || z < 0 || x >= gx || y >= gy || z >= gz || v >= (unsigned)F) {
    atomicOr(status, kStatusBadCode);
    return;
  }
  const int64_t cell = x + (int64_t)gx * (y + (int64_t)gy * z);
  unsigned int* word = reinterpret_cast<unsigned int*>(overlay + (cell & ~(int64_t)3));
  const int sh = (int)(cell & 3) * 8;
  unsigned int old = *word;
  for (int it = 0; it < (1 << 20); ++it) {
    const unsigned cur = (old >> sh) & 0xFFu;
    if (v >= cur) return;
    const unsigned int nw = (old & ~(0xFFu << sh)) | (v << sh);
    const unsigned int prev = atomicCAS(word, old, nw);
    if (prev == old) return;
    old = prev;
  }
  atomicOr(status, kStatusTimeout);
}

// Crop the padded grids of n_real realizations into the caller's output,
// undoing each realization's path mirroring (Algorithm 1, line 3): one CTA
// per output row at a time (rows row0 .. row1 - 1 of the gy * gz rows of
// every realization), 32-bit words when every row start is aligned.
__global__ void k_crop_out(const uint8_t* __restrict__ sg, int64_t gp_vol, int gpx, int gpy,
                           uint8_t* __restrict__ out, int gx, int gy, int gz, int d, int gpz,
                           int path_random, uint64_t seed, int real_base, int vec, int row0,
                           int row1) {
  const int slot = blockIdx.y;
  const uint32_t r = (uint32_t)(real_base + slot);
  const uint32_t flips = path_random ? (draw_word(seed, r, 0u, 1u) & ((1u << d) - 1u)) : 0u;
  const int ox = (flips & 1u) ? gpx - gx : 0;
  const int oy = (flips & 2u) ? gpy - gy : 0;
  const int oz = (flips & 4u) ? gpz - gz : 0;
  const int rows = gy * gz;
  const uint8_t* src = sg + (int64_t)slot * gp_vol;
  uint8_t* dst = out + (int64_t)slot * gx * rows;
  const bool words = vec && ((ox & 3) == 0);
  for (int row = row0 + blockIdx.x; row < row1 && row < rows; row += gridDim.x) {
    const int y = row % gy, z = row / gy;
    const uint8_t* s = src + ox + (int64_t)gpx * ((y + oy) + (int64_t)gpy * (z + oz));
    uint8_t* o = dst + (int64_t)row * gx;
    if (words) {
      const uint32_t* s4 = reinterpret_cast<const uint32_t*>(s);
      uint32_t* o4 = reinterpret_cast<uint32_t*>(o);
      for (int i = threadIdx.x; i < gx / 4; i += blockDim.x) o4[i] = __ldg(s4 + i);
    } else {
      for (int i = threadIdx.x; i < gx; i += blockDim.x) o[i] = __ldg(s + i);
    }
  }
}

// The 8-shift view of the linearised level-J planes used by the tensor-core
// CCF. Plane p is read as a line lin_p[x + px8 * y] = plane p at (x, y),
// 0 for x >= nc0 or y >= nc1; z8[p][q][r][e] = lin_p[8 q + r + e] (16-bit,
// exact for the integer counts). With this copy the im2col matrix of any
// 128 consecutive line positions and 16 consecutive taps is a plain strided
// view (8 x 8 core matrices 128 bytes apart along both the candidate and the
// tap direction).
template <typename Th>
__global__ void k_z8(const float* __restrict__ planes, int px, int64_t plane_vol, int nc0, int nc1,
                     int px8, int64_t nq, int nplanes, Th* __restrict__ z8) {
  const int64_t per = nq * 64;
  const int64_t total = per * nplanes;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / per);
    const int64_t rem = i - p * per;
    const int64_t q = rem >> 6;
    const int r = (int)((rem >> 3) & 7), e = (int)(rem & 7);
    const int64_t L = 8 * q + r + e;
    const int64_t x = L % px8, y = L / px8;
    float v = 0.f;
    if (x < nc0 && y < nc1) v = planes[p * plane_vol + x + (int64_t)px * y];
    if constexpr (sizeof(Th) == 2 && std::is_same<Th, __half>::value)
      z8[i] = __float2half_rn(v);
    else
      z8[i] = __float2bfloat16_rn(v);
  }
}

// Level-J planes of one phase of the all-shift candidates (2D): block (ux,
// uy) covers fine cells (ph0 + s ux + bx, ph1 + s uy + by), bx, by < s, of
// the cropped TI; planes [F][nc1][px]: counts of facies 0..F-2, then the
// code sums (the layout of the decimated planes).
__global__ void k_phase_planes(const uint8_t* __restrict__ ti, int nx, int s, int F, int ph0,
                               int ph1, int nc0, int nc1, float* __restrict__ planes, int px,
                               int64_t plane_vol) {
  const int64_t nb = (int64_t)nc0 * nc1;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int ux = (int)(b % nc0), uy = (int)(b / nc0);
    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int code = 0;
    for (int by = 0; by < s; ++by)
      for (int bx = 0; bx < s; ++bx) {
        const int v = ti[(ph0 + s * ux + bx) + (int64_t)nx * (ph1 + s * uy + by)];
        code += v;
#pragma unroll
        for (int f = 0; f < 8; ++f) cnt[f] += (v == f);
      }
    const int64_t o = ux + (int64_t)px * uy;
#pragma unroll
    for (int f = 0; f < 7; ++f)
      if (f < F - 1) planes[f * plane_vol + o] = (float)cnt[f];
    planes[(int64_t)(F - 1) * plane_vol + o] = (float)code;
  }
}

cudaError_t launch_phase_planes(const uint8_t* ti, int nx, int s, int F, int ph0, int ph1, int nc0,
                                int nc1, float* planes, int px, int64_t plane_vol,
                                cudaStream_t st) {
  const int64_t nb = (int64_t)nc0 * nc1;
  const int blocks = (int)std::min<int64_t>((nb + 255) / 256, 152 * 8);
  k_phase_planes<<<blocks, 256, 0, st>>>(ti, nx, s, F, ph0, ph1, nc0, nc1, planes, px, plane_vol);
  return cudaGetLastError();
}

cudaError_t launch_z8(const float* planes, int px, int64_t plane_vol, int nc0, int nc1, int px8,
                      int64_t nq, int nplanes, void* z8_f16, void* z8_bf16, cudaStream_t st) {
  const int64_t total = nq * 64 * nplanes;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
  k_z8<__half><<<blocks, 256, 0, st>>>(planes, px, plane_vol, nc0, nc1, px8, nq, nplanes,
                                       (__half*)z8_f16);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_z8<__nv_bfloat16><<<blocks, 256, 0, st>>>(planes, px, plane_vol, nc0, nc1, px8, nq, nplanes,
                                              (__nv_bfloat16*)z8_bf16);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
cudaError_t launch_crop_ti(const uint8_t* src, const int sdims[3], uint8_t* dst, const int n[3],
                           int F, int* status, cudaStream_t st) {
  const int64_t total = (int64_t)n[0] * n[1] * n[2];
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_crop_ti<<<blocks, 256, 0, st>>>(src, sdims[0], sdims[1], dst, n[0], n[1], n[2], F, status);
  return cudaGetLastError();
}

cudaError_t launch_pad_ti(const uint8_t* ti, const int n[3], uint8_t* dst, const int tp[3],
                          const int border[3], cudaStream_t st) {
  const int64_t total = (int64_t)tp[0] * tp[1] * tp[2];
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_pad_ti<<<blocks, 256, 0, st>>>(ti, n[0], n[1], n[2], dst, tp[0], tp[1], tp[2], border[0],
                                   border[1], border[2]);
  return cudaGetLastError();
}

cudaError_t launch_ti_pyramid(int d, const uint8_t* ti, const int n[3], const int nc[3], int s,
                              int J, int F, float* planes, int px, int16_t* pyr,
                              cudaStream_t st) {
  const int64_t ncv = (int64_t)nc[0] * nc[1] * nc[2];
  const int blocks = (int)std::min<int64_t>((ncv + 127) / 128, 152 * 16);
  if (d == 3)
    k_ti_pyramid<3><<<blocks, 128, 0, st>>>(ti, n[0], n[1], nc[0], nc[1], nc[2], s, J, F, planes,
                                            px, pyr);
  else
    k_ti_pyramid<2><<<blocks, 128, 0, st>>>(ti, n[0], n[1], nc[0], nc[1], nc[2], s, J, F, planes,
                                            px, pyr);
  return cudaGetLastError();
}

cudaError_t launch_hd_overlay(const int32_t* cells, const uint8_t* vals, int n, int d,
                              const int g[3], int F, uint8_t* overlay, int* status,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_hd_overlay<<<(n + 255) / 256, 256, 0, st>>>(cells, vals, n, d, g[0], g[1], g[2], F, overlay,
                                                status);
  return cudaGetLastError();
}

cudaError_t launch_crop_out(const uint8_t* sg, int64_t gp_vol, const int gp[3], uint8_t* out,
                            const int g[3], int d, int n_real, int path_random, uint64_t seed,
                            int real_base, cudaStream_t st, int row0, int row1) {
  if (row1 < 0) row1 = g[1] * g[2];
  const int rows = row1 - row0;
  if (rows <= 0 || n_real <= 0) return cudaSuccess;
  // word copies need 4-aligned row starts in both arrays
  const int vec = ((g[0] | gp[0]) & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 3) == 0 &&
                  (reinterpret_cast<uintptr_t>(sg) & 3) == 0;
  const int bx = std::min(rows, 64);
  const int threads = vec ? std::min(256, std::max(32, (g[0] / 4 + 31) / 32 * 32))
                          : std::min(256, std::max(32, (g[0] + 31) / 32 * 32));
  for (int r0 = 0; r0 < n_real; r0 += 65535) {
    const int nr = std::min(65535, n_real - r0);
    dim3 grid(bx, nr);
    k_crop_out<<<grid, threads, 0, st>>>(sg + (int64_t)r0 * gp_vol, gp_vol, gp[0], gp[1],
                                         out + (int64_t)r0 * g[0] * rows, g[0], g[1], g[2], d,
                                         gp[2], path_random, seed, real_base + r0, vec, row0,
                                         row1);
  }
  return cudaGetLastError();
}

}  // namespace ccw
