// eval.cu -- pattern-reproduction statistics of realizations on the GPU
// (the validation of Sec. 5.2-5.3: facies proportions, indicator
// variograms along the axes, and histograms of w x w patterns at several
// mode-downsampled resolutions for the ANODI-style comparison). Integer
// counts throughout; the variogram is a ratio of two exact counts.
#include <algorithm>
#include <cstdio>

#include "ccw_internal.cuh"

namespace ccw {

// Facies counts of every realization: out[r][f] += cells of facies f.
__global__ void k_eval_counts(const uint8_t* __restrict__ real, int64_t vol, int F,
                              unsigned long long* __restrict__ out) {
  __shared__ unsigned int loc[8];
  const int r = blockIdx.y;
  if (threadIdx.x < 8) loc[threadIdx.x] = 0;
  __syncthreads();
  const uint8_t* src = real + (int64_t)r * vol;
  unsigned int c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < vol;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int v = src[i];
#pragma unroll
    for (int f = 0; f < 8; ++f) c[f] += (v == f);
  }
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (f >= F) break;
    const unsigned int s = __reduce_add_sync(0xffffffffu, c[f]);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(&loc[f], s);
  }
  __syncthreads();
  if (threadIdx.x < F && loc[threadIdx.x])
    atomicAdd(&out[r * F + threadIdx.x], (unsigned long long)loc[threadIdx.x]);
}

// Indicator variogram numerators: out[r][l] += #{x : [v(x) = f] != [v(x + h_l e_axis) = f]}
// over the pairs inside the grid.
__global__ void k_eval_variogram(const uint8_t* __restrict__ real, int nx, int ny, int nz, int f,
                                 int axis, const int* __restrict__ lags, int n_lags,
                                 unsigned long long* __restrict__ out) {
  const int r = blockIdx.y;
  const int64_t vol = (int64_t)nx * ny * nz;
  const uint8_t* src = real + (int64_t)r * vol;
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? nx : (int64_t)nx * ny);
  const int n_axis = axis == 0 ? nx : (axis == 1 ? ny : nz);
  for (int l = 0; l < n_lags; ++l) {
    const int h = lags[l];
    unsigned int c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < vol;
         i += (int64_t)gridDim.x * blockDim.x) {
      const int coord = (int)(axis == 0 ? i % nx : (axis == 1 ? (i / nx) % ny : i / ((int64_t)nx * ny)));
      if (h < 0 || coord + h >= n_axis) continue;   // negative lags count nothing
      c += ((src[i] == f) != (src[i + h * stride] == f));
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&out[(int64_t)r * n_lags + l], (unsigned long long)c);
  }
}

// Mode downsampling by k (2D): the most frequent facies of every k x k block,
// ties to the lower code.
__global__ void k_eval_mode(const uint8_t* __restrict__ real, int nx, int ny, int k, int F,
                            uint8_t* __restrict__ out, int mx, int my) {
  const int r = blockIdx.y;
  const int64_t n = (int64_t)mx * my;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int bx = (int)(i % mx), by = (int)(i / mx);
    int c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint8_t* src = real + (int64_t)r * nx * ny;
    for (int y = 0; y < k; ++y)
      for (int x = 0; x < k; ++x) {
        const int v = src[(bx * k + x) + (int64_t)nx * (by * k + y)];
#pragma unroll
        for (int f = 0; f < 8; ++f) c[f] += (v == f);
      }
    int best = 0;
#pragma unroll
    for (int f = 1; f < 8; ++f)
      if (f < F && c[f] > c[best]) best = f;
    out[(int64_t)r * n + i] = (uint8_t)best;
  }
}

// Histogram of the w x w patterns (2D), each encoded base F row by row:
// hist[code] += 1 over every pattern position of every realization.
__global__ void k_eval_patterns(const uint8_t* __restrict__ real, int nx, int ny, int w, int F,
                                unsigned int* __restrict__ hist) {
  const int r = blockIdx.y;
  const int px = nx - w + 1, py = ny - w + 1;
  const int64_t n = (int64_t)px * py;
  const uint8_t* src = real + (int64_t)r * nx * ny;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x0 = (int)(i % px), y0 = (int)(i / px);
    uint32_t code = 0;
    for (int dy = 0; dy < w; ++dy)
      for (int dx = 0; dx < w; ++dx)
        code = code * (uint32_t)F + src[(x0 + dx) + (int64_t)nx * (y0 + dy)];
    atomicAdd(&hist[code], 1u);
  }
}

}  // namespace ccw

using namespace ccw;

namespace {
thread_local char g_eval_err[256] = "";
int eval_fail(int code, const char* msg) {
  snprintf(g_eval_err, sizeof(g_eval_err), "%s", msg);
  return code;
}
dim3 eval_grid(int64_t n, int n_real) {
  return dim3((unsigned)std::min<int64_t>((n + 255) / 256, 1024), (unsigned)n_real);
}
}  // namespace

extern "C" {

int ccw_eval_proportions(const uint8_t* real_dev, int32_t n_real, const int32_t dims[3],
                         int32_t n_facies, uint64_t* counts_dev, void* stream) {
  if (!real_dev || !counts_dev || !dims) return eval_fail(CCW_EINVAL, "NULL argument");
  if (n_real < 1 || n_real > 65535 || n_facies < 2 || n_facies > 8)
    return eval_fail(CCW_EINVAL, "bad n_real or n_facies");
  const int64_t vol = (int64_t)dims[0] * dims[1] * dims[2];
  if (vol <= 0) return eval_fail(CCW_EINVAL, "bad dims");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(counts_dev, 0, sizeof(uint64_t) * n_real * n_facies, st) != cudaSuccess)
    return eval_fail(CCW_ECUDA, "memset");
  k_eval_counts<<<eval_grid(vol, n_real), 256, 0, st>>>(
      real_dev, vol, n_facies, reinterpret_cast<unsigned long long*>(counts_dev));
  return cudaGetLastError() == cudaSuccess ? CCW_OK : eval_fail(CCW_ECUDA, "kernel launch");
}

int ccw_eval_variogram(const uint8_t* real_dev, int32_t n_real, const int32_t dims[3],
                       int32_t facies, int32_t axis, const int32_t* lags_dev, int32_t n_lags,
                       uint64_t* mismatch_dev, void* stream) {
  if (!real_dev || !mismatch_dev || !dims || (n_lags > 0 && !lags_dev))
    return eval_fail(CCW_EINVAL, "NULL argument");
  if (n_real < 1 || n_real > 65535 || axis < 0 || axis > 2 || n_lags < 0)
    return eval_fail(CCW_EINVAL, "bad n_real, axis or n_lags");
  const int64_t vol = (int64_t)dims[0] * dims[1] * dims[2];
  if (vol <= 0) return eval_fail(CCW_EINVAL, "bad dims");
  cudaStream_t st = (cudaStream_t)stream;
  if (n_lags == 0) return CCW_OK;
  if (cudaMemsetAsync(mismatch_dev, 0, sizeof(uint64_t) * n_real * n_lags, st) != cudaSuccess)
    return eval_fail(CCW_ECUDA, "memset");
  k_eval_variogram<<<eval_grid(vol, n_real), 256, 0, st>>>(
      real_dev, dims[0], dims[1], dims[2], facies, axis, lags_dev, n_lags,
      reinterpret_cast<unsigned long long*>(mismatch_dev));
  return cudaGetLastError() == cudaSuccess ? CCW_OK : eval_fail(CCW_ECUDA, "kernel launch");
}

int ccw_eval_patterns(const uint8_t* real_dev, int32_t n_real, const int32_t dims[3],
                      int32_t n_facies, int32_t down, int32_t w, uint8_t* scratch_dev,
                      uint32_t* hist_dev, void* stream) {
  if (!real_dev || !hist_dev || !dims) return eval_fail(CCW_EINVAL, "NULL argument");
  if (dims[2] != 1) return eval_fail(CCW_EINVAL, "pattern histograms are 2D");
  if (n_real < 1 || n_real > 65535 || n_facies < 2 || n_facies > 8 || down < 1 || w < 1)
    return eval_fail(CCW_EINVAL, "bad n_real, n_facies, down or w");
  double bins = 1.0;
  for (int i = 0; i < w * w; ++i) bins *= n_facies;
  if (bins > (double)(1 << 26)) return eval_fail(CCW_EINVAL, "n_facies^(w*w) > 2^26 bins");
  const int mx = dims[0] / down, my = dims[1] / down;
  if (mx < w || my < w) return eval_fail(CCW_EINVAL, "grid smaller than the pattern");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(hist_dev, 0, sizeof(uint32_t) * (size_t)bins, st) != cudaSuccess)
    return eval_fail(CCW_ECUDA, "memset");
  const uint8_t* src = real_dev;
  if (down > 1) {
    if (!scratch_dev) return eval_fail(CCW_EINVAL, "down > 1 needs scratch_dev");
    k_eval_mode<<<eval_grid((int64_t)mx * my, n_real), 256, 0, st>>>(
        real_dev, dims[0], dims[1], down, n_facies, scratch_dev, mx, my);
    src = scratch_dev;
  }
  k_eval_patterns<<<eval_grid((int64_t)mx * my, n_real), 256, 0, st>>>(src, mx, my, w, n_facies,
                                                                       hist_dev);
  return cudaGetLastError() == cudaSuccess ? CCW_OK : eval_fail(CCW_ECUDA, "kernel launch");
}

const char* ccw_eval_last_error(void) { return g_eval_err; }

}  // extern "C"
