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
// ---------------------------------------------------------------------------
// Probability of connection (Sec. 5.3): the 4-connected components of the
// cells of facies f by union-find over cell labels. Every label points to a
// smaller-or-equal index of its component (roots point to themselves), so
// parent chains only descend and every find ends; a union links the larger
// root under the smaller one with atomicMin and retries from the new parent
// when another thread got there first. Loops carry an iteration cap as a
// safety net; a realization whose labelling hit it reports counts of
// 2^64 - 1.
// ---------------------------------------------------------------------------
constexpr int kUfCap = 1 << 24;

__device__ __forceinline__ int uf_find(const int* L, int x) {
  for (int i = 0; i < kUfCap; ++i) {
    const int p = *(volatile const int*)(L + x);
    if (p == x) return x;
    x = p;
  }
  return -1;
}

__device__ __forceinline__ bool uf_union(int* L, int a, int b) {
  for (int it = 0; it < kUfCap; ++it) {
    a = uf_find(L, a);
    b = uf_find(L, b);
    if (a < 0 || b < 0) return false;
    if (a == b) return true;
    if (a < b) {
      const int tmp = a;
      a = b;
      b = tmp;
    }
    const int old = atomicMin(L + a, b);
    if (old == a) return true;   // a was still a root: now under b
    a = old;
  }
  return false;
}

__global__ void k_cc_init(const uint8_t* __restrict__ real, int64_t vol, int f, int* lab) {
  const int64_t base = (int64_t)blockIdx.y * vol;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < vol;
       i += (int64_t)gridDim.x * blockDim.x)
    lab[base + i] = real[base + i] == f ? (int)i : -1;
}

__global__ void k_cc_merge(const uint8_t* __restrict__ real, int nx, int ny, int f, int* lab,
                           int* fail) {
  const int64_t vol = (int64_t)nx * ny;
  const uint8_t* rr = real + (int64_t)blockIdx.y * vol;
  int* L = lab + (int64_t)blockIdx.y * vol;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < vol;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (rr[i] != f) continue;
    const int x = (int)(i % nx), y = (int)(i / nx);
    bool ok = true;
    if (x > 0 && rr[i - 1] == f) ok &= uf_union(L, (int)i, (int)i - 1);
    if (y > 0 && rr[i - nx] == f) ok &= uf_union(L, (int)i, (int)(i - nx));
    if (!ok) atomicOr(fail + blockIdx.y, 1);
  }
}

__global__ void k_cc_flatten(int64_t vol, int* lab, int* fail) {
  int* L = lab + (int64_t)blockIdx.y * vol;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < vol;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (L[i] < 0) continue;
    const int r = uf_find(L, (int)i);
    if (r < 0) atomicOr(fail + blockIdx.y, 1);
    else L[i] = r;
  }
}

// pairs[r][l] = {cell pairs (c, c + h e_axis) both of facies f, of them in
// one component}; per-block counters in shared memory, then global.
__global__ void k_cc_pairs(const int* __restrict__ lab, int nx, int ny, int axis,
                           const int* __restrict__ lags, int n_lags,
                           unsigned long long* pairs) {
  extern __shared__ unsigned int cnt[];   // [n_lags][2]
  for (int i = threadIdx.x; i < 2 * n_lags; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const int64_t vol = (int64_t)nx * ny;
  const int* L = lab + (int64_t)blockIdx.y * vol;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < vol;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int li = L[i];
    if (li < 0) continue;
    const int x = (int)(i % nx), y = (int)(i / nx);
    for (int l = 0; l < n_lags; ++l) {
      const int h = lags[l];
      int64_t j;
      if (axis == 0) {
        if (x + h >= nx) continue;
        j = i + h;
      } else {
        if (y + h >= ny) continue;
        j = i + (int64_t)h * nx;
      }
      const int lj = L[j];
      if (lj < 0) continue;
      atomicAdd(&cnt[2 * l], 1u);
      if (lj == li) atomicAdd(&cnt[2 * l + 1], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * n_lags; i += blockDim.x)
    if (cnt[i]) atomicAdd(pairs + (int64_t)blockIdx.y * 2 * n_lags + i, (unsigned long long)cnt[i]);
}

__global__ void k_cc_mark_failed(const int* fail, int n_lags, unsigned long long* pairs) {
  const int r = blockIdx.x;
  if (!fail[r]) return;
  for (int i = threadIdx.x; i < 2 * n_lags; i += blockDim.x)
    pairs[(int64_t)r * 2 * n_lags + i] = ~0ull;
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

int ccw_eval_connectivity(const uint8_t* real_dev, int32_t n_real, const int32_t dims[3],
                          int32_t facies, int32_t axis, const int32_t* lags_dev, int32_t n_lags,
                          int32_t* labels_dev, uint64_t* pairs_dev, void* stream) {
  if (!real_dev || !dims || !labels_dev || !pairs_dev || (n_lags > 0 && !lags_dev))
    return eval_fail(CCW_EINVAL, "NULL argument");
  if (dims[2] != 1) return eval_fail(CCW_EINVAL, "the probability of connection is 2D");
  if (n_real < 1 || n_real > 65535 || axis < 0 || axis > 1 || n_lags < 0 || n_lags > 4096)
    return eval_fail(CCW_EINVAL, "bad n_real, axis or n_lags");
  const int64_t vol = (int64_t)dims[0] * dims[1];
  if (dims[0] <= 0 || dims[1] <= 0 || vol >= ((int64_t)1 << 31))
    return eval_fail(CCW_EINVAL, "bad dims (at most 2^31 - 1 cells)");
  if (n_lags == 0) return CCW_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // one give-up flag per realization, in the scratch after the labels
  int* fail = labels_dev + (int64_t)n_real * vol;
  if (cudaMemsetAsync(pairs_dev, 0, sizeof(uint64_t) * 2 * n_lags * n_real, st) != cudaSuccess ||
      cudaMemsetAsync(fail, 0, sizeof(int) * n_real, st) != cudaSuccess)
    return eval_fail(CCW_ECUDA, "memset");
  const dim3 grid = eval_grid(vol, n_real);
  k_cc_init<<<grid, 256, 0, st>>>(real_dev, vol, facies, labels_dev);
  k_cc_merge<<<grid, 256, 0, st>>>(real_dev, dims[0], dims[1], facies, labels_dev, fail);
  k_cc_flatten<<<grid, 256, 0, st>>>(vol, labels_dev, fail);
  k_cc_pairs<<<grid, 256, sizeof(unsigned int) * 2 * n_lags, st>>>(
      labels_dev, dims[0], dims[1], axis, lags_dev, n_lags,
      reinterpret_cast<unsigned long long*>(pairs_dev));
  k_cc_mark_failed<<<n_real, 256, 0, st>>>(fail, n_lags,
                                          reinterpret_cast<unsigned long long*>(pairs_dev));
  return cudaGetLastError() == cudaSuccess ? CCW_OK : eval_fail(CCW_ECUDA, "kernel launch");
}

const char* ccw_eval_last_error(void) { return g_eval_err; }

}  // extern "C"
