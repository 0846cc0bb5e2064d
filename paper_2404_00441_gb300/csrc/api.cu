// api.cu -- host side of the C ABI declared in include/ccw.h.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "ccw_internal.cuh"

namespace ccw {
// search.cu
int search_smem_bytes(int d, int nch, int Tj, int TjP);
void search_tiles(int d, const int cd[3], int tiles[3]);
cudaError_t launch_search(int d, int mode, const SearchArgs& a, int smem, cudaStream_t st);
cudaError_t launch_idwt_paste(int d, const SearchArgs& a, int B, const int32_t* picks,
                              const int32_t* origins, uint8_t* grid, const int gdim[3],
                              cudaStream_t st);
// prepare.cu
cudaError_t launch_crop_ti(const uint8_t* src, const int sdims[3], uint8_t* dst, const int n[3],
                           int F, int* status, cudaStream_t st);
cudaError_t launch_ti_pyramid(int d, const uint8_t* ti, const int n[3], const int nc[3], int s,
                              int J, int F, float* planes, int16_t* pyr, cudaStream_t st);
cudaError_t launch_hd_overlay(const int32_t* cells, const uint8_t* vals, int n, int d,
                              const int g[3], int F, uint8_t* overlay, int* status,
                              cudaStream_t st);
cudaError_t launch_crop_out(const uint8_t* sg, int64_t gp_vol, const int gp[3], uint8_t* out,
                            const int g[3], int d, int n_real, int path_random, uint64_t seed,
                            int real_base, cudaStream_t st);
}  // namespace ccw

using namespace ccw;

struct ccw_ti {
  int ndim, F, J, s, sd, T, O, Tj, TjP;
  int n[3], nc[3], cd[3];
  int64_t ncv, P;
  int device;
  uint8_t* d_ti;      // cropped fine TI
  float* d_planes;    // F planes: counts of facies 0..F-2, then code sums
  int16_t* d_pyr;     // [ncv][sd]
  int* d_status;      // device status word
};

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(CCW_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

std::atomic<int64_t> g_launches{0};

// profiling state
struct Profiler {
  std::mutex mu;
  bool enabled = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  unsigned long long* d_work = nullptr;
  int device = -1;
} g_prof;

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Fill the TI part of the kernel arguments.
void fill_ti_args(const ccw_ti* t, int score_mode, SearchArgs& a) {
  memset(&a, 0, sizeof(a));
  a.nch = score_mode == 0 ? t->F - 1 : 1;
  a.planes = t->d_planes + (score_mode == 0 ? 0 : (int64_t)(t->F - 1) * t->ncv);
  a.ti = t->d_ti;
  a.pyr = t->d_pyr;
  a.F = t->F;
  a.J = t->J;
  a.s = t->s;
  a.sd = t->sd;
  a.T = t->T;
  a.Tj = t->Tj;
  a.TjP = t->TjP;
  a.d = t->ndim;
  a.score_mode = score_mode;
  for (int i = 0; i < 3; ++i) {
    a.n[i] = t->n[i];
    a.nc[i] = t->nc[i];
    a.cd[i] = t->cd[i];
  }
  a.ncv = t->ncv;
  a.P = t->P;
  search_tiles(t->ndim, t->cd, a.tiles);
  a.n_tiles = a.tiles[0] * a.tiles[1] * a.tiles[2];
  a.status = t->d_status;
}

int check_score_bound(const ccw_ti* t, int score_mode) {
  // exact FP32 accumulation: every partial sum of integers stays below 2^24
  const int64_t Td = ipow(t->T, t->ndim);
  const int64_t bound = (score_mode == 0) ? (int64_t)(t->F - 1) * Td * t->sd
                                          : (int64_t)(t->F - 1) * (t->F - 1) * Td * t->sd;
  if (bound >= (int64_t)1 << 24)
    return fail(CCW_EINVAL,
                "score range %lld exceeds the exact FP32 bound 2^24 (lower T, J or F, or "
                "use the one-hot score)",
                (long long)bound);
  return CCW_OK;
}

// Launch the search kernel in chunks of at most 65535 items (grid.y limit),
// with profiling events around each launch when enabled.
int run_search(const ccw_ti* t, int mode, SearchArgs a, int n_items, int item_stride_sim,
               cudaStream_t st) {
  const int smem = search_smem_bytes(t->ndim, a.nch, t->Tj, t->TjP);
  std::unique_lock<std::mutex> lk(g_prof.mu);
  const bool prof = g_prof.enabled;
  if (prof && !g_prof.d_work) {
    if (cudaMalloc(&g_prof.d_work, 2 * sizeof(unsigned long long)) != cudaSuccess)
      return fail(CCW_ENOMEM, "profiling counters");
    cudaMemset(g_prof.d_work, 0, 2 * sizeof(unsigned long long));
  }
  a.work = prof ? g_prof.d_work : nullptr;
  lk.unlock();
  const int64_t tv = ipow(t->T, t->ndim);
  for (int i0 = 0; i0 < n_items; i0 += 65535) {
    SearchArgs c = a;
    c.n_items = std::min(65535, n_items - i0);
    if (mode == kModeSim) {
      c.items = a.items + i0;
    } else {
      c.de = a.de + (int64_t)i0 * tv;
      c.hd = a.hd ? a.hd + (int64_t)i0 * tv : nullptr;
      if (a.ctr) c.ctr = a.ctr + 2 * (int64_t)i0;
      if (a.topk_idx) {
        c.topk_idx = a.topk_idx + (int64_t)i0 * a.K;
        c.topk_score = a.topk_score + (int64_t)i0 * a.K;
        c.topk_mis = a.topk_mis + (int64_t)i0 * a.K;
      }
      if (a.pick) c.pick = a.pick + i0;
      if (a.map_score) c.map_score = a.map_score + (int64_t)i0 * t->P;
      if (a.map_mis) c.map_mis = a.map_mis + (int64_t)i0 * t->P;
    }
    (void)item_stride_sim;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, st);
    }
    cudaError_t e = launch_search(t->ndim, mode, c, smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "search kernel launch");
    ++g_launches;
    if (prof) {
      cudaEventRecord(e1, st);
      std::lock_guard<std::mutex> g(g_prof.mu);
      g_prof.events.emplace_back(e0, e1);
    }
  }
  return CCW_OK;
}

struct DevBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, st);
  }
  cudaError_t alloc(size_t bytes, cudaStream_t s) {
    st = s;
    return cudaMallocAsync(&p, bytes ? bytes : 16, s);
  }
};

}  // namespace

extern "C" {

const char* ccw_last_error(void) { return g_err; }

int64_t ccw_launch_count(void) { return g_launches.load(); }

int ccw_profile_enable(int32_t enable) {
  std::lock_guard<std::mutex> g(g_prof.mu);
  g_prof.enabled = enable != 0;
  return CCW_OK;
}

int ccw_profile_read(int64_t* launches, double* total_ms, double* cand_evals, double* macs) {
  std::lock_guard<std::mutex> g(g_prof.mu);
  double ms = 0.0;
  for (auto& pr : g_prof.events) {
    cudaEventSynchronize(pr.second);
    float t = 0.f;
    cudaEventElapsedTime(&t, pr.first, pr.second);
    ms += t;
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  if (launches) *launches = (int64_t)g_prof.events.size();
  if (total_ms) *total_ms = ms;
  g_prof.events.clear();
  unsigned long long w[2] = {0, 0};
  if (g_prof.d_work) {
    cudaMemcpy(w, g_prof.d_work, sizeof(w), cudaMemcpyDeviceToHost);
    cudaMemset(g_prof.d_work, 0, sizeof(w));
  }
  if (cand_evals) *cand_evals = (double)w[0];
  if (macs) *macs = (double)w[1];
  return CCW_OK;
}

int ccw_ti_prepare(const uint8_t* ti_dev, int32_t ndim, const int32_t dims[3], int32_t n_facies,
                   int32_t level, int32_t templ, int32_t overlap, void* stream, ccw_ti** out) {
  if (!out) return fail(CCW_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ti_dev || !dims) return fail(CCW_EINVAL, "ti_dev/dims is NULL");
  if (ndim != 2 && ndim != 3) return fail(CCW_EINVAL, "ndim must be 2 or 3 (got %d)", ndim);
  if (n_facies < 2 || n_facies > 8) return fail(CCW_EINVAL, "n_facies must be in [2, 8]");
  const int maxJ = ndim == 2 ? kMaxLevel2D : kMaxLevel3D;
  if (level < 0 || level > maxJ)
    return fail(CCW_EINVAL, "level must be in [0, %d] for %dD", maxJ, ndim);
  const int s = 1 << level;
  if (templ <= 0 || templ % s || overlap < 0 || overlap % s)
    return fail(CCW_EINVAL, "template and overlap must be non-negative multiples of 2^level");
  if (templ < 2 * overlap) return fail(CCW_EINVAL, "template must be at least 2 x overlap");
  if (dims[2] != 1 && ndim == 2) return fail(CCW_EINVAL, "dims[2] must be 1 in 2D");
  ccw_ti t;
  memset(&t, 0, sizeof(t));
  t.ndim = ndim;
  t.F = n_facies;
  t.J = level;
  t.s = s;
  t.sd = ndim == 2 ? s * s : s * s * s;
  t.T = templ;
  t.O = overlap;
  t.Tj = templ / s;
  t.TjP = 4 * ((t.Tj + 3) / 4);
  for (int a = 0; a < 3; ++a) {
    const int sa = a < ndim ? s : 1;
    if (dims[a] <= 0) return fail(CCW_EINVAL, "dims must be positive");
    t.nc[a] = dims[a] / sa;
    t.n[a] = t.nc[a] * sa;
    t.cd[a] = a < ndim ? t.nc[a] - t.Tj + 1 : 1;
    if (t.cd[a] <= 0) return fail(CCW_EINVAL, "template larger than the TI along axis %d", a);
  }
  t.ncv = (int64_t)t.nc[0] * t.nc[1] * t.nc[2];
  t.P = (int64_t)t.cd[0] * t.cd[1] * t.cd[2];
  if (t.P >= (1 << 24)) return fail(CCW_EINVAL, "more than 2^24 - 1 candidates");
  if (t.Tj > 255 * 4) return fail(CCW_EINVAL, "template too large");
  {
    int rc = check_score_bound(&t, 0);
    if (rc) return rc;
  }
  const int smem = search_smem_bytes(ndim, t.F - 1, t.Tj, t.TjP);
  if (smem > 227 * 1024)
    return fail(CCW_EUNSUPPORTED, "template too large for the shared-memory tile (%d B)", smem);
  cudaGetDevice(&t.device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nv = (int64_t)t.n[0] * t.n[1] * t.n[2];
  cudaError_t e;
  if ((e = cudaMalloc(&t.d_ti, nv)) != cudaSuccess ||
      (e = cudaMalloc(&t.d_planes, sizeof(float) * t.ncv * t.F)) != cudaSuccess ||
      (e = cudaMalloc(&t.d_pyr, sizeof(int16_t) * t.ncv * t.sd)) != cudaSuccess ||
      (e = cudaMalloc(&t.d_status, sizeof(int))) != cudaSuccess) {
    cudaFree(t.d_ti);
    cudaFree(t.d_planes);
    cudaFree(t.d_pyr);
    cudaFree(t.d_status);
    return fail(CCW_ENOMEM, "TI buffers: %s", cudaGetErrorString(e));
  }
  auto cleanup = [&]() {
    cudaFree(t.d_ti);
    cudaFree(t.d_planes);
    cudaFree(t.d_pyr);
    cudaFree(t.d_status);
  };
  cudaMemsetAsync(t.d_status, 0, sizeof(int), st);
  const int sdims[3] = {dims[0], dims[1], dims[2]};
  if ((e = launch_crop_ti(ti_dev, sdims, t.d_ti, t.n, t.F, t.d_status, st)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "crop kernel");
  }
  ++g_launches;
  if ((e = launch_ti_pyramid(ndim, t.d_ti, t.n, t.nc, s, level, t.F, t.d_planes, t.d_pyr, st)) !=
      cudaSuccess) {
    cleanup();
    return cuda_fail(e, "pyramid kernel");
  }
  ++g_launches;
  int status = 0;
  if ((e = cudaMemcpyAsync(&status, t.d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "prepare");
  }
  if (status) {
    cleanup();
    return fail(CCW_EINVAL, "training image holds codes >= n_facies");
  }
  ccw_ti* h = new ccw_ti(t);
  *out = h;
  return CCW_OK;
}

int ccw_ti_describe(const ccw_ti* t, ccw_ti_desc* out) {
  if (!t || !out) return fail(CCW_EINVAL, "NULL argument");
  out->ndim = t->ndim;
  out->n_facies = t->F;
  out->level = t->J;
  out->scale = t->s;
  out->templ = t->T;
  out->overlap = t->O;
  for (int a = 0; a < 3; ++a) {
    out->dims[a] = t->n[a];
    out->coarse[a] = t->nc[a];
    out->cand[a] = t->cd[a];
  }
  out->n_cand = t->P;
  return CCW_OK;
}

void ccw_ti_free(ccw_ti* t) {
  if (!t) return;
  cudaDeviceSynchronize();
  cudaFree(t->d_ti);
  cudaFree(t->d_planes);
  cudaFree(t->d_pyr);
  cudaFree(t->d_status);
  delete t;
}

int ccw_ti_export(const ccw_ti* t, int32_t what, void* dst, void* stream) {
  if (!t || !dst) return fail(CCW_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const void* src;
  size_t bytes;
  switch (what) {
    case 0:
      src = t->d_planes;
      bytes = sizeof(float) * t->ncv * (t->F - 1);
      break;
    case 1:
      src = t->d_planes + (int64_t)(t->F - 1) * t->ncv;
      bytes = sizeof(float) * t->ncv;
      break;
    case 2:
      src = t->d_pyr;
      bytes = sizeof(int16_t) * t->ncv * t->sd;
      break;
    case 3:
      src = t->d_ti;
      bytes = (size_t)t->n[0] * t->n[1] * t->n[2];
      break;
    default:
      return fail(CCW_EINVAL, "unknown export %d", what);
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "export copy");
  return CCW_OK;
}

int ccw_ti_status(const ccw_ti* t, void* stream, int32_t* status_out) {
  if (!t || !status_out) return fail(CCW_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, t->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  *status_out = v;
  return CCW_OK;
}

static int search_common(const ccw_ti* t, int mode, int32_t B, const uint8_t* de,
                         const uint8_t* hd, int32_t k, int32_t score_mode, uint64_t seed,
                         const uint32_t* ctr, int32_t* ti_idx, int32_t* ti_sc, int32_t* ti_mm,
                         int32_t* pick, int32_t* map_sc, int32_t* map_mm, void* stream) {
  if (!t) return fail(CCW_EINVAL, "ti is NULL");
  if (B < 0) return fail(CCW_EINVAL, "B must be >= 0");
  if (score_mode != 0 && score_mode != 1) return fail(CCW_EINVAL, "score_mode must be 0 or 1");
  if (int rc = check_score_bound(t, score_mode)) return rc;
  if (B == 0) return CCW_OK;
  if (!de) return fail(CCW_EINVAL, "de_dev is NULL");
  if (mode == kModeSearch) {
    if (k < 1 || k > CCW_MAX_TOPK) return fail(CCW_EINVAL, "k must be in [1, %d]", CCW_MAX_TOPK);
    if (!ctr || !ti_idx || !ti_sc || !ti_mm || !pick)
      return fail(CCW_EINVAL, "NULL output or counter");
  } else if (!map_sc) {
    return fail(CCW_EINVAL, "score_dev is NULL");
  }
  cudaStream_t st = (cudaStream_t)stream;
  SearchArgs a;
  fill_ti_args(t, score_mode, a);
  a.de = de;
  a.hd = hd;
  a.ctr = ctr;
  a.K = mode == kModeSearch ? k : 1;
  a.seed = seed;
  a.topk_idx = ti_idx;
  a.topk_score = ti_sc;
  a.topk_mis = ti_mm;
  a.pick = pick;
  a.map_score = map_sc;
  a.map_mis = map_mm;
  DevBuf part, cnt;
  if (mode == kModeSearch) {
    const int chunk = std::min<int>(B, 65535);
    if (part.alloc(sizeof(unsigned long long) * (size_t)chunk * a.n_tiles * a.K, st) !=
            cudaSuccess ||
        cnt.alloc(sizeof(unsigned int) * (size_t)chunk, st) != cudaSuccess)
      return fail(CCW_ENOMEM, "search scratch");
    cudaMemsetAsync(cnt.p, 0, sizeof(unsigned int) * (size_t)chunk, st);
    a.part = (unsigned long long*)part.p;
    a.counters = (unsigned int*)cnt.p;
  }
  return run_search(t, mode, a, B, 0, st);
}

int ccw_ccf_search(const ccw_ti* t, int32_t B, const uint8_t* de_dev, const uint8_t* hd_dev,
                   int32_t k, int32_t score_mode, uint64_t seed, const uint32_t* ctr_dev,
                   int32_t* topk_idx_dev, int32_t* topk_score_dev, int32_t* topk_mis_dev,
                   int32_t* pick_dev, void* stream) {
  return search_common(t, kModeSearch, B, de_dev, hd_dev, k, score_mode, seed, ctr_dev,
                       topk_idx_dev, topk_score_dev, topk_mis_dev, pick_dev, nullptr, nullptr,
                       stream);
}

// Scratch of ccw_ccf_search_noalloc: one array per device, part of the
// library image, so using it needs no allocation. Host code reaches it only
// through the device address looked up below; the symbol itself is a host
// stand-in that no kernel may be given.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CCW_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};   // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device; looked up once
// per device, on the first call made with that device current.
int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(CCW_EUNSUPPORTED, "device index %d", dev);
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CCW_OK;
}
}  // namespace

int ccw_ccf_search_noalloc(const ccw_ti* t, int32_t B, const uint8_t* de_dev,
                           const uint8_t* hd_dev, int32_t k, int32_t score_mode, uint64_t seed,
                           const uint32_t* ctr_dev, int32_t* topk_idx_dev,
                           int32_t* topk_score_dev, int32_t* topk_mis_dev, int32_t* pick_dev,
                           void* stream) {
  if (!t) return fail(CCW_EINVAL, "ti is NULL");
  if (B < 0) return fail(CCW_EINVAL, "B must be >= 0");
  if (score_mode != 0 && score_mode != 1) return fail(CCW_EINVAL, "score_mode must be 0 or 1");
  if (int rc = check_score_bound(t, score_mode)) return rc;
  if (k < 1 || k > CCW_MAX_TOPK) return fail(CCW_EINVAL, "k must be in [1, %d]", CCW_MAX_TOPK);
  if (B == 0) return CCW_OK;
  if (!de_dev || !ctr_dev || !topk_idx_dev || !topk_score_dev || !topk_mis_dev || !pick_dev)
    return fail(CCW_EINVAL, "NULL input, output or counter");
  SearchArgs a;
  fill_ti_args(t, score_mode, a);
  const int64_t chunk = std::min<int64_t>(B, 65535);
  const int64_t cnt_bytes = (chunk * (int64_t)sizeof(unsigned int) + 255) & ~(int64_t)255;
  const int64_t need = cnt_bytes + chunk * a.n_tiles * k * (int64_t)sizeof(unsigned long long);
  if (need > CCW_NOALLOC_SCRATCH_BYTES)
    return fail(CCW_EINVAL,
                "ccw_ccf_search_noalloc: B=%d with k=%d needs %lld scratch bytes, more than "
                "the %d-byte array; split the batch",
                B, k, (long long)need, CCW_NOALLOC_SCRATCH_BYTES);
  void* base = nullptr;
  if (int rc = noalloc_scratch(&base)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  a.de = de_dev;
  a.hd = hd_dev;
  a.ctr = ctr_dev;
  a.K = k;
  a.seed = seed;
  a.counters = (unsigned int*)base;
  a.part = (unsigned long long*)((unsigned char*)base + cnt_bytes);
  const int64_t tv = ipow(t->T, t->ndim);
  const int smem = search_smem_bytes(t->ndim, a.nch, t->Tj, t->TjP);
  for (int64_t i0 = 0; i0 < B; i0 += 65535) {
    SearchArgs c = a;
    c.n_items = (int)std::min<int64_t>(65535, B - i0);
    c.de = de_dev + i0 * tv;
    c.hd = hd_dev ? hd_dev + i0 * tv : nullptr;
    c.ctr = ctr_dev + 2 * i0;
    c.topk_idx = topk_idx_dev + i0 * k;
    c.topk_score = topk_score_dev + i0 * k;
    c.topk_mis = topk_mis_dev + i0 * k;
    c.pick = pick_dev + i0;
    cudaError_t e = cudaMemsetAsync(c.counters, 0, sizeof(unsigned int) * c.n_items, st);
    if (e != cudaSuccess) return cuda_fail(e, "scratch clear");
    e = launch_search(t->ndim, kModeSearch, c, smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "search kernel launch");
    ++g_launches;
  }
  return CCW_OK;
}

int ccw_ccf_map(const ccw_ti* t, int32_t B, const uint8_t* de_dev, const uint8_t* hd_dev,
                int32_t score_mode, int32_t* score_dev, int32_t* mis_dev, void* stream) {
  return search_common(t, kModeMap, B, de_dev, hd_dev, 1, score_mode, 0, nullptr, nullptr,
                       nullptr, nullptr, nullptr, score_dev, mis_dev, stream);
}

int ccw_idwt_paste(const ccw_ti* t, int32_t B, const int32_t* pick_dev,
                   const int32_t* dst_origin_dev, uint8_t* sg_dev, const int32_t sg_dims[3],
                   void* stream) {
  if (!t || !sg_dims) return fail(CCW_EINVAL, "NULL argument");
  if (B < 0) return fail(CCW_EINVAL, "B must be >= 0");
  if (B == 0) return CCW_OK;
  if (!pick_dev || !dst_origin_dev || !sg_dev) return fail(CCW_EINVAL, "NULL device pointer");
  for (int a = 0; a < 3; ++a)
    if (sg_dims[a] <= 0 || (a >= t->ndim && sg_dims[a] != 1))
      return fail(CCW_EINVAL, "bad sg_dims");
  SearchArgs a;
  fill_ti_args(t, 0, a);
  const int gd[3] = {sg_dims[0], sg_dims[1], sg_dims[2]};
  cudaError_t e = launch_idwt_paste(t->ndim, a, B, pick_dev, dst_origin_dev, sg_dev, gd,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "paste kernel");
  ++g_launches;
  return CCW_OK;
}

int ccw_simulate(const ccw_ti* t, const ccw_params* p, const int32_t* hd_cells_dev,
                 const uint8_t* hd_vals_dev, int32_t n_hd, uint64_t seed, uint8_t* out_dev,
                 int32_t* patch_log_dev, void* stream) {
  if (!t || !p || !out_dev) return fail(CCW_EINVAL, "NULL argument");
  const int d = t->ndim;
  if (p->ndim != d) return fail(CCW_EINVAL, "params ndim %d != TI ndim %d", p->ndim, d);
  if (p->topk < 1 || p->topk > CCW_MAX_TOPK)
    return fail(CCW_EINVAL, "topk must be in [1, %d]", CCW_MAX_TOPK);
  if (p->n_real < 1) return fail(CCW_EINVAL, "n_real must be >= 1");
  if (p->real_base < 0) return fail(CCW_EINVAL, "real_base must be >= 0");
  if (p->score_mode != 0 && p->score_mode != 1) return fail(CCW_EINVAL, "bad score_mode");
  if (p->precision != 0)
    return fail(CCW_EUNSUPPORTED, "precision %d is not available in this build", p->precision);
  if (p->path_random != 0 && p->path_random != 1) return fail(CCW_EINVAL, "bad path_random");
  for (int i = 0; i < 4; ++i)
    if (p->reserved[i]) return fail(CCW_EINVAL, "reserved fields must be 0");
  if (n_hd < 0 || (n_hd > 0 && (!hd_cells_dev || !hd_vals_dev)))
    return fail(CCW_EINVAL, "bad hard data");
  if (int rc = check_score_bound(t, p->score_mode)) return rc;
  int g[3], np_[3], gp[3];
  const int T = t->T, S = t->T - t->O;
  for (int a = 0; a < 3; ++a) {
    g[a] = p->grid[a];
    if (g[a] <= 0 || (a >= d && g[a] != 1)) return fail(CCW_EINVAL, "bad grid dims");
    if (a < d) {
      const int extra = g[a] > T ? g[a] - T : 0;
      np_[a] = 1 + (extra + S - 1) / S;
      gp[a] = T + (np_[a] - 1) * S;
    } else {
      np_[a] = 1;
      gp[a] = 1;
    }
  }
  const int64_t n_patches = (int64_t)np_[0] * np_[1] * np_[2];
  const int64_t gp_vol = (int64_t)gp[0] * gp[1] * gp[2];
  const int64_t g_vol = (int64_t)g[0] * g[1] * g[2];
  const int n_real = p->n_real;
  const int K = p->topk;

  // wavefront schedule: wave(p) = ix + 2 iy + 4 iz over the path index
  const int n_waves = (np_[0] - 1) + 2 * (np_[1] - 1) + 4 * (np_[2] - 1) + 1;
  std::vector<std::vector<int>> wave_patches(n_waves);
  for (int64_t pp = 0; pp < n_patches; ++pp) {
    const int ix = (int)(pp % np_[0]), iy = (int)((pp / np_[0]) % np_[1]),
              iz = (int)(pp / ((int64_t)np_[0] * np_[1]));
    wave_patches[ix + 2 * iy + 4 * iz].push_back((int)pp);
  }
  std::vector<int2> items;
  items.reserve((size_t)n_patches * n_real);
  std::vector<int64_t> wave_off(n_waves + 1, 0);
  int max_items = 0;
  for (int w = 0; w < n_waves; ++w) {
    wave_off[w] = (int64_t)items.size();
    for (int r = 0; r < n_real; ++r)
      for (int pp : wave_patches[w]) items.push_back(make_int2(r, pp));
    max_items = std::max<int>(max_items, (int)(items.size() - wave_off[w]));
  }
  wave_off[n_waves] = (int64_t)items.size();

  cudaStream_t st = (cudaStream_t)stream;
  SearchArgs a;
  fill_ti_args(t, p->score_mode, a);
  const int chunk = std::min(max_items, 65535);
  DevBuf sg, overlay, d_items, part, cnt;
  if (sg.alloc((size_t)gp_vol * n_real, st) != cudaSuccess ||
      overlay.alloc((size_t)((g_vol + 3) & ~3LL), st) != cudaSuccess ||
      d_items.alloc(sizeof(int2) * items.size(), st) != cudaSuccess ||
      part.alloc(sizeof(unsigned long long) * (size_t)chunk * a.n_tiles * K, st) != cudaSuccess ||
      cnt.alloc(sizeof(unsigned int) * (size_t)chunk, st) != cudaSuccess)
    return fail(CCW_ENOMEM, "simulation workspace");
  cudaError_t e;
  if ((e = cudaMemsetAsync(sg.p, 0xFF, (size_t)gp_vol * n_real, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(overlay.p, 0xFF, (size_t)((g_vol + 3) & ~3LL), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(cnt.p, 0, sizeof(unsigned int) * (size_t)chunk, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(t->d_status, 0, sizeof(int), st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_items.p, items.data(), sizeof(int2) * items.size(),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "simulation setup");
  if ((e = launch_hd_overlay(hd_cells_dev, hd_vals_dev, n_hd, d, g, t->F, (uint8_t*)overlay.p,
                             t->d_status, st)) != cudaSuccess)
    return cuda_fail(e, "hard-data kernel");
  if (n_hd > 0) ++g_launches;
  if (patch_log_dev) {
    // patches never reached cannot exist here, but keep the log well defined
    if ((e = cudaMemsetAsync(patch_log_dev, 0xFF,
                             sizeof(int32_t) * (size_t)n_real * n_patches * (4 + K), st)) !=
        cudaSuccess)
      return cuda_fail(e, "log clear");
  }

  a.sg = (uint8_t*)sg.p;
  a.overlay = (const uint8_t*)overlay.p;
  for (int i = 0; i < 3; ++i) {
    a.G[i] = g[i];
    a.Gp[i] = gp[i];
    a.np[i] = np_[i];
  }
  a.S = S;
  a.path_random = p->path_random;
  a.real_base = p->real_base;
  a.gp_vol = gp_vol;
  a.n_patches = n_patches;
  a.K = K;
  a.seed = seed;
  a.part = (unsigned long long*)part.p;
  a.counters = (unsigned int*)cnt.p;
  a.log = patch_log_dev;
  a.log_stride = 4 + K;
  for (int w = 0; w < n_waves; ++w) {
    const int n = (int)(wave_off[w + 1] - wave_off[w]);
    if (n == 0) continue;
    SearchArgs c = a;
    c.items = (const int2*)d_items.p + wave_off[w];
    if (int rc = run_search(t, kModeSim, c, n, 0, st)) return rc;
  }
  if ((e = launch_crop_out((const uint8_t*)sg.p, gp_vol, gp, out_dev, g, d, n_real,
                           p->path_random, seed, p->real_base, st)) != cudaSuccess)
    return cuda_fail(e, "crop kernel");
  ++g_launches;
  int status = 0;
  if ((e = cudaMemcpyAsync(&status, t->d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "simulation");
  if (status & kStatusBadCode)
    return fail(CCW_EINVAL, "hard data out of the grid or with a code >= n_facies");
  if (status & kStatusHdOverflow)
    return fail(CCW_EINVAL, "more than %d hard data in one template window", kMaxHd);
  if (status & kStatusTimeout) return fail(CCW_ETIMEOUT, "a bounded device wait gave up");
  return CCW_OK;
}

}  // extern "C"
