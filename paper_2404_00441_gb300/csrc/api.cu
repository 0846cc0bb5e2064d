// api.cu -- host side of the C ABI declared in include/ccw.h.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "ccw_internal.cuh"

namespace ccw {
// events.cu
cudaError_t launch_events(int mode, const WaveArgs& a, bool pdl, cudaStream_t st);
// finish.cu
cudaError_t launch_finish(int mode, const WaveArgs& a, bool pdl, cudaStream_t st);
// ccf_simt.cu
int simt_smem_bytes(int d, int nch, int rows, int chunks, int Tj, int TjP, int NB, int K,
                    int nbuf);
void simt_tile_shape(int d, int tile[3]);
void simt_tma_box(int d, int Tj, int TjP, int box[3]);
cudaError_t launch_ccf_simt(int mode, const WaveArgs& a, const CUtensorMap& tmap, int nbuf,
                            int smem, bool pdl, cudaStream_t st);
// tc.cu
int tc_smem_bytes(int nch, int a_nq, int ksteps, int nt, int K, int lane_epi);
cudaError_t launch_ccf_tc(int mode, const WaveArgs& a, int smem, bool pdl, cudaStream_t st);
// tcs.cu
int tcs_smem_bytes(int mt, int nt, int R, int px8, int k16n, int stages);
cudaError_t launch_ccf_tcs(int mode, const WaveArgs& a, int smem, bool pdl, cudaStream_t st);
// persist.cu
int persist_smem_bytes(int nch, int a_nq, int mt, int nt, int ksteps, int F, int ncells, int T,
                       int gw);
int persist_grid(int smem, bool bf16);
cudaError_t launch_persist(const WaveArgs& a, int smem, int grid, cudaStream_t st);
// prepare.cu
cudaError_t launch_phase_planes(const uint8_t* ti, int nx, int s, int F, int ph0, int ph1, int nc0,
                                int nc1, float* planes, int px, int64_t plane_vol,
                                cudaStream_t st);
cudaError_t launch_z8(const float* planes, int px, int64_t plane_vol, int nc0, int nc1, int px8,
                      int64_t nq, int nplanes, void* z8_f16, void* z8_bf16, cudaStream_t st);
cudaError_t launch_crop_ti(const uint8_t* src, const int sdims[3], uint8_t* dst, const int n[3],
                           int F, int* status, cudaStream_t st);
cudaError_t launch_ti_pyramid(int d, const uint8_t* ti, const int n[3], const int nc[3], int s,
                              int J, int F, float* planes, int px, int16_t* pyr,
                              cudaStream_t st);
cudaError_t launch_pad_ti(const uint8_t* ti, const int n[3], uint8_t* dst, const int tp[3],
                          const int border[3], cudaStream_t st);
cudaError_t launch_hd_overlay(const int32_t* cells, const uint8_t* vals, int n, int d,
                              const int g[3], int F, uint8_t* overlay, int* status,
                              cudaStream_t st);
cudaError_t launch_crop_out(const uint8_t* sg, int64_t gp_vol, const int gp[3], uint8_t* out,
                            const int g[3], int d, int n_real, int path_random, uint64_t seed,
                            int real_base, cudaStream_t st, int row0 = 0, int row1 = -1);
cudaError_t launch_idwt_paste(int d, int J, const int16_t* pyr, const int nc[3], const int cd[3],
                              int Tj, int64_t P, int B, const int32_t* picks,
                              const int32_t* origins, uint8_t* grid, const int gdim[3],
                              int* status, cudaStream_t st);
// proposal.cu
cudaError_t launch_round_weights(float* p, int C, int tj, cudaStream_t st);
cudaError_t launch_encode_items(const WaveArgs& a, float* x, float* act, bool pdl,
                                cudaStream_t st);
int64_t enc_tc_image_bytes(int C, int tj);
cudaError_t enc_tc_build_image(const float* P, int C, int tj, void* img, cudaStream_t st);
cudaError_t launch_tables_mma(const __nv_bfloat16* tables, int64_t P, __nv_bfloat16* out,
                              cudaStream_t st);
int64_t tables_mma_elems(int64_t P);
cudaError_t launch_encode_tables(const WaveArgs& a, int type, __nv_bfloat16* tables, float* x,
                                 float* act, float* emb, int chunk, cudaStream_t st);
cudaError_t launch_nnsel(const WaveArgs& a, bool pdl, cudaStream_t st);
int encode_items_launches(int F, int Tj, bool img);
bool nnsel_fuses_rerank(const WaveArgs& a);
bool nnsel_fuses_rerank_shape(int64_t P, int nch, int rows, int Tj, int n_prop);
cudaError_t launch_rerank(const WaveArgs& a, bool pdl, cudaStream_t st);
cudaError_t launch_records_from_counts(const WaveArgs& a, const uint8_t* counts,
                                      int32_t* type_out, cudaStream_t st);
cudaError_t launch_inputs(const WaveArgs& a, int what, const uint8_t* counts, const int32_t* cand,
                          int32_t* type, int n, float* out, cudaStream_t st);
// learned.cu
void net_view(const ccw_net* n, int* C, int* tj, const float** params, int64_t* count);
int64_t infer_act_floats(int C, int tj);
}  // namespace ccw

using namespace ccw;

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
std::atomic<uint32_t> g_barrier_polls{1u << 22};   // grid-barrier polls before giving up

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// profiling state
struct Profiler {
  std::mutex mu;
  bool enabled = false;
  int64_t launches = 0;
  double total_ms = 0.0;
  double phase_ms[3] = {0.0, 0.0, 0.0};   // simulations: events, CCF, finish
  double prop_ms[2] = {0.0, 0.0};          // learned proposal: encoder, selection + re-rank
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;  // direct launches
  unsigned long long* d_work = nullptr;
} g_prof;

unsigned long long* profiling_counters() {
  // caller holds g_prof.mu
  if (!g_prof.d_work) {
    if (cudaMalloc(&g_prof.d_work, 2 * sizeof(unsigned long long)) != cudaSuccess)
      return nullptr;
    cudaMemset(g_prof.d_work, 0, 2 * sizeof(unsigned long long));
  }
  return g_prof.d_work;
}

// Event-record layout (see EvDev).
void event_layout(int nch, int rows, int TjP, int hd_cap, int F, int ncells, EvDev& ev) {
  int64_t off = 64;
  ev.mask_off = (int)off;
  off = align_up(off + 4LL * rows, 16);
  ev.hd_off = (int)off;
  off = align_up(off + 8LL * hd_cap, 16);
  ev.w_off = (int)off;
  off = align_up(off + 4LL * nch * rows * TjP, 16);
  ev.counts_off = (int)off;
  off = align_up(off + (int64_t)F * ncells, 256);
  ev.stride = off;
  ev.hd_cap = hd_cap;
  ev.base = nullptr;
}

}  // namespace

// ---------------------------------------------------------------------------
// Simulation plan: workspace and the captured wave graph of one simulation
// shape, reused while the shape does not change.
// ---------------------------------------------------------------------------
struct GroupPlan {
  int grid[3], n_real;
  int g[3], np[3], gp[3];
  int64_t gp_vol, g_vol, n_patches;
  void* sg = nullptr;
  void* overlay = nullptr;
};

struct SimPlan {
  int n_groups = 0;
  std::vector<GroupPlan> groups;
  int K, score_mode, precision;
  int learned = 0, n_prop = 0, ccf_tile = 0;
  int vt_ext = 0, cut = 0;        // virtual-template extension, boundary cut
  int all_shift = 0;              // all-shift candidates (phases of the TI)
  PhaseDev* d_phases = nullptr;   // [n_phases] with this plan's M-groups and key lists
  int n_phases = 0;
  int n_waves, max_items;
  std::vector<int64_t> wave_off;
  void* items = nullptr;
  void* ev = nullptr;
  void* part = nullptr;
  void* bmat = nullptr;
  void* emb = nullptr;       // learned proposal: [max_items][64] item embeddings
  void* prop = nullptr;      // [max_items][n_prop] proposals
  void* prop_gap = nullptr;  // [max_items] relative embedding gaps
  void* enc_x = nullptr;     // encoder inputs and activations of a step
  void* enc_act = nullptr;
  CallDev* call = nullptr;
  SimGroup* dgroups = nullptr;
  int64_t* wave_off_d = nullptr;            // persistent kernel: wavefront offsets
  unsigned* gbar = nullptr;                 // persistent kernel: barrier words
  unsigned long long* phase_ns = nullptr;   // persistent kernel: profiled phase times
  cudaEvent_t pev[2] = {nullptr, nullptr};  // persistent kernel: profiled launch
  EvDev evl;
  // Realization lanes: the realizations are split into groups whose
  // wavefront chains are captured on separate streams of the same graph, so
  // that the kernels of different lanes run at the same time. Lane 0 uses
  // the buffers above; every lane has its own schedule (offsets into
  // `items`) and scratch.
  struct Lane {
    std::vector<int64_t> wave_off;   // [n_waves + 1]
    int max_items = 0;
    void* ev = nullptr;
    void* part = nullptr;
    void* bmat = nullptr;
    cudaStream_t st = nullptr;       // capture stream (lanes >= 1)
    cudaEvent_t done = nullptr;      // end of the lane's chain (lanes >= 1)
  };
  std::vector<Lane> lanes;
  int64_t launches_per_call = 0;
  void* cp = nullptr;   // CcfPlan (defined with the kernels' host helpers)
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};   // [profiling]
  // Streamed read-back (groups with a pinned out_host, unmirrored paths):
  // a third graph also crops each band of output rows once the patch rows
  // over it are pasted and copies it to the host while later wavefronts
  // run, on one copy stream per lane. It bakes in the output pointers it
  // was captured with and is captured again when they change.
  cudaGraphExec_t exec_host = nullptr;
  std::vector<uint8_t*> host_dev, host_host;   // per group, as captured
  std::vector<cudaStream_t> cst;               // per lane: copy stream
  std::vector<cudaEvent_t> cev;                // per lane: fork / join mark
  int64_t host_launches = 0;                   // band crops per call
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;   // around each CCF launch
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_bounds;   // before events, after finish
  std::vector<cudaEvent_t> prof_prop;   // learned: [3] per step: before encoder, before selection, after
  ~SimPlan() {
    for (auto& e : exec)
      if (e) cudaGraphExecDestroy(e);
    if (exec_host) cudaGraphExecDestroy(exec_host);
    for (auto s : cst) cudaStreamDestroy(s);
    for (auto e : cev) cudaEventDestroy(e);
    for (auto* v : {&prof_events, &prof_bounds})
      for (auto& pr : *v) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
      }
    for (auto ev : prof_prop) cudaEventDestroy(ev);
    if (cap) cudaStreamDestroy(cap);
    for (size_t l = 1; l < lanes.size(); ++l) {
      cudaFree(lanes[l].ev);
      cudaFree(lanes[l].part);
      cudaFree(lanes[l].bmat);
      if (lanes[l].st) cudaStreamDestroy(lanes[l].st);
      if (lanes[l].done) cudaEventDestroy(lanes[l].done);
    }
    for (auto& e : pev)
      if (e) cudaEventDestroy(e);
    cudaFree(wave_off_d);
    cudaFree(gbar);
    cudaFree(phase_ns);
    for (auto& g : groups) {
      cudaFree(g.sg);
      cudaFree(g.overlay);
    }
    cudaFree(items);
    cudaFree(ev);
    cudaFree(part);
    cudaFree(bmat);
    cudaFree(emb);
    cudaFree(prop);
    cudaFree(prop_gap);
    cudaFree(enc_x);
    cudaFree(enc_act);
    cudaFree(call);
    cudaFree(dgroups);
    cudaFree(d_phases);
    release_cp();
  }
  void release_cp();
};

struct ccw_ti {
  int ndim, F, J, s, sd, T, O, Tj, TjP, chunks, rows;
  int n[3], nc[3], cd[3];
  int64_t ncv, P;
  int px;
  int64_t plane_vol;
  int device;
  int tile[3], tiles[3], n_tiles;
  uint8_t* d_ti = nullptr;      // cropped fine TI
  uint8_t* d_tip = nullptr;     // the same inside a border of T cells of 255 (hard-data checks)
  int tp[3];                    // dims of d_tip
  int64_t tip_origin = 0;       // offset of cell (0, 0, 0) in d_tip
  float* d_planes = nullptr;    // F planes [nc2][nc1][px]: facies 0..F-2 counts, code sums
  int16_t* d_pyr = nullptr;     // [ncv][sd]
  int* d_status = nullptr;      // device status word
  CUtensorMap tmap;             // TMA view of the planes, box = one CCF tile plus halo
  // tensor-core view (2D): 8-shift copies of the planes, FP16 and BF16
  int px8 = 0, ks = 0, mtiles = 0;
  int64_t z8_nq = 0;
  void* z8_f16 = nullptr;
  void* z8_bf16 = nullptr;
  // learned proposal (2D): encoder parameters, window tables per mask type
  float* d_net = nullptr;
  __nv_bfloat16* d_tables = nullptr;   // [16][P][64]
  __nv_bfloat16* d_tables_mma = nullptr;   // the same in 128-window MMA blocks (small P)
  void* d_enc_img = nullptr;               // the encoder's tensor-core weight image
  unsigned long long* d_learn_stats = nullptr;   // [3]
  int n_prop = 0;
  float gap_theta = 0.f;
  // all-shift candidates (2D): level-J planes and 8-shift copies of every
  // phase, built on first use
  int n_phases = 0;
  int fd[2] = {0, 0};                 // fine candidate grid
  int64_t P_fine = 0;
  std::vector<PhaseDev> h_phases;
  std::vector<void*> phase_bufs;      // planes and 8-shift copies, freed with the TI
  std::mutex mu;
  SimPlan* plan = nullptr;
};

namespace {

// Fill the TI part of the kernel arguments.
void fill_ti(const ccw_ti* t, int score_mode, WaveArgs& a) {
  memset(&a, 0, sizeof(a));
  TiDev& d = a.ti;
  d.planes = t->d_planes;
  d.px = t->px;
  d.plane_vol = t->plane_vol;
  d.plane0 = score_mode == 0 ? 0 : t->F - 1;
  d.nch = score_mode == 0 ? t->F - 1 : 1;
  d.ti = t->d_tip + t->tip_origin;
  d.pyr = t->d_pyr;
  d.F = t->F;
  d.J = t->J;
  d.s = t->s;
  d.sd = t->sd;
  d.T = t->T;
  d.Tj = t->Tj;
  d.TjP = t->TjP;
  d.chunks = t->chunks;
  d.rows = t->rows;
  d.d = t->ndim;
  d.score_mode = score_mode;
  for (int i = 0; i < 3; ++i) {
    d.n[i] = t->n[i];
    d.tp[i] = t->tp[i];
    d.nc[i] = t->nc[i];
    d.cd[i] = t->cd[i];
    d.tile[i] = t->tile[i];
    d.tiles[i] = t->tiles[i];
  }
  d.ncv = t->ncv;
  d.P = t->P;
  d.n_tiles = t->n_tiles;
  a.status = t->d_status;
  a.Oj = t->O / t->s;
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

// Items per CTA and TI tile buffers of the CCF kernel.
void choose_simt(const ccw_ti* t, int nch, int K, int n_items, int& nb, int& nbuf, int& smem,
                 int nb_hint = 0) {
  nb = (t->ndim == 3) ? 2 : 4;
  while (nb > 1 && n_items < nb / 2 + 1) nb /= 2;
  if (nb_hint) nb = nb_hint;
  nbuf = 2;
  smem = simt_smem_bytes(t->ndim, nch, t->rows, t->chunks, t->Tj, t->TjP, nb, K, nbuf);
  if (smem > 110 * 1024) {
    nbuf = 1;
    smem = simt_smem_bytes(t->ndim, nch, t->rows, t->chunks, t->Tj, t->TjP, nb, K, nbuf);
  }
  while (!nb_hint && smem > 220 * 1024 && nb > 1) {
    nb /= 2;
    smem = simt_smem_bytes(t->ndim, nch, t->rows, t->chunks, t->Tj, t->TjP, nb, K, nbuf);
  }
}

// Hard data kept per event record: the window, grown by the virtual
// template's extension when there is one.
int hd_capacity(const ccw_ti* t, int vt_ext = 0) {
  return (int)std::min<int64_t>(kMaxHd, ipow(t->T + vt_ext, t->ndim));
}

// Precision check: the tensor-core path is exact while every operand fits
// the 16-bit format exactly (FP16: |v| <= 2048, BF16: |v| <= 256).
int check_precision(const ccw_ti* t, int precision, int score_mode, int K = 1, int hint = 0) {
  if (precision == 0) return CCW_OK;
  if (precision != 1 && precision != 2 && precision != (1 | CCW_PRECISION_INEXACT) &&
      precision != (2 | CCW_PRECISION_INEXACT))
    return fail(CCW_EINVAL, "precision must be 0, 1 or 2, optionally with CCW_PRECISION_INEXACT");
  // the streamed tensor-core kernel (3D, or 2D on request) keeps the K best
  // keys of each thread in registers: K <= 8
  if ((t->ndim == 3 || ((hint >> 25) & 1)) && K > 8)
    return fail(CCW_EUNSUPPORTED, "the streamed tensor-core CCF supports K <= 8");
  // beyond the format's exact integers only on request: operands are then
  // rounded to it and the scores are approximate
  if (precision & CCW_PRECISION_INEXACT) return CCW_OK;
  const int64_t vmax = (int64_t)(score_mode == 0 ? 1 : t->F - 1) * t->sd;
  const int64_t lim = precision == 1 ? 2048 : 256;
  if (vmax > lim)
    return fail(CCW_EINVAL,
                "%s operands up to %lld are beyond its exact integer range (%lld); lower the "
                "level or use precision 0",
                precision == 1 ? "FP16" : "BF16", (long long)vmax, (long long)lim);
  return CCW_OK;
}

int tc_a_nq(const ccw_ti* t, int mt) {
  return 16 * (mt - 1) + (t->rows - 1) * t->px8 / 8 + 2 * (t->ks / 16 - 1) + 17;
}

// Tensor-core tiling: items per N-tile, M-tiles per CTA, shared memory.
void choose_tc(const ccw_ti* t, int nch, int K, int n_items, WaveArgs& a, int& smem,
               bool& streamed, int hint = 0) {
  // streamed operands (tcs.cu) in 3D, where a CTA's whole Hankel view does
  // not fit in shared memory, and in 2D when the hint asks for them
  streamed = t->ndim == 3 || ((hint >> 25) & 1);
  a.nt = n_items <= 16 ? 16 : n_items <= 32 ? 32 : n_items <= 64 ? 64 : 128;
  // epilogue: per-thread K-lists pay off for K = 1; lanes on candidates
  // keep every lane busy when the item count is small and K > 1
  a.tc_lane_epi = K > 1 ? 1 : 0;
  // K > 1: the epilogue per item dominates; narrow N-tiles spread it over
  // more CTAs (timed: 20 x 512^2, K = 5, 200 items per wavefront, 4x faster
  // than 128-wide tiles)
  if (K > 1) a.nt = 16;
  if (hint) {
    a.nt = hint & 0xFFFF;
    a.tc_lane_epi = (hint >> 24) & 1;
  }
  a.ks = t->ks;
  a.ksteps = nch * t->rows * (t->ks / 16);
  a.px8 = t->px8;
  a.mtiles = t->mtiles;
  const int n_ntiles = (n_items + a.nt - 1) / a.nt;
  // M-tiles per CTA: about one CTA per SM, at most 4 (and mt * nt TMEM
  // columns <= 512)
  int mt = (int)std::max<int64_t>(1, std::min<int64_t>(4, ((int64_t)t->mtiles * n_ntiles + 151) / 152));
  if (hint) mt = (hint >> 16) & 0xFF;
  while (mt * a.nt > 512) --mt;
  for (;;) {
    if (streamed) {
      // double-buffered slices (two CTAs can then share an SM); three
      // stages on request (bit 26 of the hint), four with bit 29
      a.tcs_stages = ((hint >> 29) & 1) ? 4 : ((hint >> 26) & 1) ? 3 : 2;
      // rows per stage: Tj, or Tj split in 2 or 4 blocks (bits 27-28)
      const int split = 1 << ((hint >> 27) & 3);
      a.tcs_rows = (t->Tj + split - 1) / split;
      smem = tcs_smem_bytes(mt, a.nt, a.tcs_rows, t->px8, t->ks / 16, a.tcs_stages);
    } else {
      smem = tc_smem_bytes(nch, tc_a_nq(t, mt), a.ksteps, a.nt, K, a.tc_lane_epi);
    }
    if (hint || smem <= 220 * 1024 || (mt == 1 && a.nt == 16)) break;
    if (mt > 1) --mt;
    else a.nt /= 2;
  }
  a.mt = mt;
  a.a_nq = streamed ? 0 : tc_a_nq(t, mt);
  a.n_mgroups = (t->mtiles + mt - 1) / mt;
  a.z8_nq = t->z8_nq;
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

// How phase B runs for a batch shape: the FP32 SIMT kernel (precision 0) or
// the tensor-core kernel (precision 1: FP16, 2: BF16), its tiling and the
// scratch it needs per chunk of at most 65535 items.
struct CcfPlan {
  int precision = 0;
  int nb = 1, nbuf = 1, smem = 0;   // SIMT
  bool streamed = false;             // tensor cores with streamed operands (tcs.cu)
  WaveArgs tc;                       // tensor-core tiling fields
  int n_parts = 0;                   // partial key lists per item
  int64_t ev_bytes = 0, part_bytes = 0, bmat_bytes = 0;
  // one cooperative kernel for every wavefront of a call (persist.cu)
  bool persist = false;
  int p_grid = 0, p_gw = 32;
};

}  // namespace

void SimPlan::release_cp() { delete static_cast<CcfPlan*>(cp); }

namespace {

// ccf_tile bits 20-22: realization lanes - 1 (the graph path); the other
// bits give the CCF tiling.
constexpr int kTileLaneMask = 7 << 20;
int tile_lanes(int hint) { return ((hint >> 20) & 7) + 1; }

// Valid values of the `ccf_tile` hint (0 = the library's heuristic).
bool valid_tile_hint(const ccw_ti* t, int precision, int hint) {
  hint &= ~kTileLaneMask;
  if (hint == 0) return true;
  if (precision == 0)
    return t->ndim == 2 ? (hint == 1 || hint == 2 || hint == 4 || hint == 8)
                        : (hint == 1 || hint == 2 || hint == 4);
  const int nt = hint & 0xFFFF, mt = (hint >> 16) & 0xFF, flags = hint >> 24;
  if (flags == kTilePersist >> 24)   // persistent kernel: nt up to 256, mt 0 = automatic
    return (nt == 16 || nt == 32 || nt == 64 || nt == 128 || nt == 256) && mt <= kTcMaxMt &&
           mt * nt <= 512;
  return (nt == 16 || nt == 32 || nt == 64 || nt == 128) && mt >= 1 && mt <= kTcMaxMt &&
         mt * nt <= 512 && flags >= 0 && flags <= 63 && ((flags >> 3) & 3) != 3 &&
         !((flags >> 5) & 1 && (flags >> 2) & 1);
}

bool tile_is_persist(int precision, int hint) {
  return precision != 0 && (hint >> 24) == (kTilePersist >> 24);
}

// The persistent form of a simulation plan: M-tiles per CTA so that every
// M-group has a CTA of the cooperative grid, threads per item in the gather
// and paste phases from the widest wavefront. Returns CCW_OK or a refusal.
int plan_persist(const ccw_ti* t, int nch, int K, int max_items, int hint, int vt_ext, int cut,
                 int learned, CcfPlan& cp) {
  if (t->ndim != 2) return fail(CCW_EINVAL, "the persistent kernel is 2D only");
  if (K > 8) return fail(CCW_EINVAL, "the persistent kernel needs K <= 8");
  if (vt_ext || cut || learned)
    return fail(CCW_EINVAL,
                "the persistent kernel does not run the virtual template, the boundary cut or "
                "the learned proposal");
  WaveArgs& a = cp.tc;
  memset(&a, 0, sizeof(a));
  a.nt = hint & 0xFFFF;
  a.ks = t->ks;
  a.ksteps = nch * t->rows * (t->ks / 16);
  a.px8 = t->px8;
  a.mtiles = t->mtiles;
  a.z8_nq = t->z8_nq;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return fail(CCW_ECUDA, "multiprocessor count");
  int mt = (hint >> 16) & 0xFF;
  if (mt == 0) mt = (t->mtiles + sms - 1) / sms;
  if (mt > kTcMaxMt || mt * a.nt > 512)
    return fail(CCW_EINVAL, "persistent kernel: %d M-tiles per CTA needed (at most %d, mt x nt "
                "<= 512)", mt, kTcMaxMt);
  a.mt = mt;
  a.n_mgroups = (t->mtiles + mt - 1) / mt;
  a.a_nq = tc_a_nq(t, mt);
  const int gw = max_items <= sms ? 256 : max_items <= 2 * sms ? 128 : max_items <= 4 * sms ? 64
                                                                                            : 32;
  cp.p_gw = gw;
  cp.smem = persist_smem_bytes(nch, a.a_nq, mt, a.nt, a.ksteps, t->F, t->Tj * t->Tj, t->T, gw);
  if (cp.smem > 227 * 1024)
    return fail(CCW_EINVAL, "persistent kernel: %d bytes of shared memory needed", cp.smem);
  cp.p_grid = persist_grid(cp.smem, cp.precision == 2);
  if (cp.p_grid < a.n_mgroups)
    return fail(CCW_EINVAL, "persistent kernel: %d M-groups for %d resident CTAs", a.n_mgroups,
                cp.p_grid);
  cp.persist = true;
  cp.streamed = false;
  cp.n_parts = a.n_mgroups;
  cp.bmat_bytes = ((max_items + a.nt - 1) / a.nt) * (int64_t)a.ksteps * 32 * a.nt;
  cp.part_bytes = (int64_t)max_items * cp.n_parts * K * 8;
  return CCW_OK;
}

void plan_ccf(const ccw_ti* t, int precision, int nch, int K, int n_items, const EvDev& ev,
              CcfPlan& cp, int hint = 0) {
  cp.precision = precision;
  const int64_t chunk = std::min(n_items, 65535);
  if (precision == 0) {
    choose_simt(t, nch, K, (int)chunk, cp.nb, cp.nbuf, cp.smem, hint);
    cp.n_parts = t->n_tiles;
    cp.bmat_bytes = 0;
  } else {
    memset(&cp.tc, 0, sizeof(cp.tc));
    choose_tc(t, nch, K, (int)chunk, cp.tc, cp.smem, cp.streamed, hint);
    cp.n_parts = cp.tc.n_mgroups;
    cp.bmat_bytes = ((chunk + cp.tc.nt - 1) / cp.tc.nt) * (int64_t)cp.tc.ksteps * 32 * cp.tc.nt;
  }
  cp.ev_bytes = chunk * ev.stride;
  cp.part_bytes = chunk * (int64_t)cp.n_parts * K * 8;
}

// Copy the phase-B configuration into the kernel arguments.
void apply_ccf(const ccw_ti* t, const CcfPlan& cp, void* bmat, WaveArgs& c) {
  c.precision = cp.precision;
  c.nb = cp.nb;
  c.n_parts = cp.n_parts;
  if (cp.precision) {
    c.z8 = cp.precision == 2 ? t->z8_bf16 : t->z8_f16;
    c.z8_nq = cp.tc.z8_nq;
    c.px8 = cp.tc.px8;
    c.ks = cp.tc.ks;
    c.ksteps = cp.tc.ksteps;
    c.mtiles = cp.tc.mtiles;
    c.mt = cp.tc.mt;
    c.n_mgroups = cp.tc.n_mgroups;
    c.nt = cp.tc.nt;
    c.a_nq = cp.tc.a_nq;
    c.tc_lane_epi = cp.tc.tc_lane_epi;
    c.tcs_stages = cp.tc.tcs_stages;
    c.tcs_rows = cp.tc.tcs_rows;
    c.bmat = bmat;
  }
}

cudaError_t launch_ccf(const ccw_ti* t, int mode, const CcfPlan& cp, const WaveArgs& c, bool pdl,
                       cudaStream_t st) {
  if (cp.precision && cp.streamed) return launch_ccf_tcs(mode, c, cp.smem, pdl, st);
  if (cp.precision) return launch_ccf_tc(mode, c, cp.smem, pdl, st);
  return launch_ccf_simt(mode, c, t->tmap, cp.nbuf, cp.smem, pdl, st);
}

// Phases A, B (and C when searching) on explicit data events, in chunks of
// at most 65535 items. Scratch comes from the caller (sizes from plan_ccf).
// `profiled` = false keeps the launches out of the profiler, whose counters
// and per-launch events would otherwise be allocated here.
int run_explicit(const ccw_ti* t, int mode, WaveArgs a, int B, const CcfPlan& cp,
                 unsigned char* ev_base, unsigned long long* part, void* bmat, cudaStream_t st,
                 bool profiled = true) {
  const int64_t tv = ipow(t->T, t->ndim);
  unsigned long long* work = nullptr;
  bool prof = false;
  if (profiled) {
    std::lock_guard<std::mutex> g(g_prof.mu);
    prof = g_prof.enabled;
    if (prof) work = profiling_counters();
  }
  for (int i0 = 0; i0 < B; i0 += 65535) {
    WaveArgs c = a;
    c.n_items = std::min(65535, B - i0);
    apply_ccf(t, cp, bmat, c);
    c.ev.base = ev_base;
    c.part = part;
    c.work = work;
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
    cudaError_t e = launch_events(mode, c, false, st);
    if (e != cudaSuccess) return cuda_fail(e, "event kernel launch");
    ++g_launches;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, st);
    }
    e = launch_ccf(t, mode, cp, c, !prof, st);
    if (e != cudaSuccess) return cuda_fail(e, "CCF kernel launch");
    ++g_launches;
    if (prof) {
      cudaEventRecord(e1, st);
      std::lock_guard<std::mutex> g(g_prof.mu);
      g_prof.pending.emplace_back(e0, e1);
    }
    if (mode == kModeSearch) {
      e = launch_finish(mode, c, !prof, st);
      if (e != cudaSuccess) return cuda_fail(e, "finish kernel launch");
      ++g_launches;
    }
  }
  return CCW_OK;
}

// score_mode argument of the search entry points: bits 0-3 the score mode,
// bits 4-7 the precision.
int split_mode(int32_t mode, int& score_mode, int& precision) {
  score_mode = mode & 0xF;
  precision = (mode >> 4) & 0xF;
  if ((mode & ~0xFF) != 0 || (score_mode != 0 && score_mode != 1))
    return fail(CCW_EINVAL, "score_mode must be 0 or 1 (bits 0-3), precision in bits 4-7");
  return CCW_OK;
}

int search_common(const ccw_ti* t, int mode, int32_t B, const uint8_t* de, const uint8_t* hd,
                  int32_t k, int32_t score_arg, uint64_t seed, const uint32_t* ctr,
                  int32_t* ti_idx, int32_t* ti_sc, int32_t* ti_mm, int32_t* pick,
                  int32_t* map_sc, int32_t* map_mm, void* stream) {
  if (!t) return fail(CCW_EINVAL, "ti is NULL");
  if (B < 0) return fail(CCW_EINVAL, "B must be >= 0");
  int score_mode, precision;
  if (int rc = split_mode(score_arg, score_mode, precision)) return rc;
  if (int rc = check_score_bound(t, score_mode)) return rc;
  if (int rc = check_precision(t, precision, score_mode, mode == kModeSearch ? k : 1)) return rc;
  precision &= 3;   // the format; checked above
  if (mode == kModeSearch && (k < 1 || k > CCW_MAX_TOPK))
    return fail(CCW_EINVAL, "k must be in [1, %d]", CCW_MAX_TOPK);
  if (B == 0) return CCW_OK;
  if (!de) return fail(CCW_EINVAL, "de_dev is NULL");
  if (mode == kModeSearch) {
    if (!ctr || !ti_idx || !ti_sc || !ti_mm || !pick)
      return fail(CCW_EINVAL, "NULL output or counter");
  } else if (!map_sc) {
    return fail(CCW_EINVAL, "score_dev is NULL");
  }
  cudaStream_t st = (cudaStream_t)stream;
  WaveArgs a;
  fill_ti(t, score_mode, a);
  event_layout(a.ti.nch, t->rows, t->TjP, hd_capacity(t), t->F, t->rows * t->Tj, a.ev);
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
  CcfPlan cp;
  plan_ccf(t, precision, a.ti.nch, a.K, B, a.ev, cp);
  DevBuf evb, part, bm;
  if (evb.alloc((size_t)cp.ev_bytes, st) != cudaSuccess ||
      (mode == kModeSearch && part.alloc((size_t)cp.part_bytes, st) != cudaSuccess) ||
      (cp.bmat_bytes && bm.alloc((size_t)cp.bmat_bytes, st) != cudaSuccess))
    return fail(CCW_ENOMEM, "search scratch");
  return run_explicit(t, mode, a, B, cp, (unsigned char*)evb.p, (unsigned long long*)part.p,
                      bm.p, st);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Scratch of ccw_ccf_search_noalloc: one array per device, part of the
// library image, so using it needs no allocation. Host code reaches it only
// through the device address looked up below; the symbol itself is a host
// stand-in that no kernel may be given.
__device__ __align__(256) unsigned char g_noalloc_scratch[CCW_NOALLOC_SCRATCH_BYTES];

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

extern "C" {

const char* ccw_last_error(void) { return g_err; }

int64_t ccw_launch_count(void) { return g_launches.load(); }

int ccw_set_barrier_polls(int64_t polls) {
  if (polls < 0 || polls > 0xFFFFFFFFll) return fail(CCW_EINVAL, "polls out of range");
  g_barrier_polls.store(polls == 0 ? (1u << 22) : (uint32_t)polls);
  return CCW_OK;
}

int ccw_profile_enable(int32_t enable) {
  std::lock_guard<std::mutex> g(g_prof.mu);
  g_prof.enabled = enable != 0;
  return CCW_OK;
}

int ccw_profile_read_phases(double ms[3]) {
  if (!ms) return fail(CCW_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(g_prof.mu);
  for (int i = 0; i < 3; ++i) {
    ms[i] = g_prof.phase_ms[i];
    g_prof.phase_ms[i] = 0.0;
  }
  return CCW_OK;
}

int ccw_profile_read_proposal(double ms[2]) {
  if (!ms) return fail(CCW_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(g_prof.mu);
  for (int i = 0; i < 2; ++i) {
    ms[i] = g_prof.prop_ms[i];
    g_prof.prop_ms[i] = 0.0;
  }
  return CCW_OK;
}

int ccw_profile_read(int64_t* launches, double* total_ms, double* cand_evals, double* macs) {
  std::lock_guard<std::mutex> g(g_prof.mu);
  for (auto& pr : g_prof.pending) {
    cudaEventSynchronize(pr.second);
    float t = 0.f;
    cudaEventElapsedTime(&t, pr.first, pr.second);
    g_prof.total_ms += t;
    ++g_prof.launches;
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  g_prof.pending.clear();
  if (launches) *launches = g_prof.launches;
  if (total_ms) *total_ms = g_prof.total_ms;
  g_prof.launches = 0;
  g_prof.total_ms = 0.0;
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
  ccw_ti* t = new ccw_ti();
  t->ndim = ndim;
  t->F = n_facies;
  t->J = level;
  t->s = s;
  t->sd = ndim == 2 ? s * s : s * s * s;
  t->T = templ;
  t->O = overlap;
  t->Tj = templ / s;
  t->TjP = 4 * ((t->Tj + 3) / 4);
  t->chunks = t->TjP / 4;
  t->rows = ndim == 3 ? t->Tj * t->Tj : t->Tj;
  auto reject = [&](int code, const char* msg) {
    delete t;
    return fail(code, "%s", msg);
  };
  for (int a = 0; a < 3; ++a) {
    const int sa = a < ndim ? s : 1;
    if (dims[a] <= 0) return reject(CCW_EINVAL, "dims must be positive");
    t->nc[a] = dims[a] / sa;
    t->n[a] = t->nc[a] * sa;
    t->cd[a] = a < ndim ? t->nc[a] - t->Tj + 1 : 1;
    if (t->cd[a] <= 0) return reject(CCW_EINVAL, "template larger than the TI");
  }
  t->ncv = (int64_t)t->nc[0] * t->nc[1] * t->nc[2];
  t->P = (int64_t)t->cd[0] * t->cd[1] * t->cd[2];
  if (t->P >= (1 << 24)) return reject(CCW_EINVAL, "more than 2^24 - 1 candidates");
  if (t->chunks > kMaxChunks) return reject(CCW_EINVAL, "template too large (T/2^J > 128)");
  if (check_score_bound(t, 0)) {
    delete t;
    return CCW_EINVAL;
  }
  t->px = (int)align_up(t->nc[0], 4);
  t->plane_vol = (int64_t)t->px * t->nc[1] * t->nc[2];
  simt_tile_shape(ndim, t->tile);
  for (int a = 0; a < 3; ++a) t->tiles[a] = (t->cd[a] + t->tile[a] - 1) / t->tile[a];
  t->n_tiles = t->tiles[0] * t->tiles[1] * t->tiles[2];
  {
    int nb, nbuf, smem;
    choose_simt(t, t->F - 1, CCW_MAX_TOPK, 1, nb, nbuf, smem);
    if (smem > 227 * 1024) return reject(CCW_EUNSUPPORTED, "template too large for the CCF tile");
  }
  cudaGetDevice(&t->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nv = (int64_t)t->n[0] * t->n[1] * t->n[2];
  cudaError_t e;
  for (int a = 0; a < 3; ++a) t->tp[a] = a < ndim ? t->n[a] + 2 * t->T : 1;
  t->tip_origin = t->T + (int64_t)t->tp[0] * (t->T + (ndim == 3 ? (int64_t)t->tp[1] * t->T : 0));
  const int64_t tipv = (int64_t)t->tp[0] * t->tp[1] * t->tp[2];
  auto release = [&]() {
    cudaFree(t->d_ti);
    cudaFree(t->d_tip);
    cudaFree(t->d_planes);
    cudaFree(t->d_pyr);
    cudaFree(t->d_status);
    delete t;
  };
  if ((e = cudaMalloc(&t->d_ti, nv)) != cudaSuccess ||
      (e = cudaMalloc(&t->d_tip, tipv)) != cudaSuccess ||
      (e = cudaMalloc(&t->d_planes, sizeof(float) * t->plane_vol * t->F)) != cudaSuccess ||
      (e = cudaMalloc(&t->d_pyr, sizeof(int16_t) * t->ncv * t->sd)) != cudaSuccess ||
      (e = cudaMalloc(&t->d_status, sizeof(int))) != cudaSuccess) {
    release();
    return fail(CCW_ENOMEM, "TI buffers: %s", cudaGetErrorString(e));
  }
  if ((e = cudaMemsetAsync(t->d_status, 0, sizeof(int), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(t->d_planes, 0, sizeof(float) * t->plane_vol * t->F, st)) !=
          cudaSuccess) {
    release();
    return cuda_fail(e, "prepare clear");
  }
  const int sdims[3] = {dims[0], dims[1], dims[2]};
  if ((e = launch_crop_ti(ti_dev, sdims, t->d_ti, t->n, t->F, t->d_status, st)) != cudaSuccess) {
    release();
    return cuda_fail(e, "crop kernel");
  }
  ++g_launches;
  if ((e = launch_ti_pyramid(ndim, t->d_ti, t->n, t->nc, s, level, t->F, t->d_planes, t->px,
                             t->d_pyr, st)) != cudaSuccess) {
    release();
    return cuda_fail(e, "pyramid kernel");
  }
  ++g_launches;
  {
    const int border[3] = {t->T, t->T, ndim == 3 ? t->T : 0};
    if ((e = launch_pad_ti(t->d_ti, t->n, t->d_tip, t->tp, border, st)) != cudaSuccess) {
      release();
      return cuda_fail(e, "padded TI kernel");
    }
    ++g_launches;
  }
  // TMA view of the planes: (x: px, y: nc1, z: nc2, plane: F), one tile box
  auto encode = tensor_map_encoder();
  if (!encode) {
    release();
    return fail(CCW_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  }
  int box[3];
  simt_tma_box(ndim, t->Tj, t->TjP, box);
  if (box[0] > 256 || box[1] > 256 || box[2] > 256) {
    release();
    return fail(CCW_EUNSUPPORTED, "CCF tile box beyond the TMA limit");
  }
  cuuint64_t gdim[4] = {(cuuint64_t)t->px, (cuuint64_t)t->nc[1], (cuuint64_t)t->nc[2],
                        (cuuint64_t)t->F};
  cuuint64_t gstride[3] = {(cuuint64_t)t->px * 4, (cuuint64_t)t->px * t->nc[1] * 4,
                           (cuuint64_t)t->plane_vol * 4};
  cuuint32_t bdim[4] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2], 1};
  cuuint32_t estride[4] = {1, 1, 1, 1};
  CUresult cr = encode(&t->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, t->d_planes, gdim, gstride,
                       bdim, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    release();
    return fail(CCW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  }
  {
    // 8-shift copies of the planes for the tensor-core CCF, over the line
    // L = x + px8 (y + nc1 z) of the level-J grid
    t->px8 = (int)align_up(t->nc[0], 8);
    t->ks = 16 * ((t->Tj + 15) / 16);
    const int64_t lines = (ndim == 2) ? t->cd[1] : (int64_t)t->nc[1] * (t->cd[2] - 1) + t->cd[1];
    t->mtiles = (int)(((int64_t)t->px8 * lines + 127) / 128);
    const int64_t roff_max =
        (int64_t)t->px8 * ((t->Tj - 1) + (ndim == 3 ? (int64_t)t->nc[1] * (t->Tj - 1) : 0));
    t->z8_nq = std::max<int64_t>(
        16LL * t->mtiles + 128 + (int64_t)(t->rows - 1) * t->px8 / 8 + 2 * (t->ks / 16) + 32,
        (128LL * (t->mtiles + kTcMaxMt) + roff_max + t->ks + 256) / 8 + 8);
    const size_t zb = (size_t)t->F * t->z8_nq * 128;
    if ((e = cudaMalloc(&t->z8_f16, zb)) != cudaSuccess ||
        (e = cudaMalloc(&t->z8_bf16, zb)) != cudaSuccess) {
      cudaFree(t->z8_f16);
      cudaFree(t->z8_bf16);
      release();
      return fail(CCW_ENOMEM, "tensor-core TI buffers: %s", cudaGetErrorString(e));
    }
    if ((e = launch_z8(t->d_planes, t->px, t->plane_vol, t->nc[0], t->nc[1] * t->nc[2], t->px8,
                       t->z8_nq, t->F, t->z8_f16, t->z8_bf16, st)) != cudaSuccess) {
      cudaFree(t->z8_f16);
      cudaFree(t->z8_bf16);
      release();
      return cuda_fail(e, "8-shift kernel");
    }
    g_launches += 2;
  }
  int status = 0;
  if ((e = cudaMemcpyAsync(&status, t->d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess) {
    cudaFree(t->z8_f16);
    cudaFree(t->z8_bf16);
    release();
    return cuda_fail(e, "prepare");
  }
  if (status) {
    cudaFree(t->z8_f16);
    cudaFree(t->z8_bf16);
    release();
    return fail(CCW_EINVAL, "training image holds codes >= n_facies");
  }
  *out = t;
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
  delete t->plan;
  cudaFree(t->z8_f16);
  cudaFree(t->z8_bf16);
  cudaFree(t->d_ti);
  cudaFree(t->d_tip);
  cudaFree(t->d_planes);
  cudaFree(t->d_pyr);
  cudaFree(t->d_status);
  cudaFree(t->d_net);
  cudaFree(t->d_tables);
  cudaFree(t->d_tables_mma);
  cudaFree(t->d_enc_img);
  cudaFree(t->d_learn_stats);
  for (void* b : t->phase_bufs) cudaFree(b);
  delete t;
}

int ccw_ti_export(const ccw_ti* t, int32_t what, void* dst, void* stream) {
  if (!t || !dst) return fail(CCW_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  switch (what) {
    case 0:
    case 1: {
      // drop the row padding: planes are [nc2][nc1][px]
      const int p0 = what == 0 ? 0 : t->F - 1;
      const int np = what == 0 ? t->F - 1 : 1;
      for (int p = 0; p < np && e == cudaSuccess; ++p)
        e = cudaMemcpy2DAsync((float*)dst + (int64_t)p * t->ncv, sizeof(float) * t->nc[0],
                              t->d_planes + (int64_t)(p0 + p) * t->plane_vol,
                              sizeof(float) * t->px, sizeof(float) * t->nc[0],
                              (size_t)t->nc[1] * t->nc[2], cudaMemcpyDeviceToDevice, st);
      break;
    }
    case 2:
      e = cudaMemcpyAsync(dst, t->d_pyr, sizeof(int16_t) * t->ncv * t->sd,
                          cudaMemcpyDeviceToDevice, st);
      break;
    case 3:
      e = cudaMemcpyAsync(dst, t->d_ti, (size_t)t->n[0] * t->n[1] * t->n[2],
                          cudaMemcpyDeviceToDevice, st);
      break;
    case 4:
      if (!t->d_tables) return fail(CCW_EINVAL, "no proposal attached");
      e = cudaMemcpyAsync(dst, t->d_tables, sizeof(__nv_bfloat16) * 16 * 64 * (size_t)t->P,
                          cudaMemcpyDeviceToDevice, st);
      break;
    default:
      return fail(CCW_EINVAL, "unknown export %d", what);
  }
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

int ccw_ccf_search(const ccw_ti* t, int32_t B, const uint8_t* de_dev, const uint8_t* hd_dev,
                   int32_t k, int32_t score_mode, uint64_t seed, const uint32_t* ctr_dev,
                   int32_t* topk_idx_dev, int32_t* topk_score_dev, int32_t* topk_mis_dev,
                   int32_t* pick_dev, void* stream) {
  return search_common(t, kModeSearch, B, de_dev, hd_dev, k, score_mode, seed, ctr_dev,
                       topk_idx_dev, topk_score_dev, topk_mis_dev, pick_dev, nullptr, nullptr,
                       stream);
}

int ccw_ccf_search_noalloc(const ccw_ti* t, int32_t B, const uint8_t* de_dev,
                           const uint8_t* hd_dev, int32_t k, int32_t score_mode, uint64_t seed,
                           const uint32_t* ctr_dev, int32_t* topk_idx_dev,
                           int32_t* topk_score_dev, int32_t* topk_mis_dev, int32_t* pick_dev,
                           void* stream) {
  if (!t) return fail(CCW_EINVAL, "ti is NULL");
  if (B < 0) return fail(CCW_EINVAL, "B must be >= 0");
  int sm, precision;
  if (int rc = split_mode(score_mode, sm, precision)) return rc;
  if (int rc = check_score_bound(t, sm)) return rc;
  if (int rc = check_precision(t, precision, sm, k)) return rc;
  precision &= 3;   // the format; checked above
  if (k < 1 || k > CCW_MAX_TOPK) return fail(CCW_EINVAL, "k must be in [1, %d]", CCW_MAX_TOPK);
  if (B == 0) return CCW_OK;
  if (!de_dev || !ctr_dev || !topk_idx_dev || !topk_score_dev || !topk_mis_dev || !pick_dev)
    return fail(CCW_EINVAL, "NULL input, output or counter");
  WaveArgs a;
  fill_ti(t, sm, a);
  event_layout(a.ti.nch, t->rows, t->TjP, hd_capacity(t), t->F, t->rows * t->Tj, a.ev);
  CcfPlan cp;
  plan_ccf(t, precision, a.ti.nch, k, B, a.ev, cp);
  const int64_t part_off = align_up(cp.ev_bytes, 256);
  const int64_t bmat_off = align_up(part_off + cp.part_bytes, 256);
  const int64_t need = bmat_off + cp.bmat_bytes;
  if (need > CCW_NOALLOC_SCRATCH_BYTES)
    return fail(CCW_EINVAL,
                "ccw_ccf_search_noalloc: B=%d with k=%d needs %lld scratch bytes, more than "
                "the %d-byte array; split the batch",
                B, k, (long long)need, CCW_NOALLOC_SCRATCH_BYTES);
  void* base = nullptr;
  if (int rc = noalloc_scratch(&base)) return rc;
  unsigned char* b = (unsigned char*)base;
  a.de = de_dev;
  a.hd = hd_dev;
  a.ctr = ctr_dev;
  a.K = k;
  a.seed = seed;
  a.topk_idx = topk_idx_dev;
  a.topk_score = topk_score_dev;
  a.topk_mis = topk_mis_dev;
  a.pick = pick_dev;
  // event records, ranking keys, weight matrix; every slot read is written
  // first in the same call, so nothing needs clearing
  // never profiled: the profiler's counters and timing events are allocated
  return run_explicit(t, kModeSearch, a, B, cp, b, (unsigned long long*)(b + part_off),
                      cp.bmat_bytes ? b + bmat_off : nullptr, (cudaStream_t)stream,
                      /*profiled=*/false);
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
  const int gd[3] = {sg_dims[0], sg_dims[1], sg_dims[2]};
  cudaError_t e = launch_idwt_paste(t->ndim, t->J, t->d_pyr, t->nc, t->cd, t->Tj, t->P, B,
                                    pick_dev, dst_origin_dev, sg_dev, gd, t->d_status,
                                    (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "paste kernel");
  ++g_launches;
  return CCW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ccw_simulate / ccw_simulate_groups
// ---------------------------------------------------------------------------
namespace {

// The all-shift phases of a 2D TI (built once): for phase (ph0, ph1) in
// [0, s)^2 the level-J planes of the blocks at (ph0 + s ux, ph1 + s uy), the
// candidate grid of the fine origins of that phase with origin + T <= n, and
// the planes' 8-shift copies for the tensor cores.
int prepare_phases(ccw_ti* t, cudaStream_t st) {
  if (t->n_phases) return CCW_OK;
  if (t->ndim != 2) return fail(CCW_EINVAL, "all-shift candidates are 2D only");
  const int s = t->s, T = t->T;
  t->fd[0] = t->n[0] - T + 1;
  t->fd[1] = t->n[1] - T + 1;
  t->P_fine = (int64_t)t->fd[0] * t->fd[1];
  if (t->P_fine >= (1 << 24)) return fail(CCW_EINVAL, "more than 2^24 - 1 all-shift candidates");
  std::vector<PhaseDev> ph;
  std::vector<void*> bufs;
  cudaError_t e = cudaSuccess;
  auto cleanup = [&]() {
    for (void* b : bufs) cudaFree(b);
  };
  for (int ph1 = 0; ph1 < s; ++ph1)
    for (int ph0 = 0; ph0 < s; ++ph0) {
      const int nc0 = (t->n[0] - ph0) / s, nc1 = (t->n[1] - ph1) / s;
      const int cd0 = nc0 - t->Tj + 1, cd1 = nc1 - t->Tj + 1;
      if (cd0 <= 0 || cd1 <= 0) continue;   // no fine origin of this phase fits
      PhaseDev d;
      memset(&d, 0, sizeof(d));
      d.ph0 = ph0;
      d.ph1 = ph1;
      d.cd0 = cd0;
      d.cd1 = cd1;
      d.px8 = (int)align_up(nc0, 8);
      d.mtiles = (int)(((int64_t)d.px8 * cd1 + 127) / 128);
      const int64_t roff_max = (int64_t)d.px8 * (t->Tj - 1);
      d.z8_nq = std::max<int64_t>(
          16LL * d.mtiles + 128 + (int64_t)(t->rows - 1) * d.px8 / 8 + 2 * (t->ks / 16) + 32,
          (128LL * (d.mtiles + kTcMaxMt) + roff_max + t->ks + 256) / 8 + 8);
      const int px = (int)align_up(nc0, 4);
      const int64_t pv = (int64_t)px * nc1;
      float* planes = nullptr;
      void *zf = nullptr, *zb = nullptr;
      const size_t zbytes = (size_t)t->F * d.z8_nq * 128;
      if ((e = cudaMalloc(&planes, sizeof(float) * pv * t->F)) != cudaSuccess ||
          (bufs.push_back(planes), (e = cudaMalloc(&zf, zbytes)) != cudaSuccess) ||
          (bufs.push_back(zf), (e = cudaMalloc(&zb, zbytes)) != cudaSuccess)) {
        cleanup();
        return fail(CCW_ENOMEM, "all-shift planes: %s", cudaGetErrorString(e));
      }
      bufs.push_back(zb);
      if ((e = cudaMemsetAsync(planes, 0, sizeof(float) * pv * t->F, st)) != cudaSuccess ||
          (e = launch_phase_planes(t->d_ti, t->n[0], s, t->F, ph0, ph1, nc0, nc1, planes, px,
                                   pv, st)) != cudaSuccess ||
          (e = launch_z8(planes, px, pv, nc0, nc1, d.px8, d.z8_nq, t->F, zf, zb, st)) !=
              cudaSuccess) {
        cleanup();
        return cuda_fail(e, "all-shift planes");
      }
      g_launches += 3;
      d.z8_f16 = zf;
      d.z8_bf16 = zb;
      ph.push_back(d);
    }
  t->h_phases = ph;
  t->phase_bufs = bufs;
  t->n_phases = (int)ph.size();
  return CCW_OK;
}

bool plan_matches(const SimPlan* pl, const ccw_params* p, const ccw_group* groups, int n_groups) {
  if (!pl || pl->n_groups != n_groups || pl->K != p->topk || pl->score_mode != p->score_mode ||
      pl->precision != p->precision || pl->learned != p->learned ||
      pl->ccf_tile != p->ccf_tile || pl->vt_ext != p->vt_ext || pl->cut != p->boundary_cut ||
      pl->all_shift != p->all_shift)
    return false;
  for (int i = 0; i < n_groups; ++i) {
    const GroupPlan& g = pl->groups[i];
    if (g.n_real != groups[i].n_real) return false;
    for (int a = 0; a < 3; ++a)
      if (g.grid[a] != groups[i].grid[a]) return false;
  }
  return true;
}

int build_plan(ccw_ti* t, const ccw_params* p, const ccw_group* groups, int n_groups,
               SimPlan*& out) {
  SimPlan* pl = new SimPlan();
  const int d = t->ndim;
  const int T = t->T, S = t->T - t->O;
  pl->n_groups = n_groups;
  pl->groups.resize(n_groups);
  pl->K = p->topk;
  pl->score_mode = p->score_mode;
  pl->precision = p->precision;
  pl->learned = p->learned;
  pl->ccf_tile = p->ccf_tile;
  pl->vt_ext = p->vt_ext;
  pl->cut = p->boundary_cut;
  pl->all_shift = p->all_shift;
  pl->n_prop = p->learned ? t->n_prop : 0;
  pl->n_waves = 0;
  for (int i = 0; i < n_groups; ++i) {
    GroupPlan& g = pl->groups[i];
    g.n_real = groups[i].n_real;
    for (int a = 0; a < 3; ++a) {
      g.grid[a] = groups[i].grid[a];
      g.g[a] = groups[i].grid[a];
      if (a < d) {
        const int extra = g.g[a] > T ? g.g[a] - T : 0;
        g.np[a] = 1 + (extra + S - 1) / S;
        g.gp[a] = T + (g.np[a] - 1) * S;
      } else {
        g.np[a] = 1;
        g.gp[a] = 1;
      }
    }
    g.n_patches = (int64_t)g.np[0] * g.np[1] * g.np[2];
    g.gp_vol = (int64_t)g.gp[0] * g.gp[1] * g.gp[2];
    g.g_vol = (int64_t)g.g[0] * g.g[1] * g.g[2];
    pl->n_waves = std::max(pl->n_waves,
                           (g.np[0] - 1) + 2 * (g.np[1] - 1) + 4 * (g.np[2] - 1) + 1);
  }
  // realization lanes (ccf_tile bits 20-22: lanes - 1); one lane for the
  // learned proposal and the one-kernel form
  int n_lanes = tile_lanes(p->ccf_tile);
  int64_t total_real = 0;
  for (int i = 0; i < n_groups; ++i) total_real += pl->groups[i].n_real;
  if (p->learned || tile_is_persist(p->precision & 3, p->ccf_tile)) n_lanes = 1;
  n_lanes = (int)std::max<int64_t>(1, std::min<int64_t>(n_lanes, total_real));
  // wavefront schedule: wave(p) = ix + 2 iy + 4 iz over the lattice index of
  // every group; the items of one wave of all groups (of one lane) share the
  // launches; lane l takes slots [l n / L, (l + 1) n / L) of every group
  std::vector<std::vector<std::vector<int4>>> waves(
      n_lanes, std::vector<std::vector<int4>>(pl->n_waves));
  // Within a wave the items run patch-major: consecutive items are the same
  // patch of successive realizations, so they share the overlap mask type
  // (the learned proposal's selector scores one table per CTA).
  for (int i = 0; i < n_groups; ++i) {
    const GroupPlan& g = pl->groups[i];
    for (int64_t pp = 0; pp < g.n_patches; ++pp) {
      const int ix = (int)(pp % g.np[0]), iy = (int)((pp / g.np[0]) % g.np[1]),
                iz = (int)(pp / ((int64_t)g.np[0] * g.np[1]));
      for (int r = 0; r < g.n_real; ++r) {
        const int lane = (int)((int64_t)r * n_lanes / g.n_real);
        waves[lane][ix + 2 * iy + 4 * iz].push_back(make_int4(i, r, (int)pp, 0));
      }
    }
  }
  std::vector<int4> items;
  const bool learned_fused =
      p->learned && nnsel_fuses_rerank_shape(t->P, p->score_mode == 0 ? t->F - 1 : 1, t->rows,
                                             t->Tj, t->n_prop);
  pl->lanes.resize(n_lanes);
  pl->max_items = 0;
  pl->launches_per_call = 0;
  for (int l = 0; l < n_lanes; ++l) {
    SimPlan::Lane& ln = pl->lanes[l];
    ln.wave_off.assign(pl->n_waves + 1, 0);
    for (int w = 0; w < pl->n_waves; ++w) {
      ln.wave_off[w] = (int64_t)items.size();
      items.insert(items.end(), waves[l][w].begin(), waves[l][w].end());
      ln.max_items = std::max<int>(ln.max_items, (int)waves[l][w].size());
      // learned: events, the encoder, the selector, the re-rank unless the
      // selector does it, the CCF of the fallbacks, finish
      pl->launches_per_call +=
          (p->learned ? 4 + encode_items_launches(t->F, t->Tj, t->d_enc_img != nullptr) +
                            (learned_fused ? 0 : 1)
                      : 3) *
          ((waves[l][w].size() + 65534) / 65535);
    }
    ln.wave_off[pl->n_waves] = (int64_t)items.size();
    pl->max_items = std::max(pl->max_items, ln.max_items);
  }
  pl->wave_off = pl->lanes[0].wave_off;
  const int nch = p->score_mode == 0 ? t->F - 1 : 1;
  event_layout(nch, t->rows, t->TjP, hd_capacity(t, p->vt_ext), t->F, t->rows * t->Tj, pl->evl);
  CcfPlan* cp = new CcfPlan();
  pl->cp = cp;
  const int fmt = p->precision & 3;   // the format (the exactness flag was checked)
  const int tiling = p->ccf_tile & ~kTileLaneMask;
  if (tile_is_persist(fmt, tiling)) {
    cp->precision = fmt;
    if (int rc = plan_persist(t, nch, pl->K, pl->max_items, tiling, p->vt_ext,
                              p->boundary_cut, p->learned, *cp)) {
      delete pl;
      return rc;
    }
    cp->ev_bytes = (int64_t)pl->max_items * pl->evl.stride;
  } else {
    plan_ccf(t, fmt, nch, pl->K, pl->max_items, pl->evl, *cp, tiling);
    if (p->all_shift) {
      // every phase is searched by the CTAs of its grid layer, with the
      // decimated plan's tiling; key lists [phase M-groups] per item
      std::vector<PhaseDev> ph = t->h_phases;
      const int mt = cp->tc.mt;
      int parts = 0, mg_max = 0, a_nq_max = 0;
      for (PhaseDev& d : ph) {
        d.a_nq = 16 * (mt - 1) + (t->rows - 1) * d.px8 / 8 + 2 * (t->ks / 16 - 1) + 17;
        d.n_mgroups = (d.mtiles + mt - 1) / mt;
        d.part_base = parts;
        parts += d.n_mgroups;
        mg_max = std::max(mg_max, d.n_mgroups);
        a_nq_max = std::max(a_nq_max, d.a_nq);
      }
      cp->tc.a_nq = a_nq_max;
      cp->tc.n_mgroups = mg_max;
      cp->n_parts = parts;
      cp->smem = tc_smem_bytes(nch, a_nq_max, cp->tc.ksteps, cp->tc.nt, pl->K, cp->tc.tc_lane_epi);
      cp->part_bytes = (int64_t)pl->max_items * parts * pl->K * 8;
      pl->n_phases = (int)ph.size();
      if (cudaMalloc((void**)&pl->d_phases, sizeof(PhaseDev) * ph.size()) != cudaSuccess ||
          cudaMemcpy(pl->d_phases, ph.data(), sizeof(PhaseDev) * ph.size(),
                     cudaMemcpyHostToDevice) != cudaSuccess) {
        delete pl;
        return fail(CCW_ENOMEM, "all-shift phase table");
      }
    }
  }
  if (!cp->persist && cp->smem > 220 * 1024) {
    const int need = cp->smem;   // the plan owns cp
    delete pl;
    return fail(CCW_EINVAL, "ccf_tile 0x%x needs %d bytes of shared memory", p->ccf_tile, need);
  }
  cudaError_t e = cudaSuccess;
  for (auto& g : pl->groups) {
    if ((e = cudaMalloc(&g.sg, (size_t)g.gp_vol * g.n_real)) != cudaSuccess ||
        (e = cudaMalloc(&g.overlay, (size_t)align_up(g.g_vol, 4))) != cudaSuccess)
      break;
  }
  if (e != cudaSuccess ||
      (e = cudaMalloc(&pl->items, sizeof(int4) * std::max<size_t>(items.size(), 1))) !=
          cudaSuccess ||
      (e = cudaMalloc(&pl->ev, (size_t)cp->ev_bytes)) != cudaSuccess ||
      (e = cudaMalloc(&pl->part, (size_t)cp->part_bytes)) != cudaSuccess ||
      (cp->bmat_bytes && (e = cudaMalloc(&pl->bmat, (size_t)cp->bmat_bytes)) != cudaSuccess) ||
      (pl->learned &&
       ((e = cudaMalloc(&pl->emb, sizeof(float) * 64 * (size_t)pl->max_items)) != cudaSuccess ||
        (e = cudaMalloc(&pl->prop, sizeof(int) * (size_t)pl->n_prop * pl->max_items)) !=
            cudaSuccess ||
        (e = cudaMalloc(&pl->prop_gap, sizeof(float) * (size_t)pl->max_items)) !=
            cudaSuccess ||
        (e = cudaMalloc(&pl->enc_x, sizeof(float) * (size_t)t->F * t->Tj * t->Tj *
                                        pl->max_items)) != cudaSuccess ||
        (e = cudaMalloc(&pl->enc_act, sizeof(float) * (size_t)infer_act_floats(t->F, t->Tj) *
                                          pl->max_items)) != cudaSuccess)) ||
      (e = cudaMalloc((void**)&pl->call, sizeof(CallDev))) != cudaSuccess ||
      (e = cudaMalloc((void**)&pl->dgroups, sizeof(SimGroup) * n_groups)) != cudaSuccess ||
      (cp->persist &&
       ((e = cudaMalloc((void**)&pl->wave_off_d, sizeof(int64_t) * (pl->n_waves + 1))) !=
            cudaSuccess ||
        (e = cudaMalloc((void**)&pl->gbar, 2 * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc((void**)&pl->phase_ns, 3 * sizeof(unsigned long long))) !=
            cudaSuccess))) {
    delete pl;
    return fail(CCW_ENOMEM, "simulation workspace: %s", cudaGetErrorString(e));
  }
  pl->lanes[0].ev = pl->ev;
  pl->lanes[0].part = pl->part;
  pl->lanes[0].bmat = pl->bmat;
  for (size_t l = 1; l < pl->lanes.size(); ++l) {
    SimPlan::Lane& ln = pl->lanes[l];
    if ((e = cudaMalloc(&ln.ev, (size_t)cp->ev_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&ln.part, (size_t)cp->part_bytes)) != cudaSuccess ||
        (cp->bmat_bytes && (e = cudaMalloc(&ln.bmat, (size_t)cp->bmat_bytes)) != cudaSuccess) ||
        (e = cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming)) != cudaSuccess) {
      delete pl;
      return fail(CCW_ENOMEM, "simulation lane workspace: %s", cudaGetErrorString(e));
    }
  }
  pl->evl.base = (unsigned char*)pl->ev;
  if ((cp->persist &&
       (e = cudaMemcpy(pl->wave_off_d, pl->wave_off.data(), sizeof(int64_t) * (pl->n_waves + 1),
                       cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemcpy(pl->items, items.data(), sizeof(int4) * items.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking)) != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "simulation plan");
  }
  out = pl;
  return CCW_OK;
}

// Output rows of group g that become final with wavefront w, as a range
// [b0, b1) of indices along the slowest axis (y in 2D, z in 3D); b0 == b1
// when none. Patch row i of that axis (lattice index i_y in 2D, i_z in 3D)
// ends with the wave of its last patch, (np_x - 1) + 2 i in 2D and
// (np_x - 1) + 2 (np_y - 1) + 4 i in 3D; the next patch row starts at
// (i + 1)(T - OR), so every row before it is final from then on.
void band_at_wave(const GroupPlan& g, int d, int S, int w, int& b0, int& b1) {
  b0 = b1 = 0;
  const int slow = d - 1, step = d == 3 ? 4 : 2;
  const int base = (g.np[0] - 1) + (d == 3 ? 2 * (g.np[1] - 1) : 0);
  if (w < base || (w - base) % step) return;
  const int i = (w - base) / step;
  if (i >= g.np[slow]) return;
  const int G = g.g[slow];
  b0 = std::min(G, i * S);
  b1 = i == g.np[slow] - 1 ? G : std::min(G, (i + 1) * S);
}

// Streamed read-back after wavefront w of lane `lane` (captured on `st`):
// every band that wave completes is cropped into out_dev and copied to
// out_host on the lane's copy stream, for the lane's realizations.
int launch_band_copies(ccw_ti* t, SimPlan* pl, const ccw_group* hosts, int lane, int w,
                       cudaStream_t st, std::vector<char>& used) {
  const int d = t->ndim, S = t->T - t->O, L = (int)pl->lanes.size();
  bool forked = false;
  for (int i = 0; i < pl->n_groups; ++i) {
    const GroupPlan& g = pl->groups[i];
    if (!hosts[i].out_host) continue;
    int b0, b1;
    band_at_wave(g, d, S, w, b0, b1);
    if (b0 >= b1) continue;
    // the lane's realizations: slots r with r L / n_real == lane
    const int r0 = (int)(((int64_t)lane * g.n_real + L - 1) / L);
    const int r1 = (int)(((int64_t)(lane + 1) * g.n_real + L - 1) / L);
    if (r0 >= r1) continue;
    cudaError_t e;
    if (!forked) {
      if ((e = cudaEventRecord(pl->cev[lane], st)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(pl->cst[lane], pl->cev[lane], 0)) != cudaSuccess)
        return cuda_fail(e, "read-back fork");
      forked = true;
      used[lane] = 1;
    }
    const int rs = d == 3 ? g.g[1] : 1;   // output rows per slow-axis index
    const int64_t vol = g.g_vol;
    uint8_t* dev = hosts[i].out_dev + r0 * vol;
    if ((e = launch_crop_out((const uint8_t*)g.sg + r0 * g.gp_vol, g.gp_vol, g.gp, dev, g.g, d,
                             r1 - r0, 0, 0, hosts[i].real_base + r0, pl->cst[lane], b0 * rs,
                             b1 * rs)) != cudaSuccess)
      return cuda_fail(e, "crop kernel");
    ++pl->host_launches;
    const size_t off = (size_t)b0 * rs * g.g[0];
    if ((e = cudaMemcpy2DAsync(hosts[i].out_host + r0 * vol + off, (size_t)vol, dev + off,
                               (size_t)vol, (size_t)(b1 - b0) * rs * g.g[0], (size_t)(r1 - r0),
                               cudaMemcpyDeviceToHost, pl->cst[lane])) != cudaSuccess)
      return cuda_fail(e, "read-back copy");
  }
  return CCW_OK;
}

// Launch phases A, B and C of every wave of lane `lane` on `st` (while `st`
// is being captured into the plan's graph); `pe` counts the profiled steps.
// With `hosts`, also the streamed read-back of the bands each wave completes.
int launch_waves(ccw_ti* t, SimPlan* pl, bool prof, int lane, cudaStream_t st, size_t& pe,
                 const ccw_group* hosts, std::vector<char>& used) {
  const SimPlan::Lane& ln = pl->lanes[lane];
  WaveArgs a;
  fill_ti(t, pl->score_mode, a);
  a.ev = pl->evl;
  a.ev.base = (unsigned char*)ln.ev;
  a.groups = pl->dgroups;
  a.S = t->T - t->O;
  a.call = pl->call;
  a.K = pl->K;
  a.part = (unsigned long long*)ln.part;
  a.vt_ext = pl->vt_ext;
  a.cut = pl->cut;
  if (pl->all_shift) {
    a.allshift = 1;
    a.phases = pl->d_phases;
    a.n_phases = pl->n_phases;
    a.fd0 = t->fd[0];
    a.ti.P = t->P_fine;   // draws and K' range over the fine candidates
  }
  if (pl->learned) {
    a.learned = 1;
    a.net = t->d_net;
    a.tables = t->d_tables;
    a.tables_mma = t->d_tables_mma;
    a.enc_img = t->d_enc_img;
    a.n_prop = pl->n_prop;
    a.emb = (float*)pl->emb;
    a.prop = (int*)pl->prop;
    a.prop_gap = (float*)pl->prop_gap;
    a.enc_x = (float*)pl->enc_x;
    a.enc_act = (float*)pl->enc_act;
  }
  const CcfPlan& cp = *static_cast<const CcfPlan*>(pl->cp);
  for (int w = 0; w < pl->n_waves; ++w) {
    for (int64_t i0 = ln.wave_off[w]; i0 < ln.wave_off[w + 1]; i0 += 65535) {
      WaveArgs c = a;
      c.items = (const int4*)pl->items + i0;
      c.n_items = (int)std::min<int64_t>(65535, ln.wave_off[w + 1] - i0);
      if (c.n_items <= 0) continue;
      apply_ccf(t, cp, ln.bmat, c);
      if (prof) {
        if (pe >= pl->prof_bounds.size()) {
          cudaEvent_t e0, e1;
          cudaEventCreate(&e0);
          cudaEventCreate(&e1);
          pl->prof_bounds.emplace_back(e0, e1);
        }
        cudaEventRecordWithFlags(pl->prof_bounds[pe].first, st, cudaEventRecordExternal);
      }
      cudaError_t e = launch_events(kModeSim, c, true, st);
      if (e != cudaSuccess) return cuda_fail(e, "event kernel launch");
      if (pl->learned) {
        // learned proposal: embed, nearest windows, exact re-rank; the CCF
        // kernel then skips the items the proposal settled
        cudaEvent_t* pev = nullptr;
        if (prof) {
          while (pl->prof_prop.size() < 3 * (pe + 1)) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            pl->prof_prop.push_back(ev);
          }
          pev = &pl->prof_prop[3 * pe];
          cudaEventRecordWithFlags(pev[0], st, cudaEventRecordExternal);
        }
        if ((e = launch_encode_items(c, c.enc_x, c.enc_act, !prof, st)) != cudaSuccess)
          return cuda_fail(e, "proposal kernel launch");
        if (prof) cudaEventRecordWithFlags(pev[1], st, cudaEventRecordExternal);
        if ((e = launch_nnsel(c, !prof, st)) != cudaSuccess ||
            (!nnsel_fuses_rerank(c) && (e = launch_rerank(c, true, st)) != cudaSuccess))
          return cuda_fail(e, "proposal kernel launch");
        if (prof) cudaEventRecordWithFlags(pev[2], st, cudaEventRecordExternal);
      }
      if (prof) {
        if (pe >= pl->prof_events.size()) {
          cudaEvent_t e0, e1;
          cudaEventCreate(&e0);
          cudaEventCreate(&e1);
          pl->prof_events.emplace_back(e0, e1);
        }
        cudaEventRecordWithFlags(pl->prof_events[pe].first, st, cudaEventRecordExternal);
      }
      e = launch_ccf(t, kModeSim, cp, c, !prof, st);
      if (e != cudaSuccess) return cuda_fail(e, "CCF kernel launch");
      if (prof)
        cudaEventRecordWithFlags(pl->prof_events[pe].second, st, cudaEventRecordExternal);
      e = launch_finish(kModeSim, c, !prof, st);
      if (e != cudaSuccess) return cuda_fail(e, "finish kernel launch");
      if (prof) cudaEventRecordWithFlags(pl->prof_bounds[pe++].second, st, cudaEventRecordExternal);
    }
    if (hosts)
      if (int rc = launch_band_copies(t, pl, hosts, lane, w, st, used)) return rc;
  }
  return CCW_OK;
}

int capture_waves(ccw_ti* t, SimPlan* pl, bool prof, const ccw_group* hosts = nullptr) {
  cudaGraph_t graph = nullptr;
  const size_t nl = pl->lanes.size();
  std::vector<char> used(nl, 0);   // lanes whose copy stream joined the capture
  if (hosts) {
    pl->host_launches = 0;
    while (pl->cst.size() < nl) {
      cudaStream_t cs = nullptr;
      cudaEvent_t ce = nullptr;
      cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ce, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        if (cs) cudaStreamDestroy(cs);
        return cuda_fail(e, "read-back streams");
      }
      pl->cst.push_back(cs);
      pl->cev.push_back(ce);
    }
  }
  cudaError_t e = cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "begin capture");
  // lanes >= 1 fork from the capture stream and join it at the end
  int rc = CCW_OK;
  size_t pe = 0;
  cudaEvent_t fork = nullptr;
  if (pl->lanes.size() > 1) {
    if ((e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(fork, pl->cap)) != cudaSuccess)
      rc = cuda_fail(e, "capture fork");
    for (size_t l = 1; l < pl->lanes.size() && !rc; ++l)
      if ((e = cudaStreamWaitEvent(pl->lanes[l].st, fork, 0)) != cudaSuccess)
        rc = cuda_fail(e, "capture fork");
  }
  for (size_t l = 0; l < pl->lanes.size() && !rc; ++l)
    rc = launch_waves(t, pl, prof, (int)l, l == 0 ? pl->cap : pl->lanes[l].st, pe, hosts, used);
  for (size_t l = 1; l < pl->lanes.size() && !rc; ++l)
    if ((e = cudaEventRecord(pl->lanes[l].done, pl->lanes[l].st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(pl->cap, pl->lanes[l].done, 0)) != cudaSuccess)
      rc = cuda_fail(e, "capture join");
  for (size_t l = 0; l < nl; ++l)   // copy streams join even after an error
    if (used[l] && ((e = cudaEventRecord(pl->cev[l], pl->cst[l])) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(pl->cap, pl->cev[l], 0)) != cudaSuccess) &&
        !rc)
      rc = cuda_fail(e, "read-back join");
  e = cudaStreamEndCapture(pl->cap, &graph);
  if (fork) cudaEventDestroy(fork);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  e = cudaGraphInstantiate(hosts ? &pl->exec_host : &pl->exec[prof ? 1 : 0], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
  return CCW_OK;
}

// The whole call as one cooperative kernel (persist.cu), launched on `st`.
int launch_persist_call(ccw_ti* t, SimPlan* pl, bool prof, cudaStream_t st) {
  const CcfPlan& cp = *static_cast<const CcfPlan*>(pl->cp);
  WaveArgs a;
  fill_ti(t, pl->score_mode, a);
  a.ev = pl->evl;
  a.groups = pl->dgroups;
  a.S = t->T - t->O;
  a.call = pl->call;
  a.K = pl->K;
  a.part = (unsigned long long*)pl->part;
  a.items = (const int4*)pl->items;
  a.precision = cp.precision;
  a.z8 = cp.precision == 2 ? t->z8_bf16 : t->z8_f16;
  a.z8_nq = cp.tc.z8_nq;
  a.px8 = cp.tc.px8;
  a.ks = cp.tc.ks;
  a.ksteps = cp.tc.ksteps;
  a.mtiles = cp.tc.mtiles;
  a.mt = cp.tc.mt;
  a.n_mgroups = cp.tc.n_mgroups;
  a.nt = cp.tc.nt;
  a.a_nq = cp.tc.a_nq;
  a.bmat = pl->bmat;
  a.n_parts = cp.n_parts;
  a.wave_off = pl->wave_off_d;
  a.n_waves = pl->n_waves;
  a.gbar = pl->gbar;
  a.spin_limit = g_barrier_polls.load();
  a.gw = cp.p_gw;
  a.phase_ns = prof ? pl->phase_ns : nullptr;
  cudaError_t e;
  if ((e = cudaMemsetAsync(pl->gbar, 0, 2 * sizeof(unsigned), st)) != cudaSuccess ||
      (prof && (e = cudaMemsetAsync(pl->phase_ns, 0, 3 * sizeof(unsigned long long), st)) !=
                   cudaSuccess))
    return cuda_fail(e, "persistent kernel setup");
  if (prof) {
    for (auto& ev : pl->pev)
      if (!ev && (e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "event");
    cudaEventRecord(pl->pev[0], st);
  }
  if ((e = launch_persist(a, cp.smem, cp.p_grid, st)) != cudaSuccess)
    return cuda_fail(e, "persistent kernel launch");
  ++g_launches;
  if (prof) cudaEventRecord(pl->pev[1], st);
  return CCW_OK;
}

int simulate_groups(ccw_ti* t, const ccw_params* p, const ccw_group* groups, int n_groups,
                    uint64_t seed, void* stream) {
  const int d = t->ndim;
  if (p->ndim != d) return fail(CCW_EINVAL, "params ndim %d != TI ndim %d", p->ndim, d);
  if (p->topk < 1 || p->topk > CCW_MAX_TOPK)
    return fail(CCW_EINVAL, "topk must be in [1, %d]", CCW_MAX_TOPK);
  if (p->score_mode != 0 && p->score_mode != 1) return fail(CCW_EINVAL, "bad score_mode");
  if (int rc = check_precision(t, p->precision, p->score_mode, p->topk, p->ccf_tile)) return rc;
  if (p->path_random != 0 && p->path_random != 1) return fail(CCW_EINVAL, "bad path_random");
  if (p->learned != 0 && p->learned != 1) return fail(CCW_EINVAL, "bad learned flag");
  if (!valid_tile_hint(t, p->precision & 3, p->ccf_tile))
    return fail(CCW_EINVAL, "ccf_tile 0x%x is not a valid tiling for precision %d", p->ccf_tile,
                p->precision);
  if (p->learned) {
    if (!t->d_tables) return fail(CCW_EINVAL, "learned = 1 needs an attached proposal");
    if (p->score_mode != 0) return fail(CCW_EINVAL, "learned = 1 needs the one-hot score");
    if (p->topk > t->n_prop) return fail(CCW_EINVAL, "topk > the proposal's n_prop");
  }
  if (p->vt_ext < 0 || p->vt_ext > t->T)
    return fail(CCW_EINVAL, "vt_ext must be in [0, templ = %d]", t->T);
  if (p->boundary_cut != 0 && p->boundary_cut != 1) return fail(CCW_EINVAL, "bad boundary_cut");
  if (p->all_shift != 0 && p->all_shift != 1) return fail(CCW_EINVAL, "bad all_shift");
  if (p->all_shift &&
      (d != 2 || (p->precision & 3) == 0 || p->learned || p->boundary_cut ||
       ((p->ccf_tile >> 25) & 1) || tile_is_persist(p->precision & 3, p->ccf_tile)))
    return fail(CCW_EINVAL,
                "all_shift needs 2D, precision 1 or 2 with resident operands, and no learned "
                "proposal, boundary cut or one-kernel form");
  if (p->boundary_cut && (d != 2 || t->T > kMaxCutTempl))
    return fail(CCW_EINVAL, "the boundary cut needs 2D and templ <= %d", kMaxCutTempl);
  if (int rc = check_score_bound(t, p->score_mode)) return rc;
  if (n_groups < 1 || !groups) return fail(CCW_EINVAL, "at least one grid group is needed");
  for (int i = 0; i < n_groups; ++i) {
    const ccw_group& g = groups[i];
    if (g.n_real < 1) return fail(CCW_EINVAL, "group %d: n_real must be >= 1", i);
    if (g.real_base < 0) return fail(CCW_EINVAL, "group %d: real_base must be >= 0", i);
    if (!g.out_dev) return fail(CCW_EINVAL, "group %d: out_dev is NULL", i);
    if (g.n_hd < 0 || (g.n_hd > 0 && (!g.hd_cells_dev || !g.hd_vals_dev)))
      return fail(CCW_EINVAL, "group %d: bad hard data", i);
    if (g.event_counts_dev && t->sd > 255)
      return fail(CCW_EINVAL, "group %d: block counts need 2^(d J) <= 255", i);
    for (int a = 0; a < 3; ++a)
      if (g.grid[a] <= 0 || (a >= d && g.grid[a] != 1))
        return fail(CCW_EINVAL, "group %d: bad grid dims", i);
  }

  std::lock_guard<std::mutex> lock(t->mu);
  cudaStream_t st = (cudaStream_t)stream;
  if (p->all_shift)
    if (int rc = prepare_phases(t, st)) return rc;
  SimPlan* pl = t->plan;
  if (!plan_matches(pl, p, groups, n_groups)) {
    cudaDeviceSynchronize();
    delete t->plan;
    t->plan = nullptr;
    if (int rc = build_plan(t, p, groups, n_groups, pl)) return rc;
    t->plan = pl;
  }
  bool prof;
  unsigned long long* work = nullptr;
  {
    std::lock_guard<std::mutex> g(g_prof.mu);
    prof = g_prof.enabled;
    if (prof) work = profiling_counters();
  }
  CallDev call;
  call.seed = seed;
  call.path_random = p->path_random;
  call.log_stride = 4 + p->topk;
  call.work = work;
  call.gap_theta = t->gap_theta;
  call.learn_stats = t->d_learn_stats;
  std::vector<SimGroup> hg(n_groups);
  for (int i = 0; i < n_groups; ++i) {
    const GroupPlan& g = pl->groups[i];
    SimGroup& s = hg[i];
    s.sg = (uint8_t*)g.sg;
    s.overlay = groups[i].n_hd > 0 ? (const uint8_t*)g.overlay : nullptr;
    for (int a = 0; a < 3; ++a) {
      s.G[a] = g.g[a];
      s.Gp[a] = g.gp[a];
      s.np[a] = g.np[a];
    }
    s.gp_vol = g.gp_vol;
    s.n_patches = g.n_patches;
    s.real_base = groups[i].real_base;
    s.log = groups[i].patch_log_dev;
    s.counts = groups[i].event_counts_dev;
  }
  cudaError_t e;
  if ((e = cudaMemcpyAsync(pl->call, &call, sizeof(call), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(pl->dgroups, hg.data(), sizeof(SimGroup) * n_groups,
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(t->d_status, 0, sizeof(int), st)) != cudaSuccess)
    return cuda_fail(e, "simulation setup");
  for (int i = 0; i < n_groups; ++i) {
    const GroupPlan& g = pl->groups[i];
    const ccw_group& u = groups[i];
    if ((e = cudaMemsetAsync(g.sg, 0xFF, (size_t)g.gp_vol * g.n_real, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(g.overlay, 0xFF, (size_t)align_up(g.g_vol, 4), st)) != cudaSuccess)
      return cuda_fail(e, "simulation setup");
    if ((e = launch_hd_overlay(u.hd_cells_dev, u.hd_vals_dev, u.n_hd, d, g.g, t->F,
                               (uint8_t*)g.overlay, t->d_status, st)) != cudaSuccess)
      return cuda_fail(e, "hard-data kernel");
    if (u.n_hd > 0) ++g_launches;
    if (u.patch_log_dev &&
        (e = cudaMemsetAsync(u.patch_log_dev, 0xFF,
                             sizeof(int32_t) * (size_t)g.n_real * g.n_patches * (4 + p->topk),
                             st)) != cudaSuccess)
      return cuda_fail(e, "log clear");
  }
  const bool persist = static_cast<const CcfPlan*>(pl->cp)->persist;
  // host read-back: streamed inside the graph when every host buffer is
  // pinned and the paths are unmirrored (a band of rows is then the same
  // rows of every realization), else one copy per group after the crop
  bool any_host = false, all_pinned = true;
  for (int i = 0; i < n_groups; ++i) {
    if (!groups[i].out_host) continue;
    any_host = true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, groups[i].out_host) != cudaSuccess ||
        at.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      all_pinned = false;
    }
  }
  const bool stream_host = any_host && all_pinned && !prof && !persist && p->path_random == 0;
  if (persist) {
    if (int rc = launch_persist_call(t, pl, prof, st)) return rc;
  } else if (stream_host) {
    bool same = pl->exec_host && (int)pl->host_dev.size() == n_groups;
    for (int i = 0; same && i < n_groups; ++i)
      same = pl->host_dev[i] == groups[i].out_dev && pl->host_host[i] == groups[i].out_host;
    if (!same) {
      if (pl->exec_host) cudaGraphExecDestroy(pl->exec_host);
      pl->exec_host = nullptr;
      pl->host_dev.clear();
      pl->host_host.clear();
      if (int rc = capture_waves(t, pl, false, groups)) return rc;
      for (int i = 0; i < n_groups; ++i) {
        pl->host_dev.push_back(groups[i].out_dev);
        pl->host_host.push_back(groups[i].out_host);
      }
    }
    if ((e = cudaGraphLaunch(pl->exec_host, st)) != cudaSuccess)
      return cuda_fail(e, "graph launch");
    g_launches += pl->launches_per_call + pl->host_launches;
  } else {
    const int gi = prof ? 1 : 0;
    if (!pl->exec[gi])
      if (int rc = capture_waves(t, pl, prof)) return rc;
    if ((e = cudaGraphLaunch(pl->exec[gi], st)) != cudaSuccess)
      return cuda_fail(e, "graph launch");
    g_launches += pl->launches_per_call;
  }
  for (int i = 0; i < n_groups; ++i) {
    const GroupPlan& g = pl->groups[i];
    if (stream_host && groups[i].out_host) continue;   // cropped and copied in the graph
    if ((e = launch_crop_out((const uint8_t*)g.sg, g.gp_vol, g.gp, groups[i].out_dev, g.g, d,
                             g.n_real, p->path_random, seed, groups[i].real_base, st)) !=
        cudaSuccess)
      return cuda_fail(e, "crop kernel");
    ++g_launches;
    if (groups[i].out_host &&
        (e = cudaMemcpyAsync(groups[i].out_host, groups[i].out_dev, (size_t)(g.g_vol * g.n_real),
                             cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "read-back copy");
  }
  int status = 0;
  if ((e = cudaMemcpyAsync(&status, t->d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "simulation");
  if (prof && persist) {
    // the persistent kernel's launch time; its phases from the device clock
    std::lock_guard<std::mutex> g(g_prof.mu);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pl->pev[0], pl->pev[1]) == cudaSuccess) {
      g_prof.total_ms += ms;
      ++g_prof.launches;
    }
    unsigned long long ns[3] = {0, 0, 0};
    if (cudaMemcpy(ns, pl->phase_ns, sizeof(ns), cudaMemcpyDeviceToHost) == cudaSuccess)
      for (int i = 0; i < 3; ++i) g_prof.phase_ms[i] += 1e-6 * (double)ns[i];
  } else if (prof) {
    std::lock_guard<std::mutex> g(g_prof.mu);
    for (size_t i = 0; i < pl->prof_events.size(); ++i) {
      const auto& pr = pl->prof_events[i];
      const auto& bd = pl->prof_bounds[i];
      float ms = 0.f, ev = 0.f, fin = 0.f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
        g_prof.total_ms += ms;
        ++g_prof.launches;
        g_prof.phase_ms[1] += ms;
      }
      if (cudaEventElapsedTime(&ev, bd.first, pr.first) == cudaSuccess) g_prof.phase_ms[0] += ev;
      if (cudaEventElapsedTime(&fin, pr.second, bd.second) == cudaSuccess)
        g_prof.phase_ms[2] += fin;
      if (pl->learned && pl->prof_prop.size() >= 3 * (i + 1)) {
        float enc = 0.f, sel = 0.f;
        if (cudaEventElapsedTime(&enc, pl->prof_prop[3 * i], pl->prof_prop[3 * i + 1]) ==
            cudaSuccess)
          g_prof.prop_ms[0] += enc;
        if (cudaEventElapsedTime(&sel, pl->prof_prop[3 * i + 1], pl->prof_prop[3 * i + 2]) ==
            cudaSuccess)
          g_prof.prop_ms[1] += sel;
      }
    }
  }
  if (status & kStatusBadCode)
    return fail(CCW_EINVAL, "hard data out of the grid or with a code >= n_facies");
  if (status & kStatusHdOverflow)
    return fail(CCW_EINVAL,
                "more than %d hard data in one template window (virtual template included)",
                kMaxHd);
  if (status & kStatusTimeout) return fail(CCW_ETIMEOUT, "a bounded device wait gave up");
  return CCW_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Learned proposal (an addition of this library; the paper has no
// counterpart).
// ---------------------------------------------------------------------------
namespace {
bool usable_mask_type(int type) { return type != 0 && (type & 3) != 3 && (type & 12) != 12; }

// Minimal event records for the query entry point: meta and block counts.
EvDev query_records(const ccw_ti* t, void* base) {
  EvDev ev;
  memset(&ev, 0, sizeof(ev));
  ev.base = (unsigned char*)base;
  ev.counts_off = 64;
  ev.stride = align_up(64 + (int64_t)t->F * t->Tj * t->Tj, 16);
  return ev;
}
}  // namespace

extern "C" int ccw_ti_attach_proposal(ccw_ti* t, const ccw_net* net, int32_t n_prop,
                                      float gap_theta, void* stream) {
  if (!t) return fail(CCW_EINVAL, "NULL TI");
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(t->mu);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "attach proposal");
  // a captured plan holds the old table pointers
  delete t->plan;
  t->plan = nullptr;
  cudaFree(t->d_net);
  cudaFree(t->d_tables);
  cudaFree(t->d_tables_mma);
  cudaFree(t->d_enc_img);
  t->d_net = nullptr;
  t->d_tables = nullptr;
  t->d_tables_mma = nullptr;
  t->d_enc_img = nullptr;
  t->n_prop = 0;
  if (!net) return CCW_OK;
  if (t->ndim != 2) return fail(CCW_EINVAL, "the learned proposal is 2D only");
  if (n_prop < 1 || n_prop > CCW_MAX_TOPK)
    return fail(CCW_EINVAL, "n_prop must be in [1, %d]", CCW_MAX_TOPK);
  if (!(gap_theta == gap_theta)) return fail(CCW_EINVAL, "gap_theta is NaN");
  if (t->sd > 255) return fail(CCW_EINVAL, "the proposal needs 2^(d J) <= 255");
  int C, tj;
  const float* params;
  int64_t count;
  net_view(net, &C, &tj, &params, &count);
  if (C != t->F || tj != t->Tj)
    return fail(CCW_EINVAL, "network shape (%d ch, %d) != TI (F %d, T/2^J %d)", C, tj, t->F, t->Tj);
  const size_t tab_bytes = sizeof(__nv_bfloat16) * 16 * 64 * (size_t)t->P;
  if ((e = cudaMalloc((void**)&t->d_net, sizeof(float) * count)) != cudaSuccess ||
      (e = cudaMalloc((void**)&t->d_tables, tab_bytes)) != cudaSuccess ||
      (!t->d_learn_stats &&
       (e = cudaMalloc((void**)&t->d_learn_stats, 3 * sizeof(unsigned long long))) !=
           cudaSuccess)) {
    cudaFree(t->d_net);
    cudaFree(t->d_tables);
    t->d_net = nullptr;
    t->d_tables = nullptr;
    return fail(CCW_ENOMEM, "proposal tables: %s", cudaGetErrorString(e));
  }
  if ((e = cudaMemcpyAsync(t->d_net, params, sizeof(float) * count, cudaMemcpyDeviceToDevice,
                           st)) != cudaSuccess ||
      (e = launch_round_weights(t->d_net, C, tj, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(t->d_tables, 0, tab_bytes, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(t->d_learn_stats, 0, 3 * sizeof(unsigned long long), st)) !=
          cudaSuccess)
    return cuda_fail(e, "attach proposal");
  ++g_launches;   // weight rounding
  const int64_t img_bytes = enc_tc_image_bytes(C, tj);
  if (img_bytes > 0) {
    if ((e = cudaMalloc(&t->d_enc_img, (size_t)img_bytes)) != cudaSuccess ||
        (e = enc_tc_build_image(t->d_net, C, tj, t->d_enc_img, st)) != cudaSuccess)
      return cuda_fail(e, "encoder weight image");
    ++g_launches;
  }
  WaveArgs a;
  fill_ti(t, 0, a);
  a.net = t->d_net;
  a.enc_img = t->d_enc_img;
  // scratch of the table passes, freed at the end
  const int chunk = (int)std::min<int64_t>(t->P, 16384);
  float *x = nullptr, *act = nullptr, *emb = nullptr;
  if ((e = cudaMalloc((void**)&x, sizeof(float) * (size_t)C * tj * tj * chunk)) != cudaSuccess ||
      (e = cudaMalloc((void**)&act, sizeof(float) * (size_t)infer_act_floats(C, tj) * chunk)) !=
          cudaSuccess ||
      (e = cudaMalloc((void**)&emb, sizeof(float) * 64 * (size_t)chunk)) != cudaSuccess) {
    cudaFree(x);
    cudaFree(act);
    return fail(CCW_ENOMEM, "proposal table scratch: %s", cudaGetErrorString(e));
  }
  for (int type = 1; type < 16 && e == cudaSuccess; ++type) {
    if (!usable_mask_type(type)) continue;
    e = launch_encode_tables(a, type, t->d_tables, x, act, emb, chunk, st);
    // per chunk: window inputs, the encoder (1 launch, or 5 layer by layer), BF16 copy
    const int enc = encode_items_launches(C, tj, t->d_enc_img != nullptr);
    g_launches += (2 + (enc == 1 ? 1 : enc - 1)) * ((t->P + chunk - 1) / chunk);
  }
  // the tensor-core selector's copy of small tables
  const int64_t mma_elems = tables_mma_elems(t->P);
  if (e == cudaSuccess && mma_elems > 0) {
    if ((e = cudaMalloc((void**)&t->d_tables_mma, sizeof(__nv_bfloat16) * mma_elems)) ==
        cudaSuccess)
      e = launch_tables_mma(t->d_tables, t->P, t->d_tables_mma, st);
    ++g_launches;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(x);
  cudaFree(act);
  cudaFree(emb);
  if (e != cudaSuccess) return cuda_fail(e, "proposal tables");
  t->n_prop = n_prop;
  t->gap_theta = gap_theta;
  return CCW_OK;
}

extern "C" int ccw_proposal_query(const ccw_ti* tc, const uint8_t* counts_dev, int32_t n,
                                  int32_t* prop_dev, float* gap_dev, int32_t* type_dev,
                                  void* stream) {
  if (!tc) return fail(CCW_EINVAL, "NULL TI");
  ccw_ti* t = const_cast<ccw_ti*>(tc);
  if (!t->d_tables) return fail(CCW_EINVAL, "no proposal attached");
  if (n < 0) return fail(CCW_EINVAL, "n must be >= 0");
  if (n == 0) return CCW_OK;
  if (!counts_dev || !prop_dev || !gap_dev) return fail(CCW_EINVAL, "NULL buffer");
  cudaStream_t st = (cudaStream_t)stream;
  const int chunk = std::min(n, 65535);
  EvDev ev = query_records(t, nullptr);
  void* rec = nullptr;
  void* emb = nullptr;
  void* x = nullptr;
  void* act = nullptr;
  cudaError_t e;
  if ((e = cudaMallocAsync(&rec, (size_t)ev.stride * chunk, st)) != cudaSuccess ||
      (e = cudaMallocAsync(&emb, sizeof(float) * 64 * (size_t)chunk, st)) != cudaSuccess ||
      (e = cudaMallocAsync(&x, sizeof(float) * (size_t)t->F * t->Tj * t->Tj * chunk, st)) !=
          cudaSuccess ||
      (e = cudaMallocAsync(&act, sizeof(float) * (size_t)infer_act_floats(t->F, t->Tj) * chunk,
                           st)) != cudaSuccess) {
    if (rec) cudaFreeAsync(rec, st);
    if (emb) cudaFreeAsync(emb, st);
    if (x) cudaFreeAsync(x, st);
    return fail(CCW_ENOMEM, "query workspace: %s", cudaGetErrorString(e));
  }
  ev.base = (unsigned char*)rec;
  const int64_t nc = (int64_t)t->F * t->Tj * t->Tj;
  int rc = CCW_OK;
  for (int i0 = 0; i0 < n && rc == CCW_OK; i0 += chunk) {
    WaveArgs a;
    fill_ti(t, 0, a);
    a.ev = ev;
    a.n_items = std::min(chunk, n - i0);
    a.net = t->d_net;
    a.tables = t->d_tables;
    a.tables_mma = t->d_tables_mma;
    a.enc_img = t->d_enc_img;
    a.n_prop = t->n_prop;
    a.emb = (float*)emb;
    a.prop = prop_dev + (int64_t)i0 * t->n_prop;
    a.prop_gap = gap_dev + i0;
    if ((e = launch_records_from_counts(a, counts_dev + i0 * nc, type_dev ? type_dev + i0 : nullptr,
                                        st)) != cudaSuccess ||
        (e = launch_encode_items(a, (float*)x, (float*)act, false, st)) != cudaSuccess ||
        (e = launch_nnsel(a, false, st)) != cudaSuccess)
      rc = cuda_fail(e, "proposal query kernels");
    g_launches += 2 + encode_items_launches(t->F, t->Tj, t->d_enc_img != nullptr);
  }
  cudaFreeAsync(act, st);
  cudaFreeAsync(x, st);
  cudaFreeAsync(emb, st);
  cudaFreeAsync(rec, st);
  return rc;
}

extern "C" int ccw_proposal_inputs(const ccw_ti* tc, int32_t what, const uint8_t* counts_dev,
                                   const int32_t* cand_dev, int32_t* type_dev, int32_t n,
                                   float* out_dev, void* stream) {
  if (!tc) return fail(CCW_EINVAL, "NULL TI");
  ccw_ti* t = const_cast<ccw_ti*>(tc);
  if (t->ndim != 2) return fail(CCW_EINVAL, "the learned proposal is 2D only");
  if (n < 0) return fail(CCW_EINVAL, "n must be >= 0");
  if (what == 0 && !counts_dev) return fail(CCW_EINVAL, "what 0 needs counts_dev");
  if (what == 1 && (!cand_dev || !type_dev)) return fail(CCW_EINVAL, "what 1 needs cand and type");
  if (what != 0 && what != 1) return fail(CCW_EINVAL, "bad what");
  if (n == 0) return CCW_OK;
  if (!out_dev) return fail(CCW_EINVAL, "NULL output");
  WaveArgs a;
  fill_ti(t, 0, a);
  cudaError_t e = launch_inputs(a, what, counts_dev, cand_dev, type_dev, n, out_dev,
                                (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "proposal input kernel");
  g_launches += (n + 65534) / 65535;
  return CCW_OK;
}

extern "C" int ccw_proposal_stats(const ccw_ti* tc, int64_t out[3], void* stream) {
  if (!tc || !out) return fail(CCW_EINVAL, "NULL argument");
  ccw_ti* t = const_cast<ccw_ti*>(tc);
  out[0] = out[1] = out[2] = 0;
  if (!t->d_learn_stats) return CCW_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long h[3];
  cudaError_t e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess ||
      (e = cudaMemcpy(h, t->d_learn_stats, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemset(t->d_learn_stats, 0, sizeof(h))) != cudaSuccess)
    return cuda_fail(e, "proposal stats");
  for (int i = 0; i < 3; ++i) out[i] = (int64_t)h[i];
  return CCW_OK;
}

extern "C" int ccw_simulate(const ccw_ti* tc, const ccw_params* p, const int32_t* hd_cells_dev,
                            const uint8_t* hd_vals_dev, int32_t n_hd, uint64_t seed,
                            uint8_t* out_dev, int32_t* patch_log_dev, void* stream) {
  if (!tc || !p || !out_dev) return fail(CCW_EINVAL, "NULL argument");
  if (p->n_real < 1) return fail(CCW_EINVAL, "n_real must be >= 1");
  if (p->real_base < 0) return fail(CCW_EINVAL, "real_base must be >= 0");
  ccw_group g;
  for (int a = 0; a < 3; ++a) g.grid[a] = p->grid[a];
  g.n_real = p->n_real;
  g.real_base = p->real_base;
  g.hd_cells_dev = hd_cells_dev;
  g.hd_vals_dev = hd_vals_dev;
  g.n_hd = n_hd;
  g.out_dev = out_dev;
  g.patch_log_dev = patch_log_dev;
  g.event_counts_dev = nullptr;
  g.out_host = nullptr;
  return simulate_groups(const_cast<ccw_ti*>(tc), p, &g, 1, seed, stream);
}

extern "C" int ccw_simulate_groups(const ccw_ti* tc, const ccw_params* p,
                                   const ccw_group* groups, int32_t n_groups, uint64_t seed,
                                   void* stream) {
  if (!tc || !p) return fail(CCW_EINVAL, "NULL argument");
  return simulate_groups(const_cast<ccw_ti*>(tc), p, groups, n_groups, seed, stream);
}
