/*
 * ccw.h -- C ABI of the GB300 (sm_103a) CCWSIM best-match search library.
 *
 * CCWSIM (Bavandsavadkoohi et al., arXiv 2404.00441) simulates a categorical
 * grid along a raster path of patches (Sec. 4.1). For every patch it takes
 * the Haar DWT approximation of the patch's overlap data event (Sec. 4.2),
 * cross-correlates it with every candidate position of the training image's
 * (TI) approximation (Eq. CCW, Sec. 4.3), keeps the K best candidates, draws
 * one (Algorithm 1, lines 11-12; Sec. 4.4), and pastes the Inverse-DWT of the
 * drawn candidate (Algorithm 1, lines 13-14).
 *
 * Conventions shared by every entry point:
 *  - Arrays are row-major with x fastest: a 2D grid of dims {nx, ny, 1} is
 *    indexed x + nx*y, a 3D grid x + nx*(y + ny*z). dims[2] is 1 in 2D.
 *  - Facies codes are uint8 in [0, n_facies); CCW_UNKNOWN (255) marks an
 *    uninformed cell (or "no hard datum").
 *  - Pointers named *_dev are device pointers on the current CUDA device;
 *    the caller allocates them and keeps ownership. `stream` is a
 *    cudaStream_t (NULL = legacy default stream). Every call is ordered on
 *    `stream`; calls that say so synchronize it once before returning.
 *  - Every call returns CCW_OK (0) or a negative CCW_E* code; the reason is
 *    kept per host thread and read with ccw_last_error(). No C++ exception
 *    crosses this boundary.
 *  - Candidates are the origins x (level-J coordinates) with x + T/2^J <=
 *    level-J TI size along every axis; candidate index = x fastest over the
 *    candidate grid. Ranking order: hard-data mismatches ascending, score
 *    descending, candidate index ascending.
 *  - Scores are the full CCW similarity of the chosen score mode: one-hot
 *    (default) sums Eq. CCW over the indicator image of every facies; the
 *    literal mode applies Eq. CCW to the facies codes.
 *  - Random draws use Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *    64-bit seed (low word first); the draw of patch p of realization r is
 *    the first output word u of counter (r, p, 0, 0) and picks rank
 *    floor(u * K' / 2^32), K' = min(K, P_c); an empty data event picks
 *    candidate floor(u * P_c / 2^32).
 */
#ifndef CCW_H
#define CCW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCW_OK 0
#define CCW_EINVAL (-1)      /* bad argument or input value */
#define CCW_ENOMEM (-2)      /* device allocation failed */
#define CCW_ECUDA (-3)       /* a CUDA call failed */
#define CCW_ETIMEOUT (-4)    /* a bounded device wait gave up */
#define CCW_EUNSUPPORTED (-5)/* valid request the library does not handle */

#define CCW_UNKNOWN 255
#define CCW_PRECISION_INEXACT 4 /* ccw_params.precision flag: FP16/BF16 past the
                                   format's exact integer range (see there) */
#define CCW_MAX_TOPK 64
#define CCW_LOG_FLAG_UNIFORM 1  /* patch log: empty data event, uniform pick */
#define CCW_LOG_FLAG_DONE 2     /* patch log: the patch was simulated */
#define CCW_LOG_FLAG_PROPOSAL 4 /* patch log: the learned proposal settled the
                                   patch (no full search) */

/* Opaque TI state, owned by the library (device buffers on the device that
 * was current at ccw_ti_prepare). */
typedef struct ccw_ti ccw_ti;

/* Simulation parameters (Algorithm 1 "Require" list: template and overlap
 * size live in the ccw_ti; K, number of realizations here). */
typedef struct {
  int32_t ndim;        /* 2 or 3; must equal the TI's */
  int32_t grid[3];     /* simulation grid dims {nx, ny, nz}; nz = 1 in 2D */
  int32_t topk;        /* K, 1..CCW_MAX_TOPK (Algorithm 1, line 11) */
  int32_t n_real;      /* realizations simulated by one call (>= 1) */
  int32_t real_base;   /* id of the first realization (Philox counter word 0) */
  int32_t path_random; /* 0: raster from the origin; 1: each realization
                          mirrors its path along the axes given by bits of the
                          first word of Philox counter (r, 0, 1, 0)
                          (Algorithm 1, line 3) */
  int32_t score_mode;  /* 0: one-hot facies indicators; 1: literal codes */
  int32_t precision;   /* CCF arithmetic: 0 FP32 FMA lanes; 1 FP16 and 2 BF16
                          tensor cores (3D: K <= 8), FP32 accumulation. Every
                          mode is exact: 1 and 2 are refused (CCW_EINVAL)
                          when an operand could exceed the format's exact
                          integer range (2048 for FP16, 256 for BF16; the
                          operands are at most 2^(d J) in the one-hot score,
                          (F - 1) 2^(d J) in the literal one), unless
                          CCW_PRECISION_INEXACT is or'ed in: the operands
                          are then rounded to the format (round to nearest
                          even) and scores, rankings and picks are
                          approximate: a score is off by at most 2^-7
                          (BF16) or 2^-10 (FP16) of the sum of the absolute
                          products of its taps, plus FP32 accumulation and
                          the rounding to an integer. */
  int32_t learned;     /* 0: full search for every patch; 1: learned proposal
                          first (an addition of this library, see
                          ccw_ti_attach_proposal): 2D, one-hot score only,
                          topk <= the attached n_prop */
  int32_t ccf_tile;    /* CCF tiling (no counterpart in the paper; results do
                          not depend on it): 0 = the library's choice; with
                          precision 0 the data events per CTA (1, 2, 4 or 8
                          in 2D; 1, 2 or 4 in 3D); with precision 1/2
                          nt | (mt << 16) | (e << 24) | (m << 25): data
                          events per N-tile nt in {16, 32, 64, 128},
                          128-candidate M-tiles per CTA mt in [1, 4],
                          mt * nt <= 512, epilogue e (0: per-thread K-lists
                          when K <= 8, 1: lanes on candidates), m = 1:
                          operands streamed through a ring of shared-memory
                          stages (always so in 3D; K <= 8), bit 26: three
                          stages instead of two, bit 29: four (not with bit
                          26), bits 27-28 = v: stages of Tj / 2^v template
                          rows (v <= 2). Bits 20-22 = L - 1 (any
                          precision, not with the learned proposal or bit
                          30): the realizations are split into L lanes
                          whose wavefront chains run concurrently on
                          separate streams of the call's graph (results
                          unchanged). Bit 30 alone among bits 24-31
                          (2D, K <= 8, no vt_ext, boundary_cut or learned):
                          every wavefront of the call in one cooperative
                          kernel, nt in {16, 32, 64, 128, 256} items per
                          N-tile, mt = 0 picks the M-tiles per CTA so that
                          every M-group has its own CTA. An autotuner
                          picks it by timing
                          (paper_2404_00441_gb300.autotune). */
  int32_t vt_ext;      /* non-causal conditioning (Sec. 4.4), 0..templ: the
                          template grown by vt_ext cells along the forward
                          direction of every axis of the path is a virtual
                          template; hard data in it but outside the template
                          add to each candidate's mismatch count, a datum
                          whose TI position falls outside the TI counting
                          as a mismatch. Scores and the empty-event rule use
                          the template alone. 0 = off. */
  int32_t boundary_cut; /* 0: the pattern overwrites its whole window; 1
                          (2D, templ <= 128): minimum-error boundary cut of
                          image quilting (Sec. 2): in the path frame, the
                          cheapest 8-connected column path through the left
                          overlap strip and row path through the top strip,
                          over the cells where the grid already holds a
                          value that differs from the pattern (ties to the
                          lower column, traced from the last row up); a
                          simulated cell takes the pattern only on the far
                          side of both cuts. Hard data are re-imposed. */
  int32_t all_shift;   /* 0: candidates are the decimated origins (multiples
                          of 2^J, Sec. 3.2); 1 (2D, precision 1 or 2 without
                          streamed operands, bit 30, learned proposal or
                          boundary cut): every fine origin c of the cropped TI
                          with c + T <= n is a candidate, its approximation the
                          2^(d J) block sums of its window; ranking index and
                          patch-log index = c's raster index over the fine
                          candidate grid, the pasted pattern = the TI crop at
                          c, an empty data event draws over the fine grid.
                          The library builds the TI's 2^(d J) phase planes on
                          first use. */
} ccw_params;

/* Shape information of a prepared TI. */
typedef struct {
  int32_t ndim, n_facies, level, scale; /* scale s = 2^level */
  int32_t templ, overlap;               /* T, OR in fine cells */
  int32_t dims[3];                      /* TI dims after cropping to multiples of s */
  int32_t coarse[3];                    /* level-J dims = dims / s */
  int32_t cand[3];                      /* candidate grid dims */
  int64_t n_cand;                       /* P_c = product of cand */
} ccw_ti_desc;

/*
 * ccw_ti_prepare -- Algorithm 1, line 2 (hoisted out of the realization
 * loop): DWT of the TI at level J (Sec. 3.1, Sec. 4.2, Haar).
 *  ti_dev    [dims[2]][dims[1]][dims[0]] uint8 facies codes, device.
 *  dims      host array of 3 ints; dims[2] = 1 when ndim = 2.
 *  n_facies  F in [2, 8]; every TI value must be < F.
 *  level     J in [0, 4] for 2D, [0, 2] for 3D.
 *  templ     T, overlap OR: fine cells, multiples of 2^J, T >= 2 OR, OR >= 0,
 *            T <= TI size after cropping along every axis.
 * The TI is cropped to multiples of s = 2^J (the candidate set is unchanged
 * by the crop). Builds the level-J facies counts of every s^d block, the
 * level-J code sums, and the full J-level Haar coefficient set of the codes
 * (kept per s^d block) used by the Inverse-DWT. Synchronizes `stream` once
 * to validate the TI values. *out receives the new handle; free it with
 * ccw_ti_free. Errors: CCW_EINVAL (bad argument, TI value >= F, score range
 * beyond the exact FP32 bound 2^24), CCW_ENOMEM, CCW_ECUDA.
 */
int ccw_ti_prepare(const uint8_t* ti_dev, int32_t ndim, const int32_t dims[3],
                   int32_t n_facies, int32_t level, int32_t templ, int32_t overlap,
                   void* stream, ccw_ti** out);

/* ccw_ti_describe -- fills *out with the shape of a prepared TI. */
int ccw_ti_describe(const ccw_ti* ti, ccw_ti_desc* out);

/* ccw_ti_free -- releases the handle and its device buffers (synchronizes the
 * device first). NULL is accepted. */
void ccw_ti_free(ccw_ti* ti);

/*
 * ccw_ti_export -- copies one of the prepared TI arrays to dst_dev (device,
 * caller-sized), for inspection and tests:
 *   what = 0: level-J facies counts, float32 [F-1][coarse], facies 0..F-2
 *             (counts of every s^d block; the scaled-Haar approximation).
 *   what = 1: level-J code sums, float32 [coarse].
 *   what = 2: Haar coefficients of the codes, int16 [coarse][s^d]: for each
 *             level-J block, the J-level scaled Haar transform of the block
 *             computed in place (level j pairs samples 2^(j-1) apart along x,
 *             then y, then z; the low-pass sum stays at the lower position,
 *             the difference goes to the upper one), so entry 0 is the
 *             block's approximation.
 *   what = 3: the cropped TI, uint8 [dims].
 *   what = 4: the attached learned proposal's window tables, bfloat16
 *             [16 mask types][P_c][64] (ccw_ti_attach_proposal; rows of
 *             unused mask types are zero); CCW_EINVAL when none is attached.
 */
int ccw_ti_export(const ccw_ti* ti, int32_t what, void* dst_dev, void* stream);

/*
 * ccw_simulate -- Algorithm 1 for params->n_real realizations of one grid
 * size, with hard-data conditioning (Sec. 4.4).
 *  hd_cells_dev  int32 [n_hd][ndim] cell coordinates (x, y[, z]), device;
 *                NULL when n_hd = 0. Every cell must lie inside the grid.
 *  hd_vals_dev   uint8 [n_hd] facies codes (< F). Two hard data on one cell
 *                keep the smaller code.
 *  out_dev       uint8 [n_real][grid] realizations (caller-allocated).
 *  patch_log_dev int32 [n_real][n_patches][4 + topk] or NULL: per patch, in
 *                path order, {pick, score of pick, mismatches of pick, flags,
 *                ranked candidates (unused slots -1)}; n_patches = product
 *                over axes of 1 + ceil(max(grid - T, 0) / (T - OR)).
 * The grid is padded to the patch lattice (T + (n - 1)(T - OR) per axis) and
 * cropped at the end. Patches are processed in wavefronts w = i_x + 2 i_y +
 * 4 i_z of the lattice index, which gives exactly the raster-order result
 * because T >= 2 OR. Synchronizes `stream` once at the end to read the
 * device status. Errors: CCW_EINVAL (parameters, hard data out of range or
 * >= F, more than 1024 hard data in one template), CCW_ENOMEM, CCW_ECUDA.
 */
int ccw_simulate(const ccw_ti* ti, const ccw_params* params, const int32_t* hd_cells_dev,
                 const uint8_t* hd_vals_dev, int32_t n_hd, uint64_t seed, uint8_t* out_dev,
                 int32_t* patch_log_dev, void* stream);

/* One grid size of a batch simulated by ccw_simulate_groups. */
typedef struct {
  int32_t grid[3];              /* grid dims {nx, ny, nz}; nz = 1 in 2D */
  int32_t n_real;               /* realizations of this size (>= 1) */
  int32_t real_base;            /* id of the first one (Philox counter word 0);
                                   give groups disjoint id ranges */
  const int32_t* hd_cells_dev;  /* int32 [n_hd][ndim] hard-data cells, or NULL */
  const uint8_t* hd_vals_dev;   /* uint8 [n_hd] hard-data codes, or NULL */
  int32_t n_hd;
  uint8_t* out_dev;             /* uint8 [n_real][grid] realizations */
  int32_t* patch_log_dev;       /* int32 [n_real][n_patches][4 + topk], or NULL */
  uint8_t* event_counts_dev;    /* uint8 [n_real][n_patches][F][(T/2^J)^d] or NULL:
                                   the facies counts of every level-J block of each
                                   patch's data event, as searched (needs 2^(d J) <=
                                   255); the learned proposal trains on them */
  uint8_t* out_host;            /* uint8 [n_real][grid] host copy of out_dev, or
                                   NULL; see ccw_simulate_groups */
} ccw_group;

/*
 * ccw_simulate_groups -- ccw_simulate for realizations of several grid
 * sizes at once (each group with its own hard data, outputs and patch log).
 * params->grid, n_real and real_base are ignored; the other fields apply to
 * every group. The patches of every group advance together, one wavefront
 * per step, so the groups share the kernel launches; each realization is
 * exactly what ccw_simulate gives for it. Synchronizes `stream` once at the
 * end. Errors as ccw_simulate.
 * Host read-back: a group with out_host also gets its realizations copied
 * into that host buffer (caller-owned, not retained) before the call
 * returns. When every out_host of the call is page-locked (cudaHostAlloc or
 * cudaHostRegister over the whole buffer) and path_random is 0, the copy
 * streams: each band of rows along the slowest axis is copied as soon as
 * the last patch row over it is pasted, while later wavefronts run, so
 * that only the last band's copy follows the simulation. The graph that
 * does this holds the out_dev and out_host pointers it was built with and
 * is built again when they change, so reuse the same buffers across calls.
 * Otherwise (pageable memory, mirrored paths) the copy runs after the
 * simulation.
 */
int ccw_simulate_groups(const ccw_ti* ti, const ccw_params* params, const ccw_group* groups,
                        int32_t n_groups, uint64_t seed, void* stream);

/*
 * ccw_ccf_search -- one batched best-match search step (Algorithm 1, lines
 * 9-12; Eq. CCW; Sec. 4.4), for B independent data events.
 *  de_dev     uint8 [B][T^d]: data events (the template window, codes or
 *             255 where unknown; hard data must already be written in).
 *  hd_dev     uint8 [B][T^d]: hard data of each window (255 = none), or NULL.
 *  k          K in [1, CCW_MAX_TOPK].
 *  score_mode bits 0-3: 0 one-hot, 1 literal score; bits 4-7: precision
 *             (as ccw_params.precision, CCW_PRECISION_INEXACT included).
 *  ctr_dev    uint32 [B][2]: (realization r, patch p) Philox counter words.
 *  topk_*_dev int32 [B][k]: ranked candidates with their score and mismatch
 *             count; slots past min(k, P_c), and all slots of an empty data
 *             event, hold -1 / 0 / 0.
 *  pick_dev   int32 [B]: the drawn candidate.
 * Asynchronous. Input values outside [0, F) other than 255 are reported by
 * ccw_ti_status. Errors: CCW_EINVAL, CCW_ENOMEM, CCW_ECUDA.
 */
int ccw_ccf_search(const ccw_ti* ti, int32_t B, const uint8_t* de_dev, const uint8_t* hd_dev,
                   int32_t k, int32_t score_mode, uint64_t seed, const uint32_t* ctr_dev,
                   int32_t* topk_idx_dev, int32_t* topk_score_dev, int32_t* topk_mis_dev,
                   int32_t* pick_dev, void* stream);

/*
 * ccw_ccf_search_noalloc -- the same search as ccw_ccf_search (same
 * arguments, same results), for callers that cannot allocate device memory
 * while they run: a serving process that has handed all of HBM to its own
 * pool up front, or a latency-critical loop that must not pay for a driver
 * allocation or the synchronization cudaMalloc may imply. ccw_ccf_search
 * takes its scratch (per-event records, per-tile ranking keys) from the
 * stream-ordered allocator on every call; this variant uses instead one
 * scratch array compiled into the library, CCW_NOALLOC_SCRATCH_BYTES bytes
 * on every device that loads the library, kept until the process exits. It
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *  - Size limit: a call needs, per data event (of min(B, 65535)), one
 *    event record (the event's level-J weights, its hard-data list and
 *    bookkeeping: a few KB, set by the template) and 8 * tiles * k bytes of
 *    ranking keys, where tiles is the number of
 *    candidate tiles of the TI (64x16 candidates per tile in 2D, 32x8x4 in
 *    3D). A call that needs more than CCW_NOALLOC_SCRATCH_BYTES returns
 *    CCW_EINVAL without running; split the batch.
 *  - Set-up: the first call on a device looks up the device address of the
 *    array (cudaGetSymbolAddress) with that device current; make that first
 *    call before any stream capture that would contain it.
 *  - Sharing: every call on a device uses the same array and leaves its
 *    contents behind; nothing in it needs to start at zero, since a call
 *    writes every scratch slot before it reads it. Calls whose work
 *    overlaps on the GPU (different streams, or host threads, without
 *    ordering between them) race on the array and give wrong results:
 *    order them on one stream.
 * The paper has no counterpart of this entry point; it only changes where
 * the scratch memory comes from. Its launches are never timed or counted by
 * the profiler (ccw_profile_enable), whose events and counters would need
 * allocations. Asynchronous. Errors: CCW_EINVAL (as
 * ccw_ccf_search, or the batch needs more scratch than the array holds),
 * CCW_ECUDA.
 */
#define CCW_NOALLOC_SCRATCH_BYTES (4 * 1024 * 1024)
int ccw_ccf_search_noalloc(const ccw_ti* ti, int32_t B, const uint8_t* de_dev,
                           const uint8_t* hd_dev, int32_t k, int32_t score_mode, uint64_t seed,
                           const uint32_t* ctr_dev, int32_t* topk_idx_dev,
                           int32_t* topk_score_dev, int32_t* topk_mis_dev, int32_t* pick_dev,
                           void* stream);

/*
 * ccw_ccf_map -- the full CCW score map and hard-data mismatch map of B data
 * events (Eq. CCW over every candidate), same inputs as ccw_ccf_search
 * (score_mode carries the precision in bits 4-7 here too).
 *  score_dev, mis_dev  int32 [B][P_c] (mis_dev may be NULL).
 * An empty data event yields an all-zero map. Asynchronous.
 */
int ccw_ccf_map(const ccw_ti* ti, int32_t B, const uint8_t* de_dev, const uint8_t* hd_dev,
                int32_t score_mode, int32_t* score_dev, int32_t* mis_dev, void* stream);

/*
 * ccw_idwt_paste -- Algorithm 1, lines 13-14: Inverse-DWT of candidate
 * pick_dev[b] from the TI's approximation and detail coefficients, pasted
 * with its first cell at dst_origin_dev[b] (int32 [B][3], x y z, may be
 * negative) into sg_dev (uint8, dims sg_dims, host array of 3). Cells that
 * fall outside the grid are skipped. Overlapping destinations within one
 * call give an unspecified winner. Asynchronous.
 */
int ccw_idwt_paste(const ccw_ti* ti, int32_t B, const int32_t* pick_dev,
                   const int32_t* dst_origin_dev, uint8_t* sg_dev, const int32_t sg_dims[3],
                   void* stream);

/*
 * ccw_ti_status -- synchronizes `stream`, returns and clears the device
 * status word of the handle: 0, or a bitwise OR of 1 (an input code >= F),
 * 2 (more than 1024 hard data in one template), 4 (a bounded wait gave up).
 */
int ccw_ti_status(const ccw_ti* ti, void* stream, int32_t* status_out);

/* ------------------------------------------------------------------------
 * Learned proposal (not in the paper; an addition of this library). A small
 * encoder maps a level-J data event, or a TI window under the same mask, to
 * a unit 64-vector; nearest neighbours of a data event's vector among the TI
 * windows' vectors are proposals that the exact CCF of Eq. CCW re-ranks.
 * Network on inputs C x tj x tj (facies counts of the level-J blocks
 * divided by 2^(d J)): conv 3x3 C->32 (pad 1) + ReLU, conv 3x3 32->32
 * stride 2 + ReLU, conv 3x3 32->32 stride 2 + ReLU, linear -> 64, L2
 * normalisation. Parameters are FP32 masters (layout: conv weights
 * [out][in][3][3] then biases, layer by layer, then the linear weight
 * [64][in] and bias). With bf16 = 1 the passes use BF16-rounded weights and
 * activations.
 * ------------------------------------------------------------------------ */
typedef struct ccw_net ccw_net;

/* ccw_set_nn_path -- which kernel scores and selects the nearest TI windows
 * of the learned proposal (the proposals are the same up to FP32 rounding of
 * the scores): 0 (default) the tcgen05 kernel for tables of at most 3072
 * windows (8 data events per CTA, 12 when a launch has more than 8 per SM
 * and 12 fit in shared memory), else the FP32-lane kernel with several data
 * events per CTA (at most 6144 windows), else one CTA per data event; 1
 * never the tensor cores; 2 always one CTA per data event; 3 as 0 with 12
 * events per CTA whenever they fit. Process-wide; CCW_EINVAL for other
 * values. */
int ccw_set_nn_path(int32_t path);

/* ccw_net_create -- new encoder for in_ch channels of tj x tj, He-normal
 * weights from `seed` (deterministic), zero biases. */
int ccw_net_create(int32_t in_ch, int32_t tj, uint64_t seed, ccw_net** out);
void ccw_net_free(ccw_net* net);
int64_t ccw_net_param_count(const ccw_net* net);
/* what = 0 copies the parameters, 1 the gradients of the last train step,
 * to host memory of ccw_net_param_count floats. */
int ccw_net_get(const ccw_net* net, int32_t what, float* host);
int ccw_net_set(ccw_net* net, const float* host);
/* ccw_net_embed -- unit embeddings float [n][64] of inputs float [n][C][tj][tj]
 * (device pointers). bf16 = 0: the training forward pass in FP32; 1: the
 * same with BF16 weights and activations; 2: the inference pass that the
 * learned proposal runs (tcgen05 tensor cores where the shape fits: C <= 8
 * and the layer planes in shared memory; inputs taken as BF16, which the
 * proposal's block-count inputs are exactly); 3: the fused FP32-lane
 * inference kernel (BF16 weights and activations, as 1). */
int ccw_net_embed(ccw_net* net, const float* x_dev, int32_t n, int32_t bf16, float* emb_dev,
                  void* stream);
/* ccw_net_train_step -- one InfoNCE step: anchors [B][C][tj][tj], candidates
 * [M][C][tj][tj] (M >= B; candidate i is the positive of anchor i, all others
 * negatives), logits a . c / tau, mean loss written to loss_dev (float, may
 * be NULL). Gradients are recomputed; with apply = 1 an AdamW step
 * (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay wd) follows. */
int ccw_net_train_step(ccw_net* net, const float* anchors_dev, int32_t B,
                       const float* cands_dev, int32_t M, float tau, float lr, float wd,
                       int32_t bf16, int32_t apply, float* loss_dev, void* stream);
const char* ccw_net_last_error(void);

/*
 * Inference of the learned proposal inside ccw_simulate (params.learned = 1).
 * Per patch: the data event's block counts are embedded; its overlap mask
 * type m (which of the four level-J overlap strips of width OR / 2^J are
 * fully known: bit 0 low x, 1 high x, 2 low y, 3 high y) selects the table of
 * TI-window embeddings under mask m; the n_prop windows with the largest dot
 * product are proposals; their exact Eq. CCW score and hard-data mismatch
 * (Sec. 4.4) rank them as the full search would, K best kept. When the
 * relative embedding gap (e_1 - e_nprop) / max(|e_1|, 1e-6) is at least
 * gap_theta the patch takes its pick from those K (log flag
 * CCW_LOG_FLAG_PROPOSAL); otherwise, and for patches without a full strip,
 * with both strips of an axis, or empty, the full search runs.
 *
 * ccw_ti_attach_proposal -- embeds every candidate window of `ti` under each
 * mask type with `net` (BF16 passes) and keeps the tables and a copy of the
 * parameters in the handle (16 x P_c x 64 BF16). The network must have
 * in_ch = F and tj = T / 2^J; 2D TIs only; 1 <= n_prop <= CCW_MAX_TOPK.
 * net = NULL detaches. Synchronizes `stream`. Later changes of `net` do not
 * affect the handle. Errors: CCW_EINVAL, CCW_ENOMEM, CCW_ECUDA.
 */
int ccw_ti_attach_proposal(ccw_ti* ti, const ccw_net* net, int32_t n_prop, float gap_theta,
                           void* stream);

/*
 * ccw_proposal_query -- the proposal step alone for n data events given by
 * their block counts counts_dev uint8 [n][F][tj^2] (as ccw_group's
 * event_counts_dev records them). Writes prop_dev int32 [n][n_prop]
 * (proposals by embedding score, best first), gap_dev float [n] (relative
 * gap, -1 when the event has no usable mask type) and type_dev int32 [n]
 * (mask type), device buffers owned by the caller. Needs an attached
 * proposal. Asynchronous on `stream`.
 */
int ccw_proposal_query(const ccw_ti* ti, const uint8_t* counts_dev, int32_t n, int32_t* prop_dev,
                       float* gap_dev, int32_t* type_dev, void* stream);

/*
 * ccw_proposal_inputs -- encoder inputs float [n][F][tj][tj] for training.
 *  what = 0: from data-event block counts counts_dev uint8 [n][F][tj^2]
 *            (counts / 2^(d J)); type_dev int32 [n] receives the mask types.
 *  what = 1: TI window of candidate cand_dev[i] under mask type type_dev[i]
 *            (facies counts of the blocks inside the mask, / 2^(d J); zero
 *            outside), the form the attached tables are built from.
 * 2D TIs only. Asynchronous on `stream`.
 */
int ccw_proposal_inputs(const ccw_ti* ti, int32_t what, const uint8_t* counts_dev,
                        const int32_t* cand_dev, int32_t* type_dev, int32_t n, float* out_dev,
                        void* stream);

/*
 * ccw_proposal_stats -- counters of the learned simulations on `ti` since
 * the last read (synchronizes `stream`, then resets them): out[0] patches
 * with a non-empty data event, out[1] patches that had proposals (a usable
 * mask type), out[2] patches settled by the proposal.
 */
int ccw_proposal_stats(const ccw_ti* ti, int64_t out[3], void* stream);

/*
 * Pattern-reproduction statistics of realizations (the validation of
 * Sec. 5.2-5.3; no counterpart as a library call in the paper). real_dev:
 * uint8 [n_real][dims[2]][dims[1]][dims[0]] facies codes, n_real <= 65535.
 * Every result is an exact integer count written to caller-owned device
 * memory; calls are asynchronous on `stream`. Errors: CCW_EINVAL, CCW_ECUDA
 * (text from ccw_eval_last_error).
 *
 * ccw_eval_proportions -- counts_dev uint64 [n_real][n_facies]: cells of
 *   each facies.
 * ccw_eval_variogram -- mismatch_dev uint64 [n_real][n_lags]: number of
 *   cell pairs (x, x + h e_axis) inside the grid whose indicators of `facies`
 *   differ, h = lags_dev[l] (int32, device); the indicator variogram is
 *   0.5 * mismatches / pairs, pairs = (n_axis - h) * (cells / n_axis).
 * ccw_eval_patterns -- hist_dev uint32 [n_facies^(w*w)] (<= 2^26 bins):
 *   histogram over all realizations of the w x w patterns (2D), each coded
 *   base n_facies row by row, after a mode downsampling by `down` (the most
 *   frequent facies of every down x down block, ties to the lower code;
 *   scratch_dev uint8 [n_real][dims[1]/down][dims[0]/down] when down > 1).
 */
int ccw_eval_proportions(const uint8_t* real_dev, int32_t n_real, const int32_t dims[3],
                         int32_t n_facies, uint64_t* counts_dev, void* stream);
int ccw_eval_variogram(const uint8_t* real_dev, int32_t n_real, const int32_t dims[3],
                       int32_t facies, int32_t axis, const int32_t* lags_dev, int32_t n_lags,
                       uint64_t* mismatch_dev, void* stream);
int ccw_eval_patterns(const uint8_t* real_dev, int32_t n_real, const int32_t dims[3],
                      int32_t n_facies, int32_t down, int32_t w, uint8_t* scratch_dev,
                      uint32_t* hist_dev, void* stream);
/*
 * ccw_eval_connectivity -- the probability of connection of Sec. 5.3 as two
 *   exact counts per lag: pairs_dev uint64 [n_real][n_lags][2] = {cell pairs
 *   (c, c + h e_axis) with both cells of `facies`, those of them in one
 *   4-connected component of `facies`}, h = lags_dev[l] (int32, device,
 *   >= 1); axis 0 = x (E-W), 1 = y (N-S); 2D only (dims[2] = 1, at most
 *   2^31 - 1 cells). The probability is the second count over the first.
 *   labels_dev: int32 scratch of n_real * (dims[0] * dims[1] + 1) entries
 *   (component labels, then one flag per realization). The components come
 *   from a union-find labelling with capped loops; a realization whose
 *   labelling hit the cap (never expected) reports 2^64 - 1 counts.
 */
int ccw_eval_connectivity(const uint8_t* real_dev, int32_t n_real, const int32_t dims[3],
                          int32_t facies, int32_t axis, const int32_t* lags_dev, int32_t n_lags,
                          int32_t* labels_dev, uint64_t* pairs_dev, void* stream);
const char* ccw_eval_last_error(void);

/* ccw_last_error -- text of the last failure on the calling host thread. */
const char* ccw_last_error(void);

/*
 * The random-number generator of every draw above (Algorithm 1: the random
 * pattern of an empty data event, line 6; the draw among the K best, line
 * 12; the path mirroring, line 3): Philox4x32-10 (Salmon et al., SC'11),
 * compiled from the same source as the kernels' own. With it a caller can
 * reproduce a draw: the draw of patch p of realization r under `seed` is
 * word 0 of counter (r, p, 0, 0) with key (seed low word, seed high word).
 *  ctr  uint32 [n][4] counters; out uint32 [n][4] output blocks; key [2].
 * ccw_philox_host -- host arrays, computed on the calling thread.
 * ccw_philox_dev  -- device arrays (16-byte aligned), asynchronous on
 *                    `stream`; key is a host array.
 * Errors: CCW_EINVAL (n < 0, NULL or misaligned arrays), CCW_ECUDA.
 */
int ccw_philox_host(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out);
int ccw_philox_dev(int64_t n, const uint32_t* ctr_dev, const uint32_t key[2], uint32_t* out_dev,
                   void* stream);

/*
 * Profiling. When enabled, every launch of the search kernel is bracketed by
 * CUDA events on its stream; ccw_profile_read returns the number of timed
 * launches, their summed duration (ms, read after the stream synchronizes)
 * and the algorithmic work they did: candidate evaluations and multiply-adds
 * over the taps of the data events (masked level-J cells times channels).
 * ccw_launch_count returns the number of kernels this library has launched
 * in the process.
 */
int ccw_profile_enable(int32_t enable);
/* ccw_set_barrier_polls -- how many times a CTA of the one-kernel simulation
 * (ccw_params.ccf_tile bit 30) polls a grid-wide barrier before it gives up;
 * the call then returns CCW_ETIMEOUT and leaves the device usable. 0 restores
 * the default (2^22 polls, seconds). Small values exist to test that error
 * path; they make calls fail. Applies to calls made after it. */
int ccw_set_barrier_polls(int64_t polls);
int ccw_profile_read(int64_t* launches, double* total_ms, double* cand_evals, double* macs);
/* ccw_profile_read_phases -- summed durations (ms, stream-ordered CUDA events
 * recorded inside the captured simulation graph) of the three phases of
 * every wavefront of the profiled simulations: ms[0] data events (and the
 * learned proposal's kernels), ms[1] CCF, ms[2] finish (top-K merge, pick,
 * inverse-DWT paste); read and reset. */
int ccw_profile_read_phases(double ms[3]);
/* ccw_profile_read_proposal -- the learned proposal's share of the profiled
 * simulations (stream-ordered events in the captured graph): ms[0] the
 * encoder (inputs and embedding of the data events), ms[1] the nearest-window
 * selection and the exact re-rank; read and reset. */
int ccw_profile_read_proposal(double ms[2]);
int64_t ccw_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* CCW_H */
