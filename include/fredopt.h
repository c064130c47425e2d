/*
 * fredopt.h - C ABI of the GB300 (sm_103a) implementation of simultaneous
 * dose and LETd proton plan optimisation by superiorized feasibility seeking
 * (arXiv 2509.20012: Sec. 2.4.3, Fig. 2, Fig. 3, Eq. 2).
 *
 * One handle holds one plan: the dose-influence matrix D (Gy per unit spot
 * weight) and the LET-weighted matrix L (Gy*keV/um; L_ij = LET_ij * D_ij,
 * the additive numerator of Eq. 1 per pencil beam, Sec. 2.2) with one shared
 * CSR sparsity pattern, the voxel -> structure bitmask, the constraint table
 * and the objective.  Everything after fredopt_load_influence is resident on
 * the device; an iteration makes no host round trip.
 *
 * Conventions for every call:
 *   - Return 0 (FREDOPT_OK) or a negative FREDOPT_ERR_* code; nothing throws
 *     across the ABI.  The handle stays usable after an error.
 *     fredopt_last_error() gives a message for the last failing call on the
 *     handle.
 *   - Pointer arguments are caller-owned.  Unless FREDOPT_DEVICE_PTR is set
 *     in `flags`, they are host pointers (pageable or pinned); with it, they
 *     are device pointers on the handle's device.  Inputs are consumed before
 *     the call returns; outputs are complete when it returns (the library
 *     synchronises its stream at the end of every call that returns data).
 *   - Voxel arrays are indexed by voxel (row of D and L), spot arrays by spot
 *     (column).  Floating point values are IEEE binary32 unless noted.
 *   - A handle is not thread-safe; distinct handles may be used from
 *     distinct threads.
 */
#ifndef FREDOPT_H
#define FREDOPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FREDOPT_OK 0
#define FREDOPT_ERR_INVALID_ARG (-1) /* bad scalar argument or null pointer */
#define FREDOPT_ERR_SHAPE (-2)       /* sizes inconsistent or out of range */
#define FREDOPT_ERR_PATTERN (-3)     /* CSR not monotone, column out of range or unsorted; in a
                                        library built with FO_CHECKED=1 also: a streaming kernel
                                        found a tile range or index out of bounds */
#define FREDOPT_ERR_NONFINITE (-4)   /* NaN or Inf in an input */
#define FREDOPT_ERR_NOT_LOADED (-5)  /* call needs a loaded plan / constraints / begun solve */
#define FREDOPT_ERR_OOM (-6)         /* device allocation failed */
#define FREDOPT_ERR_CUDA (-7)        /* CUDA runtime error (message via fredopt_last_error) */
#define FREDOPT_ERR_TIMEOUT (-8)     /* a bounded device-side wait gave up */
#define FREDOPT_ERR_UNSUPPORTED (-9) /* option not available */

/* ---- flags ---- */
#define FREDOPT_DEVICE_PTR 0x1u /* pointer args are device pointers */

/* value storage formats of fredopt_load_influence (low byte of `format`) */
#define FREDOPT_FP32 0 /* D, L stored as float */
#define FREDOPT_BF16 1 /* bfloat16 with one float scale per row and matrix */
#define FREDOPT_FP16 2 /* binary16 with one float scale per row and matrix */
/* row set of the iteration (or'ed into `format`) */
#define FREDOPT_ROWS_ALL 0x000 /* every voxel row is streamed every pass (default) */
#define FREDOPT_ROWS_ROI 0x100 /* only rows of voxels in some structure are streamed;
                                  dose/LETd of the other voxels are computed at the end */
/* index widths of the streams (or'ed into `format`).  By default the
 * forward stream keeps its column indices as 16-bit values when n_spots <=
 * 65536 and the fluence fits the forward kernel's shared memory (about 58000
 * spots on GB300), and the transposed product streams its row indices as
 * 16-bit offsets from a base row per block of 128 nonzeros (blocks whose rows
 * span 65536 or more keep 32-bit rows in a side table).  Each saves 2 bytes
 * per nonzero and pass with identical results.  FREDOPT_INDEX32 keeps both
 * streams 32-bit. */
#define FREDOPT_INDEX32 0x200
/* launch shapes (or'ed into `format`).  By default every kernel of the plan
 * is sized for the whole GPU.  FREDOPT_SHARED sizes them for running beside
 * other plans (a batch graph, a server with several plans in flight): about
 * one SM's worth of CTAs per 400000 nonzeros of the streamed rows (the whole
 * GPU from 6.08e7 nonzeros on GB300), so that small plans leave SMs to the
 * others.  Results depend only on the plan and its launch shapes: a plan
 * loaded with and without the flag agrees to rounding, and bit for bit with
 * itself alone and in a batch. */
#define FREDOPT_SHARED 0x400

/* ---- constraint kinds (Fig. 2 half-spaces; the LETd limit LETd <= Lambda as the half-space (L - Lambda D) w <= 0) ----
 * DOSE_MAX / DOSE_MIN : (D w)_i <= / >= bound                        (Gy)
 * CDL_MAX  / CDL_MIN  : c (L w)_i <= / >= bound, c = params.c_cdl    (Gy)
 * LETD_MAX / LETD_MIN : ((L - bound D) w)_i <= / >= 0, i.e. LETd_i <= / >= bound (keV/um)
 */
#define FREDOPT_DOSE_MIN 0
#define FREDOPT_DOSE_MAX 1
#define FREDOPT_CDL_MIN 2
#define FREDOPT_CDL_MAX 3
#define FREDOPT_LETD_MIN 4
#define FREDOPT_LETD_MAX 5

typedef struct fredopt_constraint {
  uint32_t struct_bit; /* 0..31: the structure whose voxels carry this constraint */
  int32_t kind;        /* FREDOPT_DOSE_MIN .. FREDOPT_LETD_MAX */
  double bound;        /* Gy (dose, cDL) or keV/um (LETd) */
  double priority;     /* structure weight p_S > 0 (Fig. 2 "w_i"; Sec. 2.4.3) */
} fredopt_constraint;

/* objective quantities of Eq. 2: q_i = (D w)_i or c (L w)_i; the volume
 * statistics also take LETd_i = (L w)_i / (D w)_i (Eq. 1, 0 where (D w)_i = 0) */
#define FREDOPT_Q_DOSE 0
#define FREDOPT_Q_CDL 1
#define FREDOPT_Q_LETD 2

typedef struct fredopt_objective_term {
  uint32_t struct_bit; /* structure whose voxels enter this term */
  int32_t quantity;    /* FREDOPT_Q_DOSE or FREDOPT_Q_CDL */
  double target;       /* D-hat_i or cDL-hat_i of Eq. 2 */
  double weight;       /* w_i of Eq. 2 (> 0) */
} fredopt_objective_term;

/* Cimmino weight normalisation */
#define FREDOPT_NORM_ALL 0      /* omega_r = p_r / sum of p over all reachable rows */
#define FREDOPT_NORM_VIOLATED 1 /* omega_r = p_r / sum of p over rows violated now */

typedef struct fredopt_params {
  double beta0;           /* first trial step; < 0 selects 0.1 * ||w0||_2 (default -1) */
  double eta;             /* priority decay per iteration, 0 < eta <= 1 (default 1) */
  int32_t reductions;     /* perturbation steps per iteration, N >= 0 (default 1; 0 = plain
                             feasibility seeking, Fig. 2 alone) */
  int32_t max_trials;     /* cap of the trial loop per step, >= 1 (default 50) */
  int32_t cimmino_norm;   /* FREDOPT_NORM_* (default FREDOPT_NORM_ALL) */
  int32_t grad_normalize; /* 1: unit direction -g/||g|| (default); 0: raw -g (Fig. 3 literal) */
  double c_cdl;           /* c of cDL = c * dose * LETd, um/keV (default 0.04, Sec. 2.4) */
  int32_t log_capacity;   /* per-iteration log entries kept on the device (default 4096) */
  int32_t use_graphs;     /* 1: replay iterations as CUDA graphs (default); 0: plain launches */
  int32_t sweep_blocks;   /* 0 (default): simultaneous feasibility step (Cimmino).  M in
                             1..FREDOPT_MAX_SWEEP_BLOCKS: block-iterative sweep of Fig. 2 over M
                             voxel blocks (see fredopt_sweep_step) */
  int32_t tile_balance;   /* 1 (default): in passes of at least 16384 nonzeros per warp, the
                             forward and transposed products' warps claim tiles of decreasing
                             size from a counter, so SMs that stream faster take more of them
                             (the SMs of a GB300 differ by up to ~13% in streaming rate);
                             2: claim tiles in every pass; 0: one static tile per warp.
                             Results do not change. */
} fredopt_params;

#define FREDOPT_MAX_SWEEP_BLOCKS 1024

typedef struct fredopt_log_entry {
  int64_t k;           /* iteration index */
  int64_t s;           /* global trial counter after this iteration's perturbation phase */
  int32_t accepted;    /* accepted perturbation steps this iteration */
  int32_t n_violated;  /* constraint rows violated at the point the feasibility step saw */
  double beta;         /* last accepted step (0 if none) */
  double f_start;      /* objective at w^k */
  double f_end;        /* objective at the perturbed point (closed form on the device) */
  double gnorm;        /* ||grad f|| of the last perturbation step */
  double max_violation;/* largest violation (bound units) at that point */
} fredopt_log_entry;

typedef struct fredopt_report {
  int64_t iters;               /* iterations run since fredopt_begin */
  int64_t s;                   /* trial counter */
  int64_t accepted;            /* accepted perturbation steps in total */
  int64_t n_rows;              /* reachable constraint rows */
  int64_t unreachable_rows;    /* rows skipped because |a_r|^2 == 0 */
  int64_t n_violated;          /* rows violated at the final w (FP64 check) */
  double objective;            /* f(w) at the final w, FP64 */
  double max_violation[6];     /* per kind (index = FREDOPT_* kind), FP64, bound units */
  double beta0;                /* step actually used */
  double device_ms;            /* device time of fredopt_iterate calls since fredopt_begin */
} fredopt_report;

typedef struct fredopt_ctx* fredopt_t;

/* Fill `p` with the defaults listed above. */
void fredopt_default_params(fredopt_params* p);

/* Human-readable name of a status code (static storage). */
const char* fredopt_strerror(int code);

/* Message of the last failing call on `h` (valid until the next call on h). */
const char* fredopt_last_error(fredopt_t h);

/* Create a handle on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * on that device that all work of the handle is ordered on, or NULL for a
 * stream owned by the handle.  The caller keeps ownership of its stream. */
int fredopt_create(fredopt_t* out, int device, void* cuda_stream);

/* Free every device resource of the handle. */
int fredopt_destroy(fredopt_t h);

/* Load the influence-matrix pair (Sec. 2.2; the stage-(iii) upload of
 * Table 2).  row_ptr int64[n_vox+1] with row_ptr[0] = 0 and row_ptr[n_vox] =
 * nnz; col int32[nnz] strictly increasing within a row, 0 <= col < n_spots;
 * D_val, L_val float[nnz] finite; voxel_mask uint32[n_vox] (bit b: voxel in
 * structure b).  `format` = FREDOPT_FP32|BF16|FP16 | FREDOPT_ROWS_ALL|ROI
 * [| FREDOPT_INDEX32].
 * The data is validated on the device (FREDOPT_ERR_PATTERN / NONFINITE),
 * the CSC copy of the streamed rows is built (values moved bit-exactly), the
 * values are quantised if asked, and the FP64 row moments |D_i|^2, |L_i|^2,
 * <D_i, L_i> are computed from the stored values.  Replaces any loaded plan
 * and clears constraints, objective and solve state. */
int fredopt_load_influence(fredopt_t h, int64_t n_vox, int32_t n_spots, int64_t nnz,
                           const int64_t* row_ptr, const int32_t* col, const float* D_val,
                           const float* L_val, const uint32_t* voxel_mask, int format,
                           uint32_t flags);

/* Constraint table (Fig. 2; priorities as in Sec. 2.4.3).  Copies `c`.
 * bound must be finite, priority > 0, struct_bit < 32.  Rows whose
 * |a_r|^2 is zero are unreachable and skipped. */
int fredopt_set_constraints(fredopt_t h, int n, const fredopt_constraint* c);

/* Objective terms (Eq. 2).  n = 0 sets no objective (plain feasibility). */
int fredopt_set_objective(fredopt_t h, int n, const fredopt_objective_term* t);

/* Start a solve at w0 (float[n_spots], >= 0): 0 < alpha < 1 (Fig. 3),
 * 0 < relaxation <= 2 (Fig. 2), params may be NULL (defaults). */
int fredopt_begin(fredopt_t h, const float* w0, double alpha, double relaxation,
                  const fredopt_params* params, uint32_t flags);

/* Run `iters` superiorized iterations (Fig. 3 around the simultaneous form
 * of Fig. 2) on the device.  Asynchronous with respect to the host unless
 * an error is detected; returns FREDOPT_ERR_TIMEOUT if a device wait gave up. */
int fredopt_iterate(fredopt_t h, int iters);

/* Finish: w_out float[n_spots]; dose_out, letd_out float[n_vox] in voxel
 * order (LETd = Lw/Dw, 0 where Dw = 0; Eq. 1) from a double-float (about 48-bit,
 * exact products) accumulated final
 * product; the FP64 feasibility and objective check goes to `rep`.  Any
 * output pointer may be NULL. */
int fredopt_end(fredopt_t h, float* w_out, float* dose_out, float* letd_out, fredopt_report* rep,
                uint32_t flags);

/* begin + iterate(iters) + end in one call. */
int fredopt_superiorize(fredopt_t h, const float* w0, int iters, double alpha, double relaxation,
                        const fredopt_params* params, float* w_out, float* dose_out,
                        float* letd_out, fredopt_report* rep, uint32_t flags);

/* Copy up to `max_entries` entries of the per-iteration log (oldest first,
 * the most recent log_capacity iterations); returns the count (>= 0) or an
 * error code. */
int fredopt_get_log(fredopt_t h, fredopt_log_entry* out, int max_entries);

/* Checkpoint / resume of a begun solve: w (float[n_spots]), iteration k and
 * trial counter s.  set_state after begin continues exactly where
 * get_state was taken (same plan, constraints and parameters). */
int fredopt_get_state(fredopt_t h, float* w, int64_t* k, int64_t* s, uint32_t flags);
int fredopt_set_state(fredopt_t h, const float* w, int64_t k, int64_t s, uint32_t flags);

/* ---- single passes of the iteration, for tests and tools ---- */

/* Dose D w and LET-weighted dose L w of every voxel (voxel order), FP32
 * accumulation, one fused pass over the stored values. */
int fredopt_forward(fredopt_t h, const float* w, float* dose_out, float* lw_out, uint32_t flags);

/* u = D^T a_D + L^T a_L over the streamed rows (the transposed product of
 * the projection and gradient steps).  a_D, a_L float[n_vox] in voxel order;
 * entries of voxels outside the streamed rows are ignored. */
int fredopt_backward(fredopt_t h, const float* a_D, const float* a_L, float* u_out, uint32_t flags);

/* One simultaneous feasibility step from x (Fig. 2, simultaneous form):
 * w_out = max(0, x + relaxation * prio_scale * sum_r omega_r t_r a_r).
 * Needs constraints.  norm = FREDOPT_NORM_*. */
int fredopt_feasibility_step(fredopt_t h, const float* x, double relaxation, double prio_scale,
                             int norm, float* w_out, uint32_t flags);

/* One block-iterative sweep from x: the block-iterative form of Fig. 2's
 * row-action sweep.  The voxels that lie in some structure and have
 * influence entries are taken in ascending voxel order and grouped into
 * blocks of S = ceil(count / n_blocks) consecutive voxels (the last block may
 * be smaller; fewer than n_blocks blocks when count < n_blocks); all
 * constraint rows of a voxel share its block.  Blocks are visited in order;
 * inside a block the rows are projected simultaneously from the block's
 * starting point,
 *   x <- x + relaxation * prio_scale * sum_{r in B} (p_r / W_B) t_r a_r,
 * with W_B the priority sum of the block's reachable rows (norm ALL) or of its
 * violated rows (norm VIOLATED); after the last block w_out = max(0, x).
 * n_blocks = 1 is the simultaneous step; one voxel per block approaches the
 * row-action sweep.  1 <= n_blocks <= FREDOPT_MAX_SWEEP_BLOCKS. */
int fredopt_sweep_step(fredopt_t h, const float* x, double relaxation, double prio_scale, int norm,
                       int n_blocks, float* w_out, uint32_t flags);

/* Objective f(x) (Eq. 2 terms, FP64 reduction) and its gradient g (float[n_spots]). */
int fredopt_objective(fredopt_t h, const float* x, double* f_out, float* grad_out, uint32_t flags);

/* ---- volume statistics of a plan (Sec. 2.4.1: DVH, LVH, cDLVH; cDL30; the
 * PTV rule "98% of the volume receives at least 95% of the prescription") ----
 *
 * The voxel values are those of fredopt_end's final pass: (D w)_i and
 * (L w)_i accumulated in double-float (about 48 bits; exact products, relative
 * error per addition <= 3 * 2^-48) over the stored values, then rounded once to
 * FP32 as dose = (D w)_i, LETd = (L w)_i / (D w)_i (0 where (D w)_i <= 0),
 * cDL = c_cdl (L w)_i, with c_cdl of the last begin (default 0.04 um/keV).
 * A structure is the set of voxels whose mask has bit struct_bit set.
 *
 * Per request:
 *   counts[b]    = number of the structure's voxels with
 *                  edges[b] <= v < edges[b+1], b < n_bins (half-open bins;
 *                  a last edge of +INFINITY makes the last bin cumulative);
 *                  edges: n_bins + 1 non-decreasing, non-NaN floats.
 *   at_volume[q] = the value received by the fraction fracs[q] of the
 *                  structure's volume: its k-th largest value with
 *                  k = ceil(fracs[q] * n), n = n_voxels; the product is taken
 *                  in FP64 and a product within 1e-9 * max(1, product) of an
 *                  integer counts as that integer; k is kept in [1, n]; NaN
 *                  when n = 0.  fracs in (0, 1].  The result is one of the
 *                  voxel values, bit for bit (an exact radix selection).
 *   n_voxels     = voxels in the structure.
 * All request arrays are host memory owned by the caller. */
typedef struct fredopt_volume_request {
  int32_t quantity;   /* FREDOPT_Q_DOSE, FREDOPT_Q_CDL or FREDOPT_Q_LETD */
  int32_t struct_bit; /* 0..31 */
  int32_t n_bins;     /* 0..FREDOPT_VOLUME_MAX_BINS in total over the requests */
  int32_t n_fracs;    /* 0..FREDOPT_VOLUME_MAX_FRACS in total over the requests */
  const float* edges; /* [n_bins + 1] (NULL when n_bins = 0) */
  const double* fracs;/* [n_fracs] (NULL when n_fracs = 0) */
  int64_t* counts;    /* out [n_bins] */
  float* at_volume;   /* out [n_fracs] */
  int64_t n_voxels;   /* out */
} fredopt_volume_request; /* 56 bytes */

#define FREDOPT_VOLUME_MAX_REQUESTS 64
#define FREDOPT_VOLUME_MAX_BINS 16384
#define FREDOPT_VOLUME_MAX_FRACS 64

/* Volume statistics of fluence w (float[n_spots]; host, or device with
 * FREDOPT_DEVICE_PTR in flags; NULL = the current iterate of a begun solve)
 * for n_req requests, from one final pass.  Needs a loaded plan.  Errors:
 * FREDOPT_ERR_INVALID_ARG for a bad request (kind, bit, sizes, unsorted or
 * NaN edges, fractions outside (0, 1]); the handle stays usable.  Does not
 * change the solve state. */
int fredopt_volume_stats(fredopt_t h, const float* w, uint32_t flags, int n_req, fredopt_volume_request* req);

/* The per-voxel map (float[n_vox], voxel order; host, or device with
 * FREDOPT_DEVICE_PTR) of one quantity for fluence w (as above), with the
 * values fredopt_volume_stats uses. */
int fredopt_quantity_map(fredopt_t h, const float* w, int quantity, float* out, uint32_t flags);

/* ---- inspection of the device data (bit-exact copies) ---- */

/* Sizes: n_vox, n_spots, nnz, number of streamed rows, nnz of the streamed rows. */
int fredopt_get_sizes(fredopt_t h, int64_t* n_vox, int64_t* n_spots, int64_t* nnz,
                      int64_t* n_rows, int64_t* nnz_rows);

/* The streamed rows: voxel index (int64[n_rows]) and structure mask
 * (uint32[n_rows]) in device order. Host pointers. */
int fredopt_get_rows(fredopt_t h, int64_t* voxel, uint32_t* mask);

/* Stored widths of the loaded plan: bytes per column index of the forward
 * stream and per row index of the transposed product's stream (2 or 4 each,
 * see FREDOPT_INDEX32), and per stored value (4 or 2).  NULL pointers are
 * skipped. */
int fredopt_get_storage(fredopt_t h, int* col_index_bytes, int* row_index_bytes, int* value_bytes);

/* The CSC copy of the streamed rows: col_ptr int64[n_spots+1], row (index
 * into the streamed rows) int32[nnz_rows], D and L values float[nnz_rows]
 * (dequantised: scale * stored value for BF16/FP16). Host pointers. */
int fredopt_get_csc(fredopt_t h, int64_t* col_ptr, int32_t* row, float* D_val, float* L_val);

/* FP64 row moments |D_i|^2, |L_i|^2, <D_i, L_i> of the streamed rows. */
int fredopt_get_moments(fredopt_t h, double* dd, double* ll, double* dl);

/* Device time (ms, CUDA events on the handle's stream) and launch count of
 * each kernel class since the last reset, when timing is enabled.  Classes:
 * 0 forward product, 1 transposed product, 2 constraint evaluation,
 * 3 column finish, 4 scalar finish, 5 other.  With timing enabled at
 * fredopt_begin and use_graphs = 1, the iteration graph holds an event-record
 * node before and after each kernel and every replay points them at fresh
 * events, so the kernels run as graph replays and are still timed one by
 * one.  Timing switched on or off after fredopt_begin runs the iterations as
 * plain launches (timed or not) until the next fredopt_begin. */
#define FREDOPT_KCLASS_N 6
int fredopt_set_timing(fredopt_t h, int enable);
int fredopt_get_timing(fredopt_t h, double* ms, int64_t* launches);

/* Number of kernels the handle has enqueued since the last
 * fredopt_set_timing call (a CUDA-graph replay counts each of its kernels);
 * -1 for a null handle. */
int64_t fredopt_launch_count(fredopt_t h);

/* Architecture of the library's code for `device`, as the CUDA runtime
 * reports it for the kernels it would launch there (cudaFuncGetAttributes):
 * the binary (SASS) version of the forward product and of the transposed
 * product, and the PTX version, each major * 10 + minor (103 for sm_103a).
 * Any pointer may be NULL.  Returns FREDOPT_OK, or FREDOPT_ERR_CUDA when no
 * usable device or code object is found.  The current device is left
 * unchanged. */
int fredopt_kernel_arch(int device, int* fwd_binary, int* bwd_binary, int* ptx_version);

/* Polls of one device-side wait before it gives up: about 1 s on GB300
 * (a failed poll suspends about 4 us); a bulk copy completes in microseconds. */
#define FREDOPT_WAIT_POLLS (1 << 18)

/* Failure-detection check of the bounded device-side wait (no GPU fault
 * involved).  Every device-side wait of the library (the mbarrier that the
 * bulk copies of x and of the CSC windows complete) polls at most
 * FREDOPT_WAIT_POLLS times; when it gives up the kernel sets the handle's device error
 * word and returns, and the next synchronising call reports
 * FREDOPT_ERR_TIMEOUT and clears the word.  This call runs that wait alone in
 * one CTA on the handle's stream, on a phase that only the CTA itself can
 * complete:
 *   arrive != 0  the CTA arrives first; the wait succeeds; returns FREDOPT_OK.
 *   arrive == 0  nothing arrives; after `spins` polls (0 = the bound the
 *                kernels use, FREDOPT_WAIT_POLLS) the wait gives up; returns FREDOPT_ERR_TIMEOUT
 *                and leaves the handle usable (error word and tile counters
 *                cleared).
 * `elapsed_ms` (may be NULL) receives the kernel's device time, which at
 * spins == 0 is the time a failed wait takes to give up.  Synchronises the
 * handle's stream.  Needs no loaded plan. */
int fredopt_check_wait(fredopt_t h, int arrive, int spins, float* elapsed_ms);

/* ---- tile autotuning and batches of plans ----
 *
 * Tiles are the contiguous ranges of rows (forward product) and of column
 * chunks (transposed product) that warps stream: one per warp, or (see
 * fredopt_params.tile_balance) 7 per warp of decreasing size, claimed in
 * order.  Their sizes are measured in nonzeros plus a weight per row end /
 * per chunk.  A segment's sum does not depend on which warp streams it, so
 * the weights change speed, never a result bit.  fredopt_autotune times the forward and transposed products
 * with `reps` repetitions for each candidate weight (rows: 16..512, chunks:
 * 4..1024) and keeps the fastest pair; it may be called after load or after
 * begin.  fredopt_get_tuning reports the weights in use. */
int fredopt_autotune(fredopt_t h, int reps, int64_t* row_cost, int64_t* chunk_cost);
int fredopt_get_tuning(fredopt_t h, int64_t* row_cost, int64_t* chunk_cost);

/* A batch runs the iterations of several begun plans (distinct handles and
 * streams, one device, timing off) as one CUDA graph per iteration whose
 * branches are the plans, so plans of uneven sizes run concurrently from a
 * single launch.  Each plan's results are bit-identical to running it alone.
 * Plans loaded with FREDOPT_SHARED leave SMs to each other (small plans use
 * few CTAs), which raises the batch's throughput.
 * Create after fredopt_begin on every handle (preferably with use_graphs = 0);
 * then fredopt_batch_iterate (asynchronous), fredopt_batch_sync (waits and
 * returns the device time of the iterate calls), fredopt_end per handle. */
typedef struct fredopt_batch* fredopt_batch_t;
int fredopt_batch_create(fredopt_batch_t* out, const fredopt_t* handles, int n);
/* The same with a second graph of `depth` iterations of every plan (1 <=
 * depth <= FREDOPT_BATCH_MAX_DEPTH): fredopt_batch_iterate replays it
 * iters / depth times and the one-iteration graph for the rest, so a batch of
 * small, launch-bound plans pays one graph launch per `depth` iterations.
 * Each plan's kernels run in the same order as alone: results are
 * bit-identical for every depth.  fredopt_superiorize_batch uses depth
 * min(iters, FREDOPT_BATCH_DEPTH). */
#define FREDOPT_BATCH_MAX_DEPTH 64
#define FREDOPT_BATCH_DEPTH 10
int fredopt_batch_create_depth(fredopt_batch_t* out, const fredopt_t* handles, int n, int depth);
int fredopt_batch_iterate(fredopt_batch_t b, int iters);
int fredopt_batch_sync(fredopt_batch_t b, double* device_ms);
int fredopt_batch_destroy(fredopt_batch_t b);

/* begin + batch iterate + end for n plans in one call; arrays of n pointers
 * (output arrays and reps may be NULL). */
int fredopt_superiorize_batch(const fredopt_t* handles, int n, const float* const* w0, int iters, double alpha,
                              double relaxation, const fredopt_params* params, float* const* w_out,
                              float* const* dose_out, float* const* letd_out, fredopt_report* reps,
                              uint32_t flags);

/* ---- serving: continuous batching of plan re-optimisations ----
 *
 * A server owns one device.  Requests (a whole plan plus its solve) are
 * admitted first-in first-out while their estimated device footprint fits
 * under `mem_cap_bytes` and fewer than `max_active` plans are loaded; each
 * admitted plan stays resident on its own stream and its iterations are
 * enqueued in rounds of `round_iters`, interleaved with the other active
 * plans, so that their kernels overlap on the device.  A plan admitted
 * with no request waiting gets a CUDA stream priority below the plans
 * already in flight (an older plan's kernels are scheduled first, younger
 * plans fill the SMs it leaves idle), so it runs about as fast as alone;
 * plans admitted from a backlog share the lowest priority and interleave.
 * With max_active > 1 the server loads every plan with FREDOPT_SHARED (launch
 * shapes for running beside other plans).  A plan's results do not depend on
 * its co-tenants (tiles depend on the plan and its launch shapes alone and a
 * tile's sums on nothing else): they are bit-identical to a
 * fredopt_superiorize call on the same inputs loaded with the same format
 * (FREDOPT_SHARED added when max_active > 1).
 * All request pointers are host pointers owned by the caller and must stay
 * valid until the request is done (status DONE or an error).  Thread-safe. */
typedef struct fredopt_request {
  int64_t n_vox;
  int64_t nnz;
  int32_t n_spots;
  int32_t format;                        /* as fredopt_load_influence */
  const int64_t* row_ptr;                /* plan, as fredopt_load_influence */
  const int32_t* col;
  const float* D_val;
  const float* L_val;
  const uint32_t* voxel_mask;
  int32_t n_constraints;
  int32_t n_objective;
  const fredopt_constraint* constraints;
  const fredopt_objective_term* objective;
  const float* w0;                       /* solve, as fredopt_superiorize */
  int32_t iters;
  int32_t pad;
  double alpha;
  double relaxation;
  fredopt_params params;
  float* w_out;                          /* outputs (float[n_spots], float[n_vox] x 2; may be NULL) */
  float* dose_out;
  float* letd_out;
} fredopt_request;

#define FREDOPT_QUEUED 0
#define FREDOPT_LOADING 1
#define FREDOPT_RUNNING 2
#define FREDOPT_DONE 3

typedef struct fredopt_ticket_info {
  int32_t status;        /* FREDOPT_QUEUED .. FREDOPT_DONE, or a negative error code */
  int32_t pad;
  double t_submit;       /* seconds since the server was created */
  double t_admit;        /* admitted (memory reserved), load starts */
  double t_start;        /* loaded, iterations start */
  double t_done;         /* outputs written */
  int64_t footprint_bytes;
  fredopt_report report; /* as fredopt_end */
} fredopt_ticket_info;

typedef struct fredopt_server* fredopt_server_t;

/* Estimate of the device memory one plan needs while it loads and runs: the
 * peak of the load (including the CSC build's scratch of one record per
 * nonzero: 16 bytes with FP32 values, 8 with 16-bit) and the resident CSR,
 * CSC, based row offsets with their block headers, vectors and tables.  The overflow table of wide 128-element
 * blocks (rows spanning 65536 or more) is counted for one such block per
 * column boundary plus one in 16 blocks; for plans with sparser rows the
 * estimate can be low, and a load that then does not fit fails with
 * FREDOPT_ERR_OOM without disturbing the plans in flight.  The server admits
 * requests while the sum of these estimates stays under its cap. */
int64_t fredopt_footprint_bytes(int64_t n_vox, int32_t n_spots, int64_t nnz, int format);

int fredopt_server_create(fredopt_server_t* out, int device, int64_t mem_cap_bytes, int max_active,
                          int round_iters);
/* Queue a request; FREDOPT_ERR_OOM if its footprint exceeds the cap. */
int fredopt_server_submit(fredopt_server_t s, const fredopt_request* r, int64_t* ticket);
int fredopt_server_poll(fredopt_server_t s, int64_t ticket, fredopt_ticket_info* info);
/* Block until the request is done or `timeout_s` passes (FREDOPT_ERR_TIMEOUT). */
int fredopt_server_wait(fredopt_server_t s, int64_t ticket, double timeout_s, fredopt_ticket_info* info);
/* Block until every submitted request is done. */
int fredopt_server_drain(fredopt_server_t s, double timeout_s);
int fredopt_server_stats(fredopt_server_t s, int64_t* mem_used, int* n_active, int* n_queued);
/* Finish the active plans, drop the queued ones and free the server. */
int fredopt_server_destroy(fredopt_server_t s);

/* ---- transposed product without device allocation ----
 *
 * The paper has no counterpart: this is a service entry point of this
 * library.  It computes u = D^T a_D + L^T a_L (the product of the
 * projection and gradient steps) from a CSC matrix pair that the caller
 * already holds in device memory, for callers that cannot allocate device
 * memory where they need it (for example a host program whose own pool owns
 * the GPU's memory, or a latency-critical loop that avoids cudaMalloc and
 * cudaFree because they can synchronise the device).  It needs no handle
 * and allocates nothing: its scratch is one fixed device array of 4.25 MiB
 * inside the library, which every GPU that loads the library keeps until
 * the process exits.
 *
 * Arguments (all pointers are device pointers on the current device):
 * col_ptr int64[n_cols+1] (ascending, col_ptr[0] = 0, col_ptr[n_cols] = nnz),
 * row int32[nnz] (row of each nonzero, 0 <= row < n_rows), D_val, L_val
 * float[nnz]; a_D, a_L float[n_rows] (either may be NULL = zeros); u_out
 * float[n_cols] (written).  The work is enqueued on `cuda_stream` (a
 * cudaStream_t, NULL = the legacy default stream) and the call returns
 * without waiting; synchronise the stream before reading u_out.
 * Limits: 1 <= n_cols <= 65536 and nnz / 4096 + n_cols <= 1048576, otherwise
 * FREDOPT_ERR_SHAPE.  Row indices outside [0, n_rows) are skipped and
 * column pointers are clamped to [0, nnz], so malformed input cannot read
 * outside the arrays.  The first call on a device looks up the scratch
 * address for that device (set-up once per device, with that device
 * current); make that first call before any stream capture.  The address is
 * kept until the process exits: after a cudaDeviceReset this entry point
 * must not be called again in the process.  All calls share the one scratch
 * array, which keeps the last call's contents (each call rewrites what it
 * reads): calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  The result is deterministic:
 * the same inputs give the same bits. */
int fredopt_backward_noalloc(int64_t n_rows, int32_t n_cols, int64_t nnz, const int64_t* col_ptr,
                             const int32_t* row, const float* D_val, const float* L_val,
                             const float* a_D, const float* a_L, float* u_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FREDOPT_H */
