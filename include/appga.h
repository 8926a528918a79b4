/*
 * appga.h -- C ABI of the GB300 (sm_103a) APPGA reconstruction library.
 *
 * The library runs the per-iteration hot path of the accelerated
 * preconditioned proximal gradient algorithm (APPGA) with generalized
 * Nesterov (GN) momentum for PET reconstruction under the smoothed
 * higher-order isotropic TV penalty (SHOITV), arXiv 2409.13344:
 *
 *   f~^k     = f^k + theta_k (f^k - f^{k-1})                       (Eq. APPGAiter)
 *   f^{k+1}  = max(f~^k - P (grad F(f~^k) + B^T grad phi~(B f~^k)), 0)
 *   grad F   = A^T (1 - g / (A f + gamma))                         (Sec. 2.2)
 *   theta_k  = (t_{k-1} - 1) / t_k,  t_k = a k^omega + b           (Eq. GNtheta)
 *   P        = beta diag(f^k / Lambda), Lambda = A^T 1 (1 where 0) (Eq. EM)
 *
 * Conventions (all calls):
 *  - Images are N x N, vectorised row-major: pixel j = r*N + c.  d = N*N.
 *  - Sinograms have m bins; A is m x d with nonnegative entries.
 *  - Pointers are DEVICE pointers unless the name ends in _host.  The caller
 *    owns every input and output buffer; the library owns matrix handles and
 *    their device workspaces.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered; a call that returns a host value
 *    (objective, stats) synchronises that stream before returning.
 *  - Every call returns an appga_status; the library never aborts, traps or
 *    exits.  appga_last_error() gives a one-line message for the calling
 *    thread's most recent failure.
 *  - A context and the matrices created from it may be used by one host
 *    thread at a time.
 */
#ifndef APPGA_H
#define APPGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  APPGA_OK = 0,
  APPGA_EINVAL = 1,   /* bad shape, CSR, parameter or null pointer */
  APPGA_ENOMEM = 2,   /* device or host allocation failed */
  APPGA_EDOMAIN = 3,  /* non-finite input, g < 0 or gamma <= 0 */
  APPGA_ETIMEOUT = 4, /* a bounded wait ran out */
  APPGA_ECUDA = 5,    /* a CUDA runtime call failed */
  APPGA_ENODEV = 6,   /* no usable CUDA device */
  APPGA_EBUSY = 7,    /* no free slot / resource in use */
  APPGA_ENUMERIC = 8  /* the device flagged a non-finite intermediate */
} appga_status;

typedef struct appga_ctx appga_ctx;
typedef struct appga_matrix appga_matrix;

/* Matrix-creation flags. */
#define APPGA_A_BF16_COPY 1u /* also keep a BF16 copy of A's values */
#define APPGA_A_NO_FOLD 2u   /* do not fold A by its quarter-turn symmetry */

/* Precision of A's values inside the projectors. */
#define APPGA_PREC_FP32 0
#define APPGA_PREC_BF16 1

/* Momentum rules. */
#define APPGA_MOMENTUM_GN 0       /* Eq. GNtheta: t_k = a k^omega + b */
#define APPGA_MOMENTUM_NONE 1     /* theta_k = 0: PPGA, Eq. PPGAiter */
#define APPGA_MOMENTUM_NESTEROV 2 /* t_k = (1 + sqrt(1 + 4 t_{k-1}^2)) / 2, Sec. 4.3 */

/* Device sticky flags reported in appga_stats.flags. */
#define APPGA_FLAG_NONFINITE 1 /* a non-finite value met in a projector */
#define APPGA_FLAG_TIMEOUT 2   /* reserved: a bounded device wait ran out (no kernel of this
                                  version waits on another block, so it is not raised) */
#define APPGA_FLAG_DOMAIN 4    /* an input failed the device-side check; no map ran */

const char* appga_status_string(appga_status s);
const char* appga_last_error(void);
/* Library version, e.g. "0.1.0". */
const char* appga_version(void);

/* ------------------------------------------------------------------ context
 * appga_ctx_create: bind the calling thread to CUDA device `device` and
 * create a context.  Errors: APPGA_ENODEV if the device does not exist,
 * APPGA_ECUDA on runtime failure. */
appga_status appga_ctx_create(int32_t device, appga_ctx** out);
appga_status appga_ctx_destroy(appga_ctx* ctx);

/* ------------------------------------------------------------------ matrix
 * appga_matrix_create: copy the host CSR of the system matrix A (m x d,
 * Sec. 2.1 "A in R_+^{m x d}") to the device and build there:
 *   - A as a row-padded CSR (each row padded with zeros to a multiple of 4
 *     entries so rows start on 16-byte boundaries),
 *   - A^T as a row-padded CSR (built on the host by a stable counting sort,
 *     so the back-projection needs no atomics),
 *   - 1/Lambda with Lambda_j = (A^T 1)_j if positive, else 1 (Eq. EM),
 *   - the quarter-turn folded copies of the solver loop, when A has that
 *     symmetry bit for bit: for a parallel-beam scanner with NPA angles
 *     a*pi/NPA (NPA even) stored angle-major (row a*nb + b, m = NPA*nb) over
 *     an N x N image (N even), the ray of angle a + NPA/2 and bin nb-1-b is
 *     the ray of angle a and bin b turned a quarter turn, which moves pixel
 *     (r, c) to (N-1-c, r).  The loop then streams only the first m/2 rows of
 *     A and of its transpose, each entry serving two products per projection;
 *     the results are those of the whole A up to the order of FP32 sums.
 *     The check is exact (same columns after the turn, same value bits); any
 *     other A, or flags with APPGA_A_NO_FOLD, keeps the unfolded loop.
 * n_side is N (d must equal N*N); n_angles is the number of projection
 * angles (NPA, used by the default initial image, Sec. 4.1, and the fold).
 * row_ptr_host: int32[m+1], col_host: int32[nnz], val_host: float[nnz]; the
 * host arrays are only read during the call.  Validation: row_ptr[0] = 0,
 * nondecreasing, row_ptr[m] = nnz; 0 <= col < d; values finite and >= 0
 * (EINVAL / EDOMAIN otherwise).  flags: APPGA_A_BF16_COPY, APPGA_A_NO_FOLD. */
appga_status appga_matrix_create(appga_ctx* ctx, int32_t m, int32_t d, int32_t n_side,
                                 int32_t n_angles, const int32_t* row_ptr_host,
                                 const int32_t* col_host, const float* val_host,
                                 uint32_t flags, appga_matrix** out);
appga_status appga_matrix_destroy(appga_matrix* mat);

typedef struct {
  int32_t m, d, n_side, n_angles;
  int64_t nnz;          /* entries of A as given */
  int64_t nnz_padded_a; /* stored entries of A (row padded) */
  int64_t nnz_padded_t; /* stored entries of A^T (row padded) */
  int32_t has_bf16;
  int64_t device_bytes; /* device memory held by the handle */
  int32_t packed_columns; /* 1 if the solver loop streams 2-byte packed column
                             indices (every column below 2^20 and, within each
                             4-entry pack of a row, within [-8192, 8191] of the
                             pack's first column); 0: 4-byte indices */
  int32_t sliced_layout;  /* 1 if the solver loop's projections stream A and
                             A^T in the sliced (ELLPACK-like) layout; 0: CSR */
  int32_t quarter_turn_folded; /* 1 if the solver loop streams the quarter-turn
                                  folded halves of A and A^T (see above) */
  int32_t reserved;
} appga_matrix_info;
appga_status appga_matrix_get_info(const appga_matrix* mat, appga_matrix_info* out);

/* --------------------------------------------------------------- parameters
 * Model parameters lambda1, lambda2 >= 0, eps > 0 (Sec. 2.1, Eq. def:smoothL2);
 * momentum a > 0, b, omega in (0, 1] (Eq. GNtheta; the paper uses a = 1/8,
 * b = 1); step size beta > 0 (Eq. EM).  max_iters >= 0 APPGA maps.
 * rel_obj_tol > 0 stops once |Phi(f^{k+1}) - Phi(f^k)| <= tol |Phi(f^k)|.
 * precond_freeze_iter = K_P >= 1 freezes P = beta f^{K_P}/Lambda after
 * iteration K_P (Sec. 4.1 allows fixing P after early iterations); -1 never
 * freezes.  track_objective = 1 evaluates Phi(f^k) in FP64 on the device
 * every iteration (forced on when rel_obj_tol > 0).  graph_iters = number of
 * iterations captured per CUDA graph replay (0 = library default); the stop
 * flag is polled once per replay. */
typedef struct {
  double lambda1, lambda2, eps;
  double omega, a, b;
  double beta;
  int32_t max_iters;
  double rel_obj_tol;
  int32_t precond_freeze_iter;
  int32_t a_precision; /* APPGA_PREC_FP32 or APPGA_PREC_BF16 */
  int32_t momentum;    /* APPGA_MOMENTUM_* */
  int32_t track_objective;
  int32_t graph_iters;
} appga_params;

/* Defaults: lambda1 = 0.1, lambda2 = 0.05, eps = 1e-3, omega = 0.5, a = 1/8,
 * b = 1, beta = 1, max_iters = 100, rel_obj_tol = 0, precond_freeze_iter = -1,
 * FP32, GN momentum, track_objective = 0, graph_iters = 0. */
void appga_params_default(appga_params* p);
/* EINVAL with a message if a field is out of range (see above; also a < 1/2
 * when omega = 1, the range of the convergence theorem, Thm. 10). */
appga_status appga_params_validate(const appga_params* p);

/* GN momentum scalar theta_k = (t_{k-1}-1)/t_k, t_k = a k^omega + b, in
 * FP64 (Eq. GNtheta).  k >= 1.  Host function, for callers and tests. */
double appga_gn_theta(int32_t k, double a, double b, double omega);

typedef struct {
  int32_t iters;        /* APPGA maps applied to produce the result */
  int32_t result_k;     /* iterate index of the result (f^{result_k}) */
  int32_t stopped_early;/* 1 if rel_obj_tol fired */
  int32_t flags;        /* APPGA_FLAG_* sticky device flags */
  int64_t guard_hits;   /* bins where A f~ + gamma < kappa*gamma (guarded) */
  double phi;           /* Phi(result) in FP64, or NaN if not tracked */
  double phi_prev;      /* Phi of the iterate before the result, or NaN */
} appga_stats;

/* ------------------------------------------------- single hot-path steps
 * Each call below runs the kernel the solver loop runs for that step, once,
 * with the given inputs (appga_forward_ratio runs the forward kernel's
 * double-float instance; the solver loop accumulates y in FP32 and gathers
 * f from a copy in an 8 x 8-tiled pixel order).
 *
 * appga_forward_ratio (steps a1-a2, Sec. 2.2 grad F): for every bin i
 *   y_i  = (A f)_i, accumulated in double-float (FP32 pairs) and stored as
 *          FP64 in y_out[m];
 *   w_i  = 1 - g_i / den_i with den_i = max(y_i + gamma_i, 1e-3 gamma_i)
 *          (FP32 in w_out[m]; the gradient uses the ratio only through w);
 *   data_out (device double[1], may be NULL) = sum_i y_i - g_i ln(y_i + gamma_i)
 *          in FP64 (the fidelity F, Eq. FidelityTerm, valid for f >= 0).
 * f: float[d]; g, gamma: float[m]. */
appga_status appga_forward_ratio(appga_ctx* ctx, const appga_matrix* mat, const float* f,
                                 const float* g, const float* gamma, double* y_out,
                                 float* w_out, double* data_out, void* stream);

/* appga_backproject (step a3): out[d] = A^T w via the transposed CSR, one
 * warp per pixel row, FP32 accumulation, no atomics.  w: float[m]. */
appga_status appga_backproject(appga_ctx* ctx, const appga_matrix* mat, const float* w,
                               float* out, void* stream);

/* appga_shoitv_grad (step a4, Sec. 2.1-2.2): out = B^T grad phi~(B f) for an
 * N x N image f (float[N*N]), with the six difference fields of B1 and B2
 * and the group norms max(||.||_2, eps), computed by a shared-memory
 * halo-tiled stencil in FP32. */
appga_status appga_shoitv_grad(appga_ctx* ctx, int32_t n_side, const float* f, double lambda1,
                               double lambda2, double eps, float* out, void* stream);

/* appga_pixel_update (steps a0, a3, a4, a5 fused, Eq. APPGAiter + Eq. EM):
 *   f~ = f_cur + theta (f_cur - f_prev),
 *   f_next = max(f~ - beta f_cur / Lambda * (A^T w + B^T grad phi~(B f~)), 0)
 * with w the back-projection weight from appga_forward_ratio evaluated at f~.
 * Uses lambda1, lambda2, eps, beta from params. */
appga_status appga_pixel_update(appga_ctx* ctx, const appga_matrix* mat, const float* f_prev,
                                const float* f_cur, const float* w, double theta,
                                const appga_params* params, float* f_next, void* stream);

/* appga_objective (step a6): Phi(f) = F(f) + phi~(B f) in FP64 (Eq. def:phi,
 * no constant terms) for f >= 0, written to *phi_out_host.  Synchronises. */
appga_status appga_objective(appga_ctx* ctx, const appga_matrix* mat, const float* f,
                             const float* g, const float* gamma, const appga_params* params,
                             double* phi_out_host, void* stream);

/* appga_initial_image: f_out = TMC * 1_disk (Sec. 4.1), TMC = ACTc/(NPFOV*NPA),
 * ACTc = sum g - sum gamma (FP64 on the device), disk = pixel centres with
 * x^2 + y^2 <= (N/2)^2. */
appga_status appga_initial_image(appga_ctx* ctx, const appga_matrix* mat, const float* g,
                                 const float* gamma, float* f_out, void* stream);

/* ------------------------------------------------------------------ solver
 * appga_reconstruct: run APPGA from f^0 = f^1 = f_init (NULL: the initial
 * image above) for params->max_iters maps or until the stopping test fires,
 * and write the result to f_out (float[d]).  g: float[m] (counts, >= 0),
 * gamma: float[m] (> 0).  stats_host may be NULL.  The iteration runs as
 * captured CUDA graphs on `stream`; the call returns once the result is in
 * f_out (it synchronises the stream).  Inputs are validated on the device
 * (EDOMAIN for negative or non-finite g, non-positive or non-finite gamma).
 * Arithmetic: FP32 projections and updates, y = A f accumulated in FP32,
 * the objective's logarithm and sums in double-float, the momentum scalars,
 * Phi and the stopping test in FP64.  ENUMERIC if a non-finite value
 * appeared. */
appga_status appga_reconstruct(appga_ctx* ctx, const appga_matrix* mat, const float* g,
                               const float* gamma, const float* f_init,
                               const appga_params* params, float* f_out,
                               appga_stats* stats_host, void* stream);

/* appga_resume: continue APPGA from the state (f^{k0-1}, f^{k0}) at iteration
 * index k0 >= 1 (theta_{k0} is the first momentum used).  Writes f^{r-1} to
 * f_out_prev (may be NULL) and the result f^{r} to f_out.  Resuming from a
 * snapshot gives the same result as running uninterrupted (theta_k depends
 * only on k). */
appga_status appga_resume(appga_ctx* ctx, const appga_matrix* mat, const float* g,
                          const float* gamma, const float* f_prev, const float* f_cur,
                          int32_t k0, const appga_params* params, float* f_out_prev,
                          float* f_out, appga_stats* stats_host, void* stream);

/* appga_reconstruct_host: appga_reconstruct with HOST buffers (g_host,
 * gamma_host: float[m]; f_init_host: float[d] or NULL; f_out_host: float[d]).
 * Copies in and out through the library's pinned staging buffers. */
appga_status appga_reconstruct_host(appga_ctx* ctx, const appga_matrix* mat, const float* g_host,
                                    const float* gamma_host, const float* f_init_host,
                                    const appga_params* params, float* f_out_host,
                                    appga_stats* stats_host, void* stream);

/* ------------------------------------------------------------------ batched
 * appga_reconstruct_batched: K independent slices (1 <= K <= 128) that share
 * this matrix, iterated together so every nonzero of A and A^T is read once
 * per iteration for all slices (CSR times a K-column block).  g, gamma:
 * float[K][m] (slice-major); f_init: float[K][d] or NULL (each slice's initial
 * image, Sec. 4.1); f_out: float[K][d]; stats_host: appga_stats[K] or NULL
 * (phi is the FP64 objective of each result).  Every slice runs `params`
 * for max_iters maps or until its own stopping test fires; a slice's result
 * does not depend on the other slices in the batch.  The projector
 * accumulation is FP32 in a different order from the single-slice path, so
 * results agree with appga_reconstruct to FP32 rounding.  Slices are held in
 * blocks of Kp = 32, 64 or 128 slots (the smallest that holds K); the
 * kernels index them with 32-bit offsets, so max(m, d) * Kp must stay below
 * 2^31 (else EINVAL).  EINVAL also for K outside [1, 128] or bad params;
 * EDOMAIN for non-finite or negative g or f_init, or gamma <= 0.  Synchronises. */
appga_status appga_reconstruct_batched(appga_ctx* ctx, const appga_matrix* mat, int32_t K,
                                       const float* g, const float* gamma, const float* f_init,
                                       const appga_params* params, float* f_out,
                                       appga_stats* stats_host, void* stream);

/* appga_gather_probe: the rate of the batched projectors' inner loop alone on
 * this matrix (a measurement utility; the paper has no counterpart).  It
 * times `launches` runs of a kernel that runs only that loop: every row
 * reduced against the width-float rows of a slot-minor block named by its
 * columns (the column/value stream and the gathers), in the projectors' row
 * order, with no epilogue, stencil or pixel update, for several grid sizes
 * (blocks per SM), and keeps the fastest.  *gbs_fwd: A's rows against an
 * image block [d][width] (the forward projection); *gbs_bwd: A^T's rows
 * against a weight block [m][width] (the back-projection); both host doubles,
 * gathered bytes (padded entries x width x 4) per second / 1e9.  width: 32,
 * 64 or 128 (max(m, d) * width below 2^31, else EINVAL); launches >= 1 per
 * grid size.  Uses the matrix's batched
 * workspace; synchronises. */
appga_status appga_gather_probe(appga_ctx* ctx, const appga_matrix* mat, int32_t width,
                                int32_t launches, double* gbs_fwd, double* gbs_bwd);

/* ------------------------------------------------------------ 3-D SHOITV
 * The paper states HOITV in 2-D (Sec. 2.1) and refers to other work for 3-D.
 * These calls use its Kronecker generalisation: for a volume of nz slices of
 * n x n pixels (voxel (z, r, c) at z*n*n + r*n + c, slice-major), D the
 * paper's backward difference (zero first row) along each axis,
 *   B1 = [Dc; Dr; Dz]  (3 components per voxel),
 *   B2 = [-Dc^T Dc; -Dr^T Dc; -Dr^T Dr; -Dr Dc^T;          (the 2-D blocks)
 *         -Dz^T Dz; -Dz^T Dc; -Dz Dc^T; -Dz^T Dr; -Dz Dr^T] (9 components),
 * and phi~ = lambda1 sum s_eps(3-vector) + lambda2 sum s_eps(9-vector)
 * (Eq. def:smoothL2).  With nz = 1 this is the 2-D SHOITV of the slice.
 *
 * appga_shoitv3d_grad: out = B^T grad phi~(B f) (Eq. gradenvL2 on the 3-D
 * groups) for the volume f; f, out: float[nz][n*n] device (distinct
 * buffers); 1 <= nz <= 128.  reg_out (device double, may be NULL): phi~(B f)
 * in FP64 (double-float sums).  Allocates a small stream-ordered scratch
 * when reg_out is given.  EINVAL for bad sizes or parameters (lambda >= 0,
 * eps > 0, all finite). */
appga_status appga_shoitv3d_grad(appga_ctx* ctx, int32_t n_side, int32_t nz, const float* f,
                                 double lambda1, double lambda2, double eps, float* out,
                                 double* reg_out, void* stream);

/* appga_reconstruct_volume: APPGA (Eq. APPGAiter, EM preconditioner Eq. EM)
 * on a volume of nz slices (1 <= nz <= 128) whose slices share this matrix
 * and have their own sinograms: Phi(f) = sum_z F(f_z) + phi~(B f) with the
 * 3-D B above.  g, gamma: float[nz][m] device; f_init: float[nz][d] or NULL
 * (each slice's TMC * 1_disk, Sec. 4.1); f_out: float[nz][d].  One momentum
 * sequence and one stopping test (params->rel_obj_tol on the volume's Phi)
 * serve the whole volume.  Runs the batched SpMM kernels on the nz slices
 * plus the 3-D stencil, under captured CUDA graphs.  stats_host (one
 * appga_stats, may be NULL): iterations, stop flag, flags, guard hits summed
 * over the slices, phi = the volume's FP64 Phi of the result when the
 * objective is tracked.  EINVAL / EDOMAIN as appga_reconstruct_batched.
 * Synchronises. */
appga_status appga_reconstruct_volume(appga_ctx* ctx, const appga_matrix* mat, int32_t nz,
                                      const float* g, const float* gamma, const float* f_init,
                                      const appga_params* params, float* f_out,
                                      appga_stats* stats_host, void* stream);

/* appga_autotune_batched: picks the launch schedule of the batched kernels
 * for this matrix, batch width and precision by timing the solver itself on
 * the caller's K slices (g, gamma: float[K][m] device; params as for
 * appga_reconstruct_batched; a_precision selects FP32 or BF16 values).  The
 * paper has no counterpart; the schedule changes only speed, never results.
 * Each trial runs 4 + 16 APPGA maps of every slice (after 4 warm-up maps)
 * and is timed with CUDA events on the library stream.  Tunables, searched
 * one after another from the kernels' defaults: the sub-batch width (run K
 * slices as several batches of 32 or 64), SpMV blocks per SM of the forward
 * phase, blocks per SM of the back-projection, stencil blocks per SM, and for
 * each projection the rows it gathers per step of its staged (column, value)
 * pairs (8, or 4: fewer loads in flight, fewer registers; separate kernel
 * instances).  The
 * best schedule is kept in the matrix handle and used by later
 * appga_reconstruct_batched calls (and server pools) with the same padded
 * width (32, 64 or 128) and precision.  out_host (may be NULL) receives the
 * choice and the measured times.  Synchronises; allocates a K x d scratch
 * image block for the trials.  A schedule never changes the image of a run
 * with a fixed number of maps (every slot's arithmetic is the same); the
 * FP64 objective is summed in a schedule-dependent grouping, so it and a
 * relative-objective stop may differ in the last bits. */
typedef struct {
  int32_t K;
  int32_t a_precision;
  int32_t spmv_per_sm;    /* 0 = kernel default */
  int32_t stencil_per_sm; /* 0 = kernel default */
  int32_t pixel_per_sm;   /* 0 = kernel default */
  int32_t chunk;          /* slices per sub-batch; 0 = the whole batch */
  int32_t gather_rows_fw; /* image rows the forward projection gathers per step: 8 or 4 (0 = 8) */
  int32_t gather_rows_px; /* weight rows the back-projection gathers per step: 8 or 4 (0 = 8) */
  double us_per_slice_iter;         /* chosen schedule, microseconds per slice-iteration */
  double us_per_slice_iter_default; /* the default schedule */
} appga_batch_tuning;
appga_status appga_autotune_batched(appga_ctx* ctx, const appga_matrix* mat, int32_t K,
                                    const float* g, const float* gamma,
                                    const appga_params* params, appga_batch_tuning* out_host);
/* Reads / sets the schedule kept for (tuning->K's padded width,
 * tuning->a_precision), e.g. to reuse a tuning saved by an earlier process;
 * only K, a_precision and the six schedule fields are used (values per SM
 * in [0, 16], 0 = default; chunk 0, 32 or 64; gather rows 0, 4 or 8).  get
 * fills the schedule fields (zeros if none is kept).  EINVAL for values out
 * of range. */
appga_status appga_batch_schedule_get(const appga_matrix* mat, appga_batch_tuning* tuning_host);
appga_status appga_batch_schedule_set(appga_matrix* mat, const appga_batch_tuning* tuning_host);

/* appga_objective_noalloc: appga_objective without any memory allocation.
 * The paper has no counterpart; this is a library-side convenience.
 * Some callers cannot let a library allocate device memory after start-up:
 * processes that give all device memory to their own pool at launch (a
 * serving process or a framework allocator that owns every byte) and
 * real-time reconstruction loops that forbid allocation once running
 * (cudaMalloc/cudaFree can synchronise the device).  This call computes the
 * same Phi(f) as appga_objective but keeps its scratch (reduction partials,
 * tickets, a scratch state) in one fixed 256 KiB device array inside the
 * library, and writes the FP64 result to the DEVICE pointer phi_out
 * (double[1]) on `stream` without synchronising.  It allocates nothing; the
 * caller passes f, g, gamma, phi_out and a matrix created beforehand.
 * Limits: matrices whose scratch needs more than 256 KiB (images larger than
 * 512 x 512 or sinograms beyond about 263 K bins) are rejected with
 * APPGA_EINVAL.  Every GPU that loads the library holds the array until the
 * process exits.  The first call on a device looks up the array's device
 * address (with that device current); make that first call before any
 * stream capture.  All calls share the one array: calls whose work overlaps
 * on the GPU (different streams, or concurrent host threads) race and give
 * wrong results; serialise them. */
appga_status appga_objective_noalloc(appga_ctx* ctx, const appga_matrix* mat, const float* f,
                                     const float* g, const float* gamma,
                                     const appga_params* params, double* phi_out, void* stream);

/* ------------------------------------------------------------------ AFPPA
 * appga_afppa_reconstruct: the accelerated fixed-point proximity algorithm
 * for the non-smooth HOITV model F(f) + lam1 sum ||(B1 f)_i|| + lam2 sum
 * ||(B2 f)_i|| + iota(f) (Eq. model:HOTV), the paper's extension of the GN
 * momentum (Sec. 4.4):
 *   f~ = f^k + theta_k (f^k - f^{k-1}), b~, c~ likewise,
 *   f^{k+1} = max(f~ - P (grad F(f~) + B1^T b~ + B2^T c~), 0),
 *   b^{k+1} = rho1 (I - prox_{(lam1/rho1)||.||})(b~/rho1 + B1 (2 f^{k+1} - f~)),
 *   c^{k+1} = rho2 (I - prox_{(lam2/rho2)||.||})(c~/rho2 + B2 (2 f^{k+1} - f~)),
 * with P = beta diag(f^k / Lambda) (Eq. EM), rho1 = 1/(2*8*p_max),
 * rho2 = 1/(2*64*p_max) from the largest entry of P each step, duals starting
 * at zero, and f^0 = f^1 = f_init (NULL: TMC * 1_disk).  params: lambda1,
 * lambda2, beta, omega, a, b, momentum (APPGA_MOMENTUM_NONE gives FPPA),
 * max_iters, precond_freeze_iter and a_precision are used; eps and
 * track_objective are not; rel_obj_tol must be 0 (the run makes max_iters
 * maps).  f_out: float[d]; b_out: float[2][d] and c_out: float[4][d] (field-
 * major, each may be NULL) receive the last duals; stats_host (may be NULL)
 * the number of maps, RE = ||f^{K+1} - f^K|| / ||f^{K+1}|| in FP64, the last
 * rho1/rho2 and the guarded-bin count.  Synchronises. */
typedef struct {
  int32_t iters;
  int32_t flags;          /* APPGA_FLAG_* sticky device flags */
  int64_t guard_hits;
  double re;              /* relative change of the last map */
  double rho1, rho2;      /* dual step sizes of the last step */
} appga_afppa_stats;
appga_status appga_afppa_reconstruct(appga_ctx* ctx, const appga_matrix* mat, const float* g,
                                     const float* gamma, const float* f_init,
                                     const appga_params* params, float* f_out, float* b_out,
                                     float* c_out, appga_afppa_stats* stats_host, void* stream);

/* ------------------------------------------------------- figures of merit
 * The comparison metrics of Sec. 4.1, for evaluating reconstructions.
 * appga_figures_of_merit: f, f_true: float[d] device images; roi_h, roi_b:
 * uint8[d] device masks of the hot region and the background region (both
 * NULL to skip the contrast figures); max_value: MAX, the largest possible
 * pixel value.  Computes in FP64-accurate arithmetic (double-float sums):
 *   mse  = ||f - f_true||^2 / d,   psnr = 10 log10(MAX^2 / mse),
 *   rc   = |E_H(f) - E_B(f)| / E_B(f) with E the region means,
 *   rc_true the same for f_true,   nrc = rc / rc_true.
 * Contrast fields are NaN when a region is empty or not given.  Allocates a
 * small scratch and synchronises.  EINVAL for d < 1, max_value <= 0, one
 * mask without the other. */
typedef struct {
  double mse, psnr, rc, rc_true, nrc;
  int64_t n_roi_h, n_roi_b;  /* pixels in each region */
} appga_fom;
appga_status appga_figures_of_merit(appga_ctx* ctx, int32_t d, const float* f,
                                    const float* f_true, const uint8_t* roi_h,
                                    const uint8_t* roi_b, double max_value, appga_fom* out_host,
                                    void* stream);
/* NOFV(f^k) = (Phi(f^k) - Phi_ref) / (Phi_0 - Phi_ref), Phi_0 the objective of
 * the initial image and Phi_ref a reference value (Sec. 4.1).  Host function. */
double appga_nofv(double phi_k, double phi_0, double phi_ref);
/* Central line profile: out[c] = f[(n_side/2) * n_side + c], c < n_side (row
 * n_side/2 of the row-major image), device to device on `stream`. */
appga_status appga_central_line_profile(appga_ctx* ctx, int32_t n_side, const float* f,
                                        float* out, void* stream);

/* appga_validate_csr_host: the host-side check appga_matrix_create runs on a
 * CSR (row_ptr[0] = 0, nondecreasing, row_ptr[m] = nnz, 0 <= col < d, values
 * finite and >= 0).  Host only; needs no device.  EINVAL / EDOMAIN with a
 * message from appga_last_error(). */
appga_status appga_validate_csr_host(int32_t m, int32_t d, const int32_t* row_ptr_host,
                                     const int32_t* col_host, const float* val_host);

/* appga_kernel_times: device time of the two phases of an iteration.
 * Sets up a run exactly as appga_reconstruct does (f_init NULL: the initial
 * image), then launches n_iters iterations of (pixel phase, forward phase)
 * back to back on the library stream with CUDA events around every phase,
 * and returns the mean duration of each in milliseconds (the pixel phase is
 * the back-projection/update kernel and its one-block step finalisation).  The
 * iterate ring of the matrix workspace is overwritten.  Synchronises. */
appga_status appga_kernel_times(appga_ctx* ctx, const appga_matrix* mat, const float* g,
                                const float* gamma, const appga_params* params, int32_t n_iters,
                                double* ms_pixel_host, double* ms_forward_host);

#ifdef __cplusplus
}
#endif

#endif /* APPGA_H */
