/*
 * ssnal_en.h -- C ABI of the GB300 (sm_103a) SsNAL-EN hot path.
 *
 * SsNAL-EN (Boschi, Reimherr, Chiaromonte, arXiv 2006.03970) solves the
 * Elastic Net
 *
 *     min_x  1/2 ||A x - b||^2 + lambda1 ||x||_1 + lambda2/2 ||x||^2      (Sec. 1)
 *
 * with an augmented Lagrangian method on the dual (Algorithm 1, upper half)
 * whose inner problem is solved by a semi-smooth Newton method
 * (Algorithm 1, lower half; Prop. 2; eqs. grad_phy, Q_def, AJ_system,
 * smw_formula, line_search) and stopped by the KKT residuals of eq. kkt_res.
 *
 * Conventions common to every entry point
 *  - A is m x n, column-major: column j starts at element j*lda.  lda >= m and
 *    lda * element size must be a multiple of 16 bytes.  Elements in rows
 *    m..lda-1 are never used (they may hold anything, NaN included).
 *  - Pointers documented "device" are CUDA device pointers owned by the caller;
 *    the library never frees them.  A must stay alive and unchanged until
 *    ssnal_en_destroy.  Pointers documented "host" are ordinary host memory.
 *  - All device work is enqueued on the stream given to ssnal_en_create.  The
 *    solve / path / op entry points return after that work has completed
 *    (they synchronise the stream), so their outputs are ready on return.
 *  - No C++ exception crosses this boundary; every call returns a status.
 *  - A context is not thread-safe: use one context per host thread / stream.
 *  - Floating-point work of the solve path is FP64 except where the options
 *    select the mixed path (see ssnal_en_options.precision).
 */
#ifndef SSNAL_EN_H
#define SSNAL_EN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssnal_en_ctx ssnal_en_ctx; /* opaque: owns the device workspaces */

/* Storage type of A. */
typedef enum {
  SSNAL_EN_F64 = 0,      /* double */
  SSNAL_EN_F32 = 1,      /* float */
  SSNAL_EN_BF16 = 2,     /* bfloat16 bit patterns (uint16) */
  SSNAL_EN_I8_GENO = 3,  /* int8 codes; entry = (code - col_mean[j]) * col_scale[j], evaluated in FP64
                            from the FP32 mean and scale (standardization applied on the fly) */
  SSNAL_EN_I2_GENO = 4   /* 2-bit genotype codes 0..3, four per byte: row i of column j is bits
                            2 (i mod 4) and 2 (i mod 4) + 1 of byte (j lda + i) / 4; lda counts codes
                            and must be a multiple of 64 (a column stride of whole 16-byte units);
                            entries as for I8_GENO */
} ssnal_en_dtype;

typedef enum {
  SSNAL_EN_OK = 0,
  SSNAL_EN_EINVAL = 1,    /* bad argument: sizes, lda, null pointer, negative or non-finite lambda */
  SSNAL_EN_ENOMEM = 2,    /* a device workspace could not be allocated */
  SSNAL_EN_ENOCONV = 3,   /* iteration caps reached; the best iterate is still returned */
  SSNAL_EN_ECUDA = 4,     /* a CUDA runtime call failed */
  SSNAL_EN_ETIMEOUT = 5,  /* reserved for bounded device-side waits */
  SSNAL_EN_ENOTSUP = 6    /* valid but unsupported request (e.g. m above the supported maximum) */
} ssnal_en_status;

/* The design matrix handed to ssnal_en_create (borrowed, never copied). */
typedef struct {
  int64_t m, n, lda;       /* rows (observations), columns (features), leading dimension in elements */
  int32_t dtype;           /* ssnal_en_dtype */
  int32_t reserved;
  const void* data;        /* device, column-major, see the conventions above */
  const float* col_mean;   /* I8_GENO only: device, length n */
  const float* col_scale;  /* I8_GENO only: device, length n */
} ssnal_en_matrix;

/* Solver options.  ssnal_en_default_options fills the paper's settings. */
typedef struct {
  double sigma0;        /* 5e-3: initial AL penalty (Sec. 4.1) */
  double sigma_growth;  /* 5: sigma multiplied by this after every AL iteration (Sec. 4.1) */
  double sigma_max;     /* 1e8: cap of the increasing sigma sequence (Algorithm 1 step (2)) */
  double mu;            /* 0.2: Armijo constant in (0, 1/2) (eq. line_search, Sec. 4.1) */
  double beta;          /* 0.5: backtracking factor, trial steps 1, beta, beta^2, ... */
  double tol;           /* 1e-6: tolerance on res(kkt1) and res(kkt3) (eq. kkt_res) */
  int32_t max_al;       /* 100: AL iterations */
  int32_t max_newton;   /* 50: SsN iterations per AL iteration */
  int32_t max_ls;       /* 40: line-search trials per SsN iteration, at most 64 */
  int32_t precision;    /* 0: FP64 results; the pass over A uses float-float arithmetic on the FP32 pipe
                           (about 2^-47 relative per product) when every entry of A is 0 or has
                           magnitude in [2^-100, 2^100], else FP64 FMAs.  For this the context
                           keeps a float-pair copy of A (same size as A) made at create time.
                           3: as 0 but without the copy (entries split on the fly, slower).
                           2: FP64 FMAs always.
                           1: mixed precision, for A stored as BF16, FP32 or I8_GENO: the Newton-step passes
                           t = A^T d sum the products in FP32; u = A^T y is recomputed in
                           float-float before every SsN stopping test, so the KKT test, the
                           x update and the duality gap use FP64-accurate values.
                           With BF16 / FP32 / I8_GENO storage and precision 0, 2 or 3 every pass over A
                           is float-float (products of the stored values are exact). */
  int32_t refine_steps; /* 1: iterative-refinement steps of the Newton solve (FP64 residual through
                           the packed A_J, FP32 factor).  The first correction also measures the
                           FP32 solve's relative error: above 1e-2 (the refinement would not
                           contract) the Newton step is redone with the FP64 system, see newton_fp64 */
  int32_t use_y0;       /* 0: y0 = A x0 - b; 1: take y0 from the y argument of ssnal_en_solve */
  int32_t ls_fused;     /* 16: trial steps evaluated inside the A^T d pass (1..16); later trials
                           are evaluated by a pass over the stored n-vectors only */
  int32_t syrk_tc;      /* 1: Newton-matrix SYRK on the tensor cores (tcgen05, BF16 operands, FP32
                           accumulation; FP64 panels as a three-way BF16 split); 0: FP32 FMA */
  int64_t max_active;   /* 0: path stops after the first point with at least this many nonzeros (0 = never) */
  int32_t newton_fp64;  /* Newton system of eqs. AJ_system / smw_formula:
                           0: formed and factored in FP32 with FP64 refinement; when that factor meets
                              a non-positive pivot or its refinement does not contract, the step is not
                              taken and its direction is recomputed with the Newton matrix formed,
                              factored (Cholesky) and solved in FP64, and the rest of that fit stays
                              on the FP64 system;
                           1: always the FP64 system */
  int32_t cg_maxit;     /* 0: CG iterations per Newton solve at most 10 m (see cg_above) */
  int64_t cg_above;     /* 10000: the Newton system is solved by conjugate gradients (matrix-free,
                           V p = p + kappa A_J (A_J^T p)) when m and r both exceed this (Algorithm 1
                           step (1), Sec. 3.2); 0 < cg_above < 10000 moves the switch */
  double cg_rtol;       /* 1e-10: CG stops at ||V d + g|| <= cg_rtol ||g|| (the paper gives no tolerance) */
} ssnal_en_options;

/* Per-fit report. */
typedef struct {
  int32_t status;        /* ssnal_en_status of this fit */
  int32_t al_iters;      /* AL iterations performed */
  int32_t newton_iters;  /* Newton directions computed (all AL iterations) */
  int32_t ls_trials;     /* line-search trials (all Newton iterations) */
  int64_t active;        /* nonzeros of the returned x */
  double kkt1;           /* ||y + b - A x|| / (1 + ||b||)            (eq. kkt_res) */
  double kkt3;           /* ||A^T y + z|| / (1 + ||y|| + ||z||)      (eq. kkt_res) */
  double primal_obj;     /* 1/2||Ax-b||^2 + lambda1||x||_1 + lambda2/2||x||^2 */
  double dual_gap;       /* primal_obj - D(y), D(y) = -h*(y) - p*(-A^T y) (lambda2 > 0) */
  double seconds;        /* wall time of the fit on the host clock */
  double sigma;          /* sigma of the last AL iteration */
  double lambda1, lambda2;
  int32_t newton_fp64;   /* Newton directions computed with the FP64 system (see ssnal_en_options) */
  int32_t cg_iters;      /* conjugate-gradient iterations (all Newton solves) */
} ssnal_en_result;

/* Fills *opts with the defaults listed above. */
void ssnal_en_default_options(ssnal_en_options* opts);

/* Human-readable name of a status code (static string). */
const char* ssnal_en_status_string(int32_t status);

/* Creates a context for the matrix *A.  opts may be NULL (defaults).  stream is
 * a cudaStream_t (NULL = the legacy default stream).  Allocates the device
 * workspaces (vectors of length n and m, the A_J panel, the Newton matrix).
 * F64 storage is copied once into a float-pair form for the stream (precision 0,
 * see ssnal_en_options); F32, BF16 and I8_GENO storage is streamed in place
 * (I8_GENO needs col_mean and col_scale; lda * element size a multiple of 16).
 * Errors: EINVAL (null pointers, m <= 0, n <= 0, lda < m, misaligned lda or
 * data, unknown dtype, I8_GENO without mean/scale), ENOTSUP (m above 4096), ENOMEM,
 * ECUDA. */
ssnal_en_status ssnal_en_create(ssnal_en_ctx** ctx, const ssnal_en_matrix* A,
                                const ssnal_en_options* opts, void* stream);

/* Releases the context's workspaces (never the caller's A). NULL is a no-op. */
void ssnal_en_destroy(ssnal_en_ctx* ctx);

/* Replaces the options of an existing context (NULL restores the defaults). */
ssnal_en_status ssnal_en_set_options(ssnal_en_ctx* ctx, const ssnal_en_options* opts);

/* One SsNAL-EN fit (Algorithm 1).
 *  b   device, length m (FP64).
 *  x   device, length n (FP64): on entry the warm start x0 (zeros for a cold
 *      start), on return the solution.
 *  y   device, length m (FP64) or NULL: on entry y0 when opts.use_y0 = 1, on
 *      return the final dual iterate.
 *  out host, may be NULL.
 * Returns OK, ENOCONV (caps reached; x, y and *out hold the last iterate), or an
 * error (EINVAL for lambda1 < 0, lambda2 < 0 or non-finite lambdas). */
ssnal_en_status ssnal_en_solve(ssnal_en_ctx* ctx, const double* b, double lambda1, double lambda2,
                               double* x, double* y, ssnal_en_result* out);

/* Warm-started regularization path (Sec. 3.3).  lambda1_k = c_k ||A^T b||_inf,
 * lambda2_k = (1 - alpha)/alpha * c_k ||A^T b||_inf (the parameterisation of
 * Sec. 4.1 with lambda_max = ||A^T b||_inf / alpha), alpha in (0, 1].
 *  b      device, length m.
 *  c_grid host, K values, visited in the given order (descending for warm starts).
 *  X      device, n x K column-major (column k = solution at c_k), or NULL.
 *  out    host, K results (may be NULL).  Points after an early stop
 *         (opts.max_active) get status EINVAL-free zeros and al_iters = 0.
 *  n_done host, may be NULL: number of grid points solved.
 * Each point starts from the previous solution (x0 = x_{k-1}, y0 = A x0 - b) and
 * restarts sigma at sigma0. */
ssnal_en_status ssnal_en_path(ssnal_en_ctx* ctx, const double* b, double alpha, const double* c_grid,
                              int32_t K, double* X, ssnal_en_result* out, int32_t* n_done);

/* Same as ssnal_en_path with b, X in HOST memory (X may be NULL): the library
 * copies b to the device and the solutions back inside the call. */
ssnal_en_status ssnal_en_path_host(ssnal_en_ctx* ctx, const double* b_host, double alpha,
                                   const double* c_grid, int32_t K, double* X_host,
                                   ssnal_en_result* out, int32_t* n_done);

/* Kernel accounting of this context.  When enabled, CUDA events are recorded on
 * the context's stream around launches of the A^T d stream (the one pass over A
 * of each Newton step, eq. line_search fused in) and their elapsed times are
 * summed as they complete.
 *  enable  1: record around every eighth launch from now on (the first, the
 *          ninth, ...: a recorded launch loses its overlap with the kernels
 *          beside it, so level 1 keeps that cost to one launch in eight), and
 *          around every u = A^T y pass (phase 4 of ssnal_en_profile_phases),
 *          2: record around every launch and also the phases of
 *          ssnal_en_profile_phases (more events on the host's path between
 *          kernels), 0: stop recording.
 *  reset   1: zero the sums before reporting.
 *  stream_ms        summed device time of the recorded launches (host, may be NULL)
 *  stream_launches  number of the recorded launches (host, may be NULL)
 *  stream_bytes     algorithmic bytes of the recorded launches: A once (m*n*elem) plus
 *                   the vectors d (read), x, u (read) and t (written)
 *  kernel_launches  kernels launched by this library in this process so far
 * Synchronises the stream.  Errors: EINVAL (null ctx), ECUDA. */
ssnal_en_status ssnal_en_profile(ssnal_en_ctx* ctx, int32_t enable, int32_t reset, double* stream_ms,
                                 int64_t* stream_launches, double* stream_bytes, int64_t* kernel_launches);

/* Per-phase device time since the last ssnal_en_profile(reset = 1), recorded
 * while profiling is enabled at level 2 (level 1 records one launch in eight of
 * phase 2 and every launch of phase 4 only).  Five phases, in this order:
 *  0 prox + active set + gather + gradient (eqs. prox_elastic, Q_def, grad_phy)
 *  1 Newton direction: SYRK, Cholesky, solves and refinement, or the CG iterations
 *    (eqs. AJ_system, smw_formula)
 *  2 the pass over A with the fused line search (eq. line_search)
 *  3 the multiplier update x <- prox(x - sigma A^T y) (eq. update_x)
 *  4 the passes u = A^T y at the start of a fit and before SsN stopping tests of the
 *    mixed precision mode (float-float over the stored values; Prop. 2)
 * phase_ms, phase_count: host arrays of SSNAL_EN_PROFILE_PHASES (either may be
 * NULL).  Time on the stream outside these phases (host round trips) is not
 * attributed.
 * Synchronises the stream.  Errors: EINVAL (null ctx), ECUDA. */
#define SSNAL_EN_PROFILE_PHASES 5
ssnal_en_status ssnal_en_profile_phases(ssnal_en_ctx* ctx, double* phase_ms, int64_t* phase_count);

/* ---------------------------------------------------------------------------
 * Parameter tuning along a path (Sec. 3.3, eq. gcv_bic).
 * ------------------------------------------------------------------------- */

/* Criteria of one solution x of the path, J its active set, r = |J|:
 *   nu   = tr(A_J (A_J^T A_J + lambda2 I)^{-1} A_J^T)  (EN degrees of freedom),
 *   rss  = ||b - A_J x_ols||^2, x_ols the least-squares fit on J (de-biasing),
 *   gcv  = rss / m / (1 - nu / m)^2,   ebic = log(rss / m) + (nu / m)(log m + log n). */
typedef struct {
  double nu, rss, gcv, ebic;
  int64_t active;
} ssnal_en_tune_point;

/* Runs ssnal_en_path (same arguments; X is required here) and evaluates the
 * criteria at each computed point: nu from the Cholesky factor of the r x r (or
 * m x m when r > m) matrix as min(r, m) - lambda2 tr(G^{-1}), rss through the
 * SMW Newton solve with kappa = infinity (r < m; rss = 0 when r >= m).
 * tr(G^{-1}) = ||L^{-1}||_F^2 from the FP32 factor (any min(r, m) <= 4096).  nu is
 * NaN when G is not positive definite in FP32, rss is NaN when the least-squares
 * normal matrix is not positive definite in FP32 nor in FP64.
 * crit: host array of K.  best_gcv / best_ebic (host, may be NULL): index of the
 * smallest finite criterion, or -1.  Errors: as ssnal_en_path. */
ssnal_en_status ssnal_en_tune(ssnal_en_ctx* ctx, const double* b, double alpha, const double* c_grid, int32_t K,
                              double* X, ssnal_en_result* out, ssnal_en_tune_point* crit, int32_t* best_gcv,
                              int32_t* best_ebic, int32_t* n_done);

/* ---------------------------------------------------------------------------
 * Many independent fits at once (Algorithm 1 per instance).
 * ------------------------------------------------------------------------- */

/* One fit of a batch: the context of its matrix, its right-hand side and its
 * penalties, as for ssnal_en_solve. */
typedef struct {
  ssnal_en_ctx* ctx;  /* borrowed; every instance of a batch has its own context */
  const double* b;    /* device, length m of ctx */
  double lambda1, lambda2;
  double* x;          /* device, length n of ctx: in = warm start, out = solution */
  double* y;          /* device, length m, or NULL */
} ssnal_en_instance;

/* Solves count independent instances concurrently: `workers` host threads, each
 * with its own CUDA stream, take instances in index order from a shared queue
 * and run ssnal_en_solve on them, so small fits overlap on the device.
 * workers = 0 tunes the thread count on the batch itself (4, 8, 16 or 32, by the
 * m*n processed per second on successive chunks).  Each instance's result equals
 * that of ssnal_en_solve on its own.  The device is synchronised on entry; all
 * outputs are complete on return.  out: host array of count results (each with
 * its own status); workers_used (host, may be NULL) receives the thread count.
 * Returns OK when every instance converged, else the first non-OK status.
 * Errors: EINVAL (null pointers, bad lambdas, a context used twice), ECUDA. */
ssnal_en_status ssnal_en_solve_batch(ssnal_en_instance* inst, int64_t count, int32_t workers,
                                     ssnal_en_result* out, int32_t* workers_used);

/* Solves count independent fits whose contexts share one matrix (created from the same
 * ssnal_en_matrix: same data, sizes and type; every instance has its own context),
 * advancing them together one Newton step at a time so that the passes over A of all
 * fits that need one are merged: one pass forms A^T [d_1 ... d_k] for up to 4 fits, each
 * with its own fused line search (eq. line_search).  Merging applies to the passes that
 * accumulate in FP32 (precision 1 with BF16, FP32 or genotype storage); otherwise the
 * fits take one pass each.  Each fit's kernels are those of ssnal_en_solve, so its
 * result is bitwise that of ssnal_en_solve on its own.  All work runs on the first
 * instance's context stream.  out: host array of count results (may be NULL);
 * passes (host, may be NULL): the passes over A of the Newton steps.  Returns OK when
 * every fit converged, else the first non-OK status.  Errors: EINVAL (null pointers,
 * bad lambdas, a context used twice), ECUDA. */
ssnal_en_status ssnal_en_solve_shared(ssnal_en_instance* inst, int32_t count, ssnal_en_result* out,
                                      int32_t* passes);

/* One fit of a device-resident batch: A stored as FP32. */
typedef struct {
  const float* A;          /* device, column-major m x n, column j at A + j*lda */
  int64_t m, n, lda;       /* m <= 1024, lda >= m */
  const double* b;         /* device, length m */
  double lambda1, lambda2;
  double* x;               /* device, length n: in = warm start, out = solution */
} ssnal_en_batch_fit;

/* Solves count independent fits in one launch of a persistent kernel (Algorithm 1 per
 * fit, entirely on the device): one CTA per SM takes the next fit from a device work
 * queue (the fits ordered by m*n, largest first) and runs its whole AL / SsN loop --
 * prox and active set, gradient, Newton matrix (FP32, read from A's columns through J)
 * with its Cholesky factor, triangular solves and one FP64 refinement step, the
 * float-float passes over A, the line search, the multiplier update and the KKT test
 * -- then takes the next.  The loads in flight of the passes over A are tuned on the
 * batch (three slices of the order with 4, 8 and 16 per lane; the rest with the fastest);
 * the choice changes no sum's order, so the results do not depend on it.  A fit whose
 * FP32 Newton solve fails or does not contract is solved again by ssnal_en_solve on a
 * temporary context (FP64 Newton system) from its warm start.  opts: NULL = defaults
 * (precision, syrk_tc, cg and ls_fused do not apply).  Device scratch of about
 * 5 n_max + 9 m_max doubles and m_max^2 floats per SM is allocated and freed inside the
 * call.  out: host array of count results; info (host, may be NULL): [loads in flight
 * chosen, fits solved again on the regular path].  Synchronises `stream`.  Returns OK
 * when every fit converged, else the first non-OK status.
 * Errors: EINVAL, ENOTSUP (m above 1024), ENOMEM, ECUDA. */
ssnal_en_status ssnal_en_solve_batch_resident(const ssnal_en_batch_fit* fits, int64_t count,
                                              const ssnal_en_options* opts, ssnal_en_result* out, int32_t* info,
                                              void* stream);

/* ---------------------------------------------------------------------------
 * Serving: resident matrices, requests admitted while others run.
 * ------------------------------------------------------------------------- */

typedef struct ssnal_en_server ssnal_en_server; /* opaque */

/* Starts a server over nmat resident matrices (descriptors copied; the device
 * data stays owned by the caller and must outlive the server) with `workers`
 * worker threads, each with its own CUDA stream.  A free worker takes the oldest
 * queued request and the queued requests on the same matrix (up to the group
 * size, ssnal_en_server_set_group) and advances their fits together, one Newton
 * step at a time, with their passes over A merged (A^T [d_1 ... d_k], as in
 * ssnal_en_solve_shared); requests on that matrix that arrive meanwhile join the
 * group as its fits finish.  A worker creates contexts per matrix (options opts,
 * NULL = defaults) and keeps them for later requests on that matrix, releasing
 * the panel of a large active set after each request.  Requests are admitted as
 * workers and group places free up and while the estimated device bytes of the
 * contexts in use stay within max_bytes (0 = no bound; one request is always
 * admitted).  A request that runs out of device memory is run once more after
 * its worker releases its contexts of other matrices.  FP64
 * matrices get a float-pair copy per worker context (see ssnal_en_create); the
 * other storage types are read in place.  Errors: EINVAL, ENOMEM, ECUDA. */
ssnal_en_status ssnal_en_server_create(ssnal_en_server** srv, const ssnal_en_matrix* mats, int32_t nmat,
                                       const ssnal_en_options* opts, int32_t workers, int64_t max_bytes);

/* Requests on one matrix that a worker advances together, their passes over A
 * merged (see ssnal_en_solve_shared): 1 (no merging) .. 64, default 8.  Applies to
 * groups formed after the call.  Errors: EINVAL. */
ssnal_en_status ssnal_en_server_set_group(ssnal_en_server* srv, int32_t max_group);

/* Queues one fit on matrix `mat` (eq. EN_pb with penalties lambda1, lambda2,
 * started from x = 0): b_host is host memory of length m, copied before
 * return.  *ticket identifies the request.  Errors: EINVAL. */
ssnal_en_status ssnal_en_server_submit(ssnal_en_server* srv, int32_t mat, const double* b_host, double lambda1,
                                       double lambda2, int64_t* ticket);

/* As ssnal_en_server_submit with the penalties of the paper's experiments
 * (Sec. 4.1): lambda1 = c ||A^T b||_inf and lambda2 = (1 - alpha)/alpha * c ||A^T b||_inf,
 * ||A^T b||_inf computed on the device at the start of the solve.  alpha in
 * (0, 1], c >= 0.  Errors: EINVAL. */
ssnal_en_status ssnal_en_server_submit_scaled(ssnal_en_server* srv, int32_t mat, const double* b_host, double alpha,
                                              double c, int64_t* ticket);

/* Result of a request: with wait != 0 blocks until it is done.  When done,
 * *done = 1, x_host (host, length n, may be NULL) receives the solution, *out
 * (may be NULL) the result (its status is the solve's), times (host, 3, may be
 * NULL) the seconds since server start at submission, start and completion, and
 * the ticket is released.  Errors: EINVAL (unknown ticket). */
ssnal_en_status ssnal_en_server_poll(ssnal_en_server* srv, int64_t ticket, int32_t wait, double* x_host,
                                     ssnal_en_result* out, double* times, int32_t* done);

/* Stops the workers after their current solves (queued requests are dropped)
 * and frees the server's contexts.  NULL is a no-op. */
void ssnal_en_server_destroy(ssnal_en_server* srv);

/* ---------------------------------------------------------------------------
 * Single steps of the hot path, exposed for tests and for callers that build
 * their own loops.  Each runs the same kernels the solver uses.
 * ------------------------------------------------------------------------- */

/* u = A^T y (the dual-to-primal stream, needed by Prop. 2 and eq. Q_def).
 * y device length m (FP64), u device length n (FP64). */
ssnal_en_status ssnal_en_op_at_y(ssnal_en_ctx* ctx, const double* y, double* u);

/* t = A^T d accumulated as in the solver's Newton steps (the pass of Algorithm 1
 * that feeds the line search of eq. line_search): in the mixed precision mode
 * (precision = 1 with BF16, FP32 or I8_GENO storage) the products are summed in FP32,
 * otherwise exactly as ssnal_en_op_at_y.  d device length m (FP64), t device
 * length n (FP64).  Errors: EINVAL (null pointer), ECUDA. */
ssnal_en_status ssnal_en_op_at_d(ssnal_en_ctx* ctx, const double* d, double* t);

/* Prox and active set (eqs. prox_elastic, Q_def): v = x - sigma*u,
 * J = { j : |v_j| > sigma*lambda1 } in ascending order, w_J = prox_{sigma p}(v)_J.
 * x, u device length n; J device int32 (capacity n); wJ device (capacity n);
 * r host: |J|. */
ssnal_en_status ssnal_en_op_prox_active(ssnal_en_ctx* ctx, const double* x, const double* u,
                                        double sigma, double lambda1, double lambda2,
                                        int32_t* J, double* wJ, int64_t* r);

/* Gradient of psi (eq. grad_phy) restricted to J: g = y + b - A_J w_J, with the
 * gather of A_J into the context's packed panel.  J device int32 (r entries),
 * wJ device (r), y, b, g device length m. */
ssnal_en_status ssnal_en_op_grad(ssnal_en_ctx* ctx, const int32_t* J, const double* wJ, int64_t r,
                                 const double* y, const double* b, double* g);

/* Newton direction (eqs. AJ_system, smw_formula): solves
 * (I_m + kappa A_J A_J^T) d = -g on the panel gathered by the preceding
 * ssnal_en_op_grad call (same J, r).  g, d device length m. */
ssnal_en_status ssnal_en_op_newton(ssnal_en_ctx* ctx, int64_t r, double kappa, const double* g, double* d);

/* ---------------------------------------------------------------------------
 * Allocation-free prox / active-set step.  The paper has no counterpart to this
 * entry point; it exists for callers that cannot allocate device memory, for
 * example code that runs while another component owns the device memory budget
 * through its own pool, latency-critical loops where cudaMalloc / cudaFree (and
 * the device synchronisation they can cause) are not acceptable, or plug-in
 * code that may only touch the buffers it is handed.
 *
 * Computes what ssnal_en_op_prox_active computes, without a context:
 *  x, u    device, length n (FP64)
 *  J, wJ   device outputs, capacity n: J ascending (int32), wJ the prox values (FP64)
 *  r       host output: |J|
 *  stream  cudaStream_t to run on (NULL = legacy default stream).
 * The call is synchronous: it copies r to the host and synchronises `stream`
 * before returning, so it must not be called while `stream` is being captured
 * into a CUDA graph.  x, u, J and wJ must live on the current device.
 * Its scratch memory is one fixed array in the library's device code (about
 * 66 KB, kept by every GPU that loads the library until the process exits):
 *  - n above SSNAL_EN_STATIC_MAX_N is rejected with ENOTSUP before any device work;
 *  - the first call on a device looks up the array's device address once
 *    (cudaGetSymbolAddress with that device current) and caches it;
 *  - all calls on a device share the array and it keeps the last call's
 *    contents; each call clears what must start at zero, and calls whose GPU
 *    work overlaps (several streams or host threads) race, so the caller must
 *    serialise them.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 * Errors: EINVAL (null pointer, n <= 0, sigma <= 0, negative or non-finite
 * lambda), ENOTSUP (n too large, device index >= 64), ECUDA. */
#define SSNAL_EN_STATIC_MAX_N 2097152
ssnal_en_status ssnal_en_prox_active_static(const double* x, const double* u, int64_t n, double sigma,
                                            double lambda1, double lambda2, int32_t* J, double* wJ, int64_t* r,
                                            void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SSNAL_EN_H */
