/*
 * adasap.h -- C-ABI of the B300-native (sm_103a) ADASAP hot path.
 *
 * ADASAP ("Turbocharging Gaussian Process Inference with Approximate
 * Sketch-and-Project", Rathore et al., NeurIPS 2025, Alg. 2) solves
 *
 *     (K(X, X) + lambda I) W = Y,      K_ij = k(x_i, x_j),
 *
 * for a stationary kernel k, by sampling a block B of b rows per iteration,
 * forming the block residual K(X_B, X) W + lambda W_B - Y_B on the fly,
 * preconditioning it with a rank-r randomized Nystrom approximation of K_BB
 * (Alg. 4, App. C.2), choosing the step by randomized powering (Alg. 5) and
 * updating three Nesterov sequences (Alg. 6).
 *
 * Conventions for every entry point below
 *   - Matrices are dense, row-major, float32 unless stated; an (n x s) matrix
 *     has row j at offset j*s.  Index arrays are int64.
 *   - Pointers are CUDA device pointers unless the entry says "host or
 *     device": those are probed with cudaPointerGetAttributes and copied.
 *   - The caller owns every pointer it passes; the context owns its own
 *     device copies and workspaces and frees them in adasap_destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     ordered after everything already queued on it.  adasap_solve* and
 *     adasap_hypergrad return after the work completed (they read results
 *     back); the other calls are asynchronous with respect to the host.
 *   - Every function returns a status and never aborts the process.
 *     Invalid sizes or pointers give ADASAP_EINVAL before any GPU work.
 *   - A context is not thread-safe; use one context per host thread/stream.
 *
 * Kernels (the paper uses them without printing the formulas; standard forms),
 * r = ||x - x'||:
 *   ADASAP_RBF       k = sigma2 * exp(-r^2 / (2 ell^2))
 *   ADASAP_MATERN32  k = sigma2 * (1 + a) exp(-a),           a = sqrt(3) r / ell
 *   ADASAP_MATERN52  k = sigma2 * (1 + a + a^2/3) exp(-a),   a = sqrt(5) r / ell
 */
#ifndef ADASAP_H
#define ADASAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adasap_ctx adasap_ctx;

typedef enum {
  ADASAP_OK = 0,
  ADASAP_EINVAL = 1,        /* invalid argument (shape, range, null pointer) */
  ADASAP_ENOMEM = 2,        /* device allocation failed */
  ADASAP_ECUDA = 3,         /* a CUDA runtime call failed (see adasap_last_error) */
  ADASAP_ENUMERIC = 4,      /* Cholesky of an r x r core failed after retries */
  ADASAP_EDIVERGED = 5,     /* residual became non-finite or exploded */
  ADASAP_ETIMEOUT = 6,      /* a bounded device wait gave up */
  ADASAP_ENOTCONVERGED = 7  /* max_iters reached before tol (W still returned) */
} adasap_status;

typedef enum { ADASAP_RBF = 0, ADASAP_MATERN32 = 1, ADASAP_MATERN52 = 2 } adasap_kernel;

/* Arithmetic of the single-right-hand-side kernel-row products (Step I, the
 * K_BB v products of Alg. 5, predict, residual checks):
 *   ADASAP_PREC_FP32    FP32 CUDA-core distances and epilogue
 *   ADASAP_PREC_TF32X3  distances on the tensor cores (tcgen05, TF32 hi/lo split
 *                       with three products; FP32 epilogue); needs d <= 30.
 * With ADASAP_PREC_TF32X3, products with more than one right-hand side use the
 * multi-RHS tensor-core kernel (W split into TF32 hi/lo as well).
 *   ADASAP_PREC_TF32    as ADASAP_PREC_TF32X3, but the multi-RHS contraction
 *                       K(X_B, X) W takes one MMA on TF32-rounded kernel values
 *                       and W (relative rounding 2^-11 per product: error below
 *                       1e-3 of sum_j |k_ij||w_j|); the low-precision mode of the
 *                       contraction.  Single-RHS products and the sketch keep
 *                       the split arithmetic. */
typedef enum { ADASAP_PREC_FP32 = 0, ADASAP_PREC_TF32X3 = 1, ADASAP_PREC_TF32 = 2 } adasap_precision;

/* Options of adasap_solve.  adasap_default_opts fills the paper's defaults. */
typedef struct {
  int64_t b;           /* block size (Alg. 2); 0 < b <= n.  Default n/100 (App. D.2). */
  int r;               /* Nystrom rank (Alg. 4); 1 <= r <= min(b, 128).  Default 100 (App. D.2). */
  int max_iters;       /* iteration cap T_max (Alg. 2). */
  double tol;          /* stop when the relative residual estimate <= tol (0: never). */
  int power_iters;     /* randomized-powering iterations N of Alg. 5.  Default 10 (App. C.3). */
  double mu, nu;       /* acceleration parameters (Alg. 2); 0 => mu = lambda, nu = n/b (Sec. 4.2). */
  int precond;         /* 0 = Nystrom (ADASAP), 1 = identity (ADASAP-I, Sec. 5), 2 = SAP with the
                          exact block solve (Alg. 1: W_B -= (K_BB + lambda I)^{-1} R_B, no stepsize,
                          no acceleration; b <= 8192; r, mu, nu, power_iters unused). */
  int literal;         /* 0: residual at Z_t and Z_{t+1} from V_{t+1} (standard accelerated
                          sketch-and-project); 1: residual at W_t and Z_{t+1} from V_t, as
                          Alg. 2 / Alg. 6 print. */
  uint64_t seed;       /* Philox4x32-10 key for B, Omega, v0. */
  int check_every;     /* evaluate the residual every this many iterations (0: only at the end). */
  int64_t check_rows;  /* residual on all rows if n <= check_rows, else on this many sampled rows. */
  double eps;          /* eps of Alg. 4's shift Delta = eps * Tr(Omega^T M Omega); 0 => 2^-23. */
  int tail_average;    /* 1: return the tail average (Alg. 1 / 2) mean(W_j, j = ceil(T/2) .. T) of
                          T = max_iters iterations; the run then has exactly T iterations (no
                          tolerance stop, residual taken at the end on the average).  Default 0. */
} adasap_opts;

typedef struct {
  int iters;           /* iterations run */
  double rel_resid;    /* last relative residual ||(K + lambda I) W - Y||_F / ||Y||_F (exact or sampled) */
  int resid_exact;     /* 1 if rel_resid used all n rows */
  double seconds;      /* device time of the iteration loop incl. residual checks (CUDA events) */
  double last_eta;     /* stepsize eta_B of the last iteration */
  double last_rho;     /* damping rho = S_rr + lambda of the last iteration */
  int status_detail;   /* stage of a device-side failure: 1 Nystrom core Cholesky (after 3
                          shift increases), 2 non-finite eigenvalue, 3 Woodbury Cholesky,
                          4 non-positive stepsize estimate, 5 schedule row out of range,
                          6 Cholesky of the test matrix's Gram (thin QR of Omega),
                          7 non-positive pivot of the exact block solve (precond 2) */
} adasap_stats;

void adasap_default_opts(adasap_opts* opts, int64_t n);
const char* adasap_status_string(adasap_status s);
/* Text of the last CUDA error seen by this host thread (empty if none). */
const char* adasap_last_error(void);

/* Create a context for the training inputs X (n x d, host or device).
 * X is centred and scaled by 1/ell into a device copy (the kernel is
 * translation invariant), so the caller may free X afterwards.
 * Requires n >= 1, 1 <= d <= 64, ell > 0, sigma2 > 0, lambda > 0. */
adasap_status adasap_create(const float* X, int64_t n, int d, int kernel, float ell,
                            float sigma2, float lambda, void* stream, adasap_ctx** out);
void adasap_destroy(adasap_ctx* ctx);
/* Select the arithmetic of later calls on this context (default: ADASAP_PREC_TF32X3
 * when d <= 30, else ADASAP_PREC_FP32).  EINVAL if unavailable. */
adasap_status adasap_set_precision(adasap_ctx* ctx, int precision);

/* Block-row kernel product (Alg. 2 Step I; App. C.1 ColDistMatMat as one kernel):
 *   out (b x s) = K(X_B, X) W,  B (b) int64 row indices into X, W (n x s).
 * Rows whose index is outside [0, n) are written as NaN (no fault). */
adasap_status adasap_kernel_rows(adasap_ctx* ctx, const int64_t* B, int64_t b, const float* W,
                                 int s, float* out, void* stream);

/* The product of adasap_kernel_rows for callers that cannot allocate device
 * memory while they run -- for example code inside a memory-pool-less runtime,
 * an allocation-free real-time loop, or a process whose device memory is
 * already fully reserved.  (The paper has no counterpart: this is a service of
 * this library.)  Same arguments and product as adasap_kernel_rows, but the
 * call allocates nothing: its scratch (an int32 copy of B and the per-split
 * partial sums) is a static device array of 8 MiB that every GPU loading this
 * library holds until the process exits.
 *   - Arithmetic: for s = 1, and for any s in ADASAP_PREC_FP32, the same kernel
 *     and result as adasap_kernel_rows.  For s >= 2 in a tensor-core precision
 *     (ADASAP_PREC_TF32X3, ADASAP_PREC_TF32) the product runs in plain FP32 on
 *     the CUDA cores (the multi-RHS tensor-core kernel needs an operand copy of
 *     W that the array does not hold), so the result agrees with
 *     adasap_kernel_rows within that precision's tolerance, not bit for bit.
 *   - The scratch must fit: 4 * b bytes for the index copy plus 4 * b * s * k
 *     for the partials, where k, the number of column splits the library
 *     chooses, GROWS as b shrinks (it aims at a fixed number of work items, so
 *     b * k stays roughly constant): b * k is at most about 1.2e6 on the
 *     tensor-core path (s = 1) and about 2368 * 64 on the CUDA-core path, so
 *     the partials take at most about 4.9 MB for s = 1 and about 0.61 MB per
 *     right-hand side otherwise.  Sizes that do not fit return ADASAP_EINVAL
 *     before any GPU work, and adasap_last_error() gives the bytes needed.
 *   - The context's device must be current, and its index below 64 (the
 *     per-device address table).  The first call on a device looks up the
 *     array's device address (cudaGetSymbolAddress); make that first call
 *     before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents;
 *     nothing in it needs clearing, but calls that overlap on the GPU (on
 *     different streams, or from different threads) race on it: serialise them. */
adasap_status adasap_kernel_rows_noalloc(adasap_ctx* ctx, const int64_t* B, int64_t b, const float* W,
                                         int s, float* out, void* stream);

/* Measurement support (the paper has no counterpart): the issue throughput of
 * the pipes that bound the block-row product on the current device, measured
 * by long independent dependency chains on every SM.  out[0] = ex2.approx,
 * out[1] = rsqrt.approx, out[2] = FP32 FMA, out[3] = sqrt.approx, each in
 * operations per SM per clock cycle; the first `count` (<= 4) are written.
 * Synchronises `stream`. */
adasap_status adasap_measure_pipes(double* out, int count, void* stream);

/* Self-test support (the paper has no counterpart): evaluates, element by
 * element, a device function of the block-row epilogues, so that tests can hold
 * it to its error bound on a dense grid.  fn = 0: the square root computed on the
 * FMA pipe that the Matern epilogues use for a share of their entries (Newton
 * steps from a bit-pattern seed; inputs below 1e-30 are taken as 1e-30, and on
 * [1e-30, 1e21] the result is the correctly rounded square root to within half an
 * ulp); fn = 1: sqrt.approx of the special-function unit.  x and out are device
 * arrays of n floats (they may alias); the call is asynchronous on `stream`.
 * ADASAP_EINVAL for another fn, n < 0, or a NULL array with n > 0. */
adasap_status adasap_eval_math(int fn, const float* x, int64_t n, float* out, void* stream);

/* Device-side failures (the paper has no counterpart).  Every wait inside the
 * tensor-core kernels is bounded in time; a kernel whose wait runs out records a
 * code in its context, writes NaN in place of the affected outputs and returns,
 * leaving the context usable.  adasap_check_device synchronises `stream`,
 * returns ADASAP_ETIMEOUT with *code (may be NULL) the first recorded code, or
 * ADASAP_OK with *code = 0, and clears the record.  The solvers check it at each
 * residual evaluation and return ADASAP_ETIMEOUT.
 * adasap_wait_selftest enqueues, for tests of this path, a one-thread kernel whose
 * bounded wait nothing completes: after limit_ns (<= 10^9) it records code 99 in
 * the context and returns, so that adasap_check_device then reports it. */
adasap_status adasap_check_device(adasap_ctx* ctx, int* code, void* stream);
adasap_status adasap_wait_selftest(adasap_ctx* ctx, uint64_t limit_ns, void* stream);

/* Work schedule of a single-RHS tensor-core block-row product (host only, no
 * device needed; the paper has no counterpart: Step I of Alg. 2 and the K_BB a
 * products of Alg. 5 are split over the CTAs of one GPU).  For an m x ncols
 * product on min(resident CTAs, max_ctas) CTAs (max_ctas <= 0: all) it returns
 * in *nsplit the partial slots per row and in *flat 1 when the launch takes
 * equal tile runs per CTA (else (row tile x column split) items).  For the
 * equal runs it walks every CTA's runs through the kernel's own decoding and
 * returns ADASAP_ENUMERIC if a tile would not be covered exactly once or a
 * (row, slot) not written exactly once; ADASAP_EINVAL for m, ncols < 1 or a
 * NULL pointer. */
adasap_status adasap_schedule_check(int64_t m, int64_t ncols, int max_ctas, int* nsplit, int* flat);

/* ADASAP (Alg. 2 with Alg. 4, 5, 6 and the stabilised Woodbury apply of App. C.2).
 * Y (n x s) and W (n x s) are host or device.  W holds W_0 on entry and the
 * returned iterate W_T on exit.  1 <= s <= 128.  Randomness (B, Omega, v0) is
 * drawn on the device from Philox4x32-10 keyed by opts->seed. */
adasap_status adasap_solve(adasap_ctx* ctx, const float* Y, int s, const adasap_opts* opts,
                           float* W, adasap_stats* stats, void* stream);

/* As adasap_solve, but iteration t < T uses the caller's randomness:
 * B_sched (T x b) int64 distinct rows, Omega_sched (T x b x r), v0_sched (T x b),
 * all device.  Runs exactly T iterations (opts->max_iters and tol are ignored).
 * trace (device, T x 2 float64, may be NULL) receives (eta_t, rho_t). */
adasap_status adasap_solve_scheduled(adasap_ctx* ctx, const float* Y, int s,
                                     const adasap_opts* opts, const int64_t* B_sched,
                                     const float* Omega_sched, const float* v0_sched, int T,
                                     float* W, double* trace, adasap_stats* stats, void* stream);

/* Many independent systems of uneven size solved together (for example the
 * GP models of a Bayesian-optimisation campaign, Sec. 5.3).  System i is
 * ctxs[i] with Y[i] and W[i] (n_i x s, host or device; W[i] holds W_0 on entry
 * and the returned iterate on exit) and its own options opts[i] (Alg. 2 as in
 * adasap_solve; tail_average must be 0, precond 0 or 1, power_iters the same
 * for all).  One CUDA graph holds one iteration of
 * every system still running, each system on its context's streams; the Step I
 * products and the K_BB a products of Alg. 5 of all systems that use the
 * single-right-hand-side tensor-core kernel (s = 1, ADASAP_PREC_TF32X3, Nystrom
 * preconditioner) run as one grouped persistent launch per kernel kind, with a
 * column split chosen before the first iteration by timing candidates.  A
 * system leaves the batch (and the graph is re-captured without it) when a
 * residual check meets opts[i].tol or after opts[i].max_iters iterations.
 * stats (nsys entries, may be NULL) as in adasap_solve, with seconds = device
 * time from the start of the batch until the system left it.  The contexts
 * must be distinct.  Returns the first error of any system, else
 * ADASAP_ENOTCONVERGED if a system with tol > 0 missed it, else ADASAP_OK. */
adasap_status adasap_solve_batched(int nsys, adasap_ctx* const* ctxs, const float* const* Y, int s,
                                   const adasap_opts* opts, float* const* W, adasap_stats* stats, void* stream);

/* Incremental form of adasap_solve (same arithmetic), for callers that step
 * the solver themselves or time it.  One active solver per context: the
 * solver uses the context's streams and device scalars.
 *   begin:    allocate the solver state (W0 host or device, NULL = zeros), copy
 *             Y and W0, and capture one iteration of Alg. 2 as a CUDA graph.
 *   step:     enqueue `iters` iterations on `stream` (no host synchronisation).
 *   residual: ||(K + lambda I) W - Y||_F / ||Y||_F on all rows when
 *             n <= opts->check_rows, else on check_rows rows drawn afresh
 *             (scaled by sqrt(n / check_rows)); synchronises.  Returns the
 *             device status (ENUMERIC / EDIVERGED) if an iteration failed.
 *   get_w:    copy the current iterate W_t (n x s) to W (host or device).
 *   scalars:  eta, rho and the device status of the last iteration (synchronises).
 *   end:      free everything. */
typedef struct adasap_solver adasap_solver;
adasap_status adasap_solver_begin(adasap_ctx* ctx, const float* Y, int s, const adasap_opts* opts,
                                  const float* W0, void* stream, adasap_solver** out);
adasap_status adasap_solver_step(adasap_solver* sol, int iters, void* stream);
adasap_status adasap_solver_residual(adasap_solver* sol, double* rel_resid, void* stream);
adasap_status adasap_solver_get_w(adasap_solver* sol, float* W, void* stream);
adasap_status adasap_solver_scalars(adasap_solver* sol, double* eta, double* rho, int* status, void* stream);
/* Checkpoint and resume of a stepped solve (the paper has no counterpart).
 * Between iterations the whole state of Alg. 2 is (W_t, V_t, Z_t) and t, since
 * the draws B, Omega, v0 of iteration t depend only on opts->seed and t.
 *   get_state: copy W, V, Z (n x s each, host or device) and t; synchronises.
 *   set_state: load them into a solver begun on the same context with the same
 *              Y and options (0 <= t < 2^32); steps then continue the same
 *              trajectory.  Synchronises `stream`. */
adasap_status adasap_solver_get_state(adasap_solver* sol, float* W, float* V, float* Z, int64_t* t, void* stream);
adasap_status adasap_solver_set_state(adasap_solver* sol, const float* W, const float* V, const float* Z, int64_t t,
                                      void* stream);
void adasap_solver_end(adasap_solver* sol);
/* Diagnostics of the last iteration (synchronises): out[0..9] = Delta, rho, eta,
 * lambda_hat, Cholesky shift increases, Jacobi sweeps, status, status detail,
 * iteration counter, and the code of the first bounded wait of a tensor-core
 * kernel that timed out in this context (0: none; its outputs are then NaN);
 * the first `count` are written. */
adasap_status adasap_solver_diag(adasap_solver* sol, double* out, int count, void* stream);
/* Number of kernel launches in one captured iteration (for launch accounting). */
adasap_status adasap_solver_graph_kernels(adasap_solver* sol, int* count);

/* Posterior mean with zero prior mean (Sec. 2, eq. post_eqns):
 *   out (m x s) = K(Xtest, X) W,  Xtest (m x d) device, W (n x s) device. */
adasap_status adasap_predict(adasap_ctx* ctx, const float* Xtest, int64_t m, const float* W, int s,
                             float* out, void* stream);

/* Exact relative residual of any W on all n rows (the convergence measure; its
 * Step I-style products over row chunks of 65,536):
 *   *rel = ||(K + lambda I) W - Y||_F / ||Y||_F,  Y and W (n x s) host or device.
 * Synchronises `stream`. */
adasap_status adasap_residual(adasap_ctx* ctx, const float* Y, const float* W, int s, double* rel,
                              void* stream);

/* Random-feature prior draws for pathwise conditioning (Sec. 2.1; Rahimi & Recht
 * features, q = 2048 in the paper's runs, App. D.3):
 *   F[i][j] = sqrt(2 sigma2 / q) * sum_l theta[l][j] cos(omega_l . x_i + phase_l),
 *   omega_l = z_l / ell (RBF) or z_l * sqrt(2 nu / u_l) / ell (Matern-nu, nu = 3/2, 5/2),
 * so that E[F[i][j] F[i'][j]] = k(x_i, x_i').  The caller draws the randomness:
 * z (q x d) ~ N(0, 1), u (q) ~ chi^2(2 nu) (ignored for RBF, may be NULL then),
 * phase (q) ~ U[0, 2 pi), theta (q x s) ~ N(0, 1).  Xq (m x d) raw points;
 * F (m x s).  All device.  Synchronises `stream`. */
adasap_status adasap_rf_prior(adasap_ctx* ctx, const float* Xq, int64_t m, const float* z, const float* u,
                              const float* phase, const float* theta, int q, int s, float* F, void* stream);

/* Posterior samples by pathwise conditioning (Sec. 2.1, eq. pathwise_conditoning,
 * with the prior cross-covariance k(X*, X) in front of the solve):
 *   f_n(X*)_j = f_j(X*) + k(X*, X) W_j,  W_j = (K + lambda I)^{-1} (y - f_j(X) - zeta_j),
 * for ns samples j, f_j the random-feature draws of adasap_rf_prior (z, u, phase,
 * theta (q x ns)) and zeta (n x ns) ~ N(0, lambda I) drawn by the caller.  All
 * ns (+ 1) systems are one ADASAP solve with opts (adasap_solve).  With
 * with_mean = 1 column 0 of W and out is the posterior mean (right-hand side y,
 * no prior draw) and the samples are columns 1..ns.  y (n), Xtest (m x d), out
 * (m x (ns + with_mean)), W (n x (ns + with_mean), W_0 on entry) all device.
 * Returns the solve's status (ADASAP_ENOTCONVERGED keeps W and out valid). */
adasap_status adasap_pathwise(adasap_ctx* ctx, const float* y, const float* Xtest, int64_t m, const float* z,
                              const float* u, const float* phase, const float* theta, int q, const float* zeta,
                              int ns, int with_mean, const adasap_opts* opts, float* out, float* W,
                              adasap_stats* stats, void* stream);

/* Test metrics of Sec. 5.1 (the paper reports them without formulas): RMSE of
 * the posterior mean, and the mean NLL of ytest under N(mean_i, var_i + noise)
 * with var_i the sample variance (divisor s - 1) of the s samples at point i.
 * mean (row stride ld_mean), samples (m x s, row stride ld_samples), ytest (m)
 * device; FP64 sums.  s >= 2.  Synchronises `stream`. */
adasap_status adasap_rmse_nll(const float* mean, int64_t ld_mean, const float* samples, int64_t ld_samples, int s,
                              const float* ytest, int64_t m, double noise, double* rmse, double* nll, void* stream);

/* Kernel adjoint for hyperparameter fitting (App. D.1):
 *   d_ell    = sum_c G[:,c]^T (dK/dell)    W[:,c]
 *   d_sigma2 = sum_c G[:,c]^T (dK/dsigma2) W[:,c]
 * over the full n x n kernel, recomputing tiles.  W, G (n x s) device;
 * d_ell, d_sigma2 host.  With W = G = (K + lambda I)^{-1} y this gives
 * -d(y^T (K + lambda I)^{-1} y)/dtheta. */
adasap_status adasap_hypergrad(adasap_ctx* ctx, const float* W, const float* G, int s,
                               double* d_ell, double* d_sigma2, void* stream);

/* The device sampler of adasap_solve at iteration t (for tests and for
 * callers that want the same randomness): B (b) int64 distinct rows of [n],
 * Omega (b x r) with N(0, 1/b) entries, v0 (b) N(0, 1); any output may be NULL.
 * Definitions: Philox4x32-10 (Salmon et al., SC'11) keyed by seed, a 4-round
 * Feistel permutation of [n] with cycle walking for B, Box-Muller normals. */
adasap_status adasap_sample(uint64_t seed, int64_t t, int64_t n, int64_t b, int r, int64_t* B,
                            float* Omega, float* v0, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ADASAP_H */
