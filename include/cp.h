/*
 * cp.h -- C ABI of the GB300 (sm_103a) library for rank-R canonical (CP)
 * tensor approximation by N-GMRES-accelerated ALS (De Sterck, "A Nonlinear
 * GMRES Optimization Algorithm for Canonical Tensor Decomposition").
 *
 * Problem (Optimization Problem I, Section 1, Eq. fA): given a tensor T of
 * size I_1 x ... x I_N, find factor matrices A^(n) (I_n x R) minimising
 *     f = 1/2 || T - [[A^(1), ..., A^(N)]] ||_F^2 .
 *
 * Conventions shared by every call
 * --------------------------------
 *  Iterate layout.  An iterate u is one FP64 vector of P = R * sum_n I_n
 *    entries holding A^(1), ..., A^(N) back to back, each row-major I_n x R
 *    (the R values of a row are contiguous).  Gradients use the same layout.
 *  Dense tensors.  Row-major with the LAST index fastest.
 *  Ownership.  Every array argument belongs to the caller and is only read or
 *    written during the call (or, for asynchronous calls, by work enqueued on
 *    the context stream).  The library never frees caller memory.  Handles
 *    own their internal copies and workspace.
 *  Pointers.  Unless stated otherwise, array arguments are DEVICE pointers
 *    on the context's device.  Calls marked "host or device" accept either;
 *    the library inspects the pointer.
 *  Streams.  Work is enqueued on the context stream.  Calls whose outputs are
 *    device arrays return without synchronising; calls with host outputs
 *    synchronise the stream before returning.
 *  Errors.  Every call returns a cp_status; nothing is thrown across the ABI.
 *    cp_last_error() gives a message for the calling thread's last failure.
 *    Arguments are validated before any work is enqueued.
 *  Threads.  A context may be used by one thread at a time.
 *  Devices.  A call that takes a context makes the context's device current
 *    on the calling thread and leaves it current.  A tensor handle belongs to
 *    the device of the context it was created with; passing it with a
 *    context of another device fails with CP_ERR_ARG.
 */
#ifndef CP_GB300_H
#define CP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CP_OK = 0,
  CP_ERR_ARG = 1,          /* bad argument (null pointer, bad mode, R < 1 ...)   */
  CP_ERR_SHAPE = 2,        /* inconsistent sizes, coordinates out of range        */
  CP_ERR_OOM = 3,          /* device allocation failed or budget exceeded          */
  CP_ERR_CUDA = 4,         /* a CUDA runtime/driver call failed                   */
  CP_ERR_NOT_SPD = 5,      /* Gammabar^(n) not positive definite after one ridge  */
  CP_ERR_NONFINITE = 6,    /* NaN or Inf met in f or g                            */
  CP_ERR_LINESEARCH = 7,   /* line search could not start (not a descent dir.)    */
  CP_ERR_MAXIT = 8,        /* cp_solve stopped at maxit without meeting tol       */
  CP_ERR_TIMEOUT = 9,      /* a bounded device wait gave up                       */
  CP_ERR_BUSY = 10,        /* server has no free slot / budget for a request      */
  CP_ERR_UNSUPPORTED = 11  /* combination not provided (e.g. precision on COO)    */
} cp_status;

typedef enum {
  CP_FP64 = 0,          /* every product and sum in FP64                               */
  CP_MIXED_BF16X3 = 1   /* MTTKRP on tensor cores: T and the Khatri-Rao tile split   */
                        /* into bf16 hi+lo, products hi*hi + hi*lo + lo*hi, FP32      */
                        /* accumulation; everything else stays FP64                   */
} cp_precision;

typedef enum { CP_DTYPE_F32 = 0, CP_DTYPE_F64 = 1 } cp_dtype;

typedef struct cp_ctx cp_ctx;
typedef struct cp_tensor cp_tensor;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to enqueue on (borrowed, not destroyed; cudaStreamLegacy selects the legacy
 * default stream), or NULL to create a private non-blocking stream.
 * Errors: CP_ERR_ARG, CP_ERR_CUDA. */
cp_status cp_ctx_create(int device, void* cuda_stream, cp_ctx** out);
void cp_ctx_destroy(cp_ctx* ctx);
/* Message of the calling thread's last failed call ("" if none).  The string
 * stays valid until the thread's next failing call. */
const char* cp_last_error(void);
/* Wait for all work on the context stream; return any error that a kernel
 * recorded in the context's device status word since the last sync. */
cp_status cp_ctx_sync(cp_ctx* ctx);
/* The context's cudaStream_t. */
void* cp_ctx_stream(cp_ctx* ctx);
/* Number of CUDA kernels this library has launched in the process so far
 * (all contexts; for accounting in benchmarks). */
unsigned long long cp_kernel_launches(void);
/* Kernel timers (profiling aid).  While enabled, every launch of an MTTKRP
 * kernel on this context's stream (outside stream capture) is bracketed by
 * CUDA events.  Enabling (or disabling) resets the sums.  cp_ctx_timer_read
 * synchronises the stream and returns the summed device time and the number
 * of launches of family `which`: 0 tensor-core (bf16x3) dense MTTKRP kernel,
 * 1 FP64 dense MTTKRP kernel, 2 sparse MTTKRP kernel. */
cp_status cp_ctx_timer_enable(cp_ctx* ctx, int enable);
cp_status cp_ctx_timer_read(cp_ctx* ctx, int which, double* total_ms, int* launches);

/* ---------------------------------------------------------------- tensors */

/* Dense tensor from `data` (host or device; row-major, last index fastest,
 * prod(dims) elements of `dtype`).  The data are copied; the handle keeps one
 * mode-n matricised copy T_(n) (I_n x prod_{m!=n} I_m, row-major) per mode
 * (Section 2.3, "mode-n matricization") and ||T||_F^2 in FP64.  2 <= N <= 8,
 * every dim >= 1.  Synchronous.  Errors: CP_ERR_ARG, CP_ERR_SHAPE, CP_ERR_OOM. */
cp_status cp_tensor_dense(cp_ctx* ctx, int N, const int64_t* dims, cp_dtype dtype,
                          const void* data, cp_tensor** out);

/* Sparse tensor in coordinate form (Section 4, "sparse tensors").  coords is
 * nnz x N int64 row-major (host or device), values FP32 (host or device);
 * coordinates must be distinct and in range (checked: CP_ERR_SHAPE).  For each
 * mode n the handle keeps the nonzeros stably sorted by the cyclic key
 * (i_n, i_{n+1}, ..., i_{n-1}) with segment pointers over runs of equal i_n.
 * nnz may be 0.  Synchronous. */
cp_status cp_tensor_coo(cp_ctx* ctx, int N, const int64_t* dims, int64_t nnz,
                        const int64_t* coords, const float* vals, cp_tensor** out);

/* Order of the tensor, its dims (array of N, host) and ||T||_F^2 (host).
 * Any output may be NULL. */
cp_status cp_tensor_info(const cp_tensor* t, int* N, int64_t* dims, double* norm2);

/* Copy mode `mode`'s sort permutation (nnz int64), segment pointers
 * (nseg + 1 int64) and segment rows (nseg int64) to HOST arrays (any may be
 * NULL; nseg is written if non-NULL).  COO tensors only; synchronous. */
cp_status cp_tensor_sorted_mode(cp_ctx* ctx, const cp_tensor* t, int mode, int64_t* perm,
                                int64_t* seg_ptr, int64_t* seg_row, int64_t* nseg);
void cp_tensor_destroy(cp_tensor* t);

/* ------------------------------------------------------ multilinear kernels */

/* MTTKRP M^(n) = T_(n) Phibar^(n) (Section 2.3, Eq. Gn and Eq. Phi): for every
 * i and r, M[i,r] = sum over all other indices of T[...] * prod_{m != n}
 * A^(m)[i_m, r].  u: iterate (P doubles); out: I_mode x R doubles, row-major.
 * CP_MIXED_BF16X3 is provided for dense tensors only.  Asynchronous. */
cp_status cp_mttkrp(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, int mode,
                    double* out, cp_precision prec);

/* Khatri-Rao variant MTTKRPs along a line x = u + beta d (Section 2.1, Eq.
 * linesearch; the CP model is multilinear in the factors): for each listed
 * mode n and each v in [0, 2^(N-1)), M_v^(n) = T_(n) times the Khatri-Rao
 * product of the other modes' factors, in which the j-th other mode (the
 * modes other than n in increasing order, j from 0) contributes d's factor
 * when bit j of v is set and u's otherwise.  Then
 * M^(n)(u + beta d) = sum_v beta^popcount(v) M_v^(n) for every beta.
 * u, d: iterate and direction (P doubles each, device); modes: HOST array of
 * nmodes distinct modes (1 <= nmodes <= N); out (device): for each listed
 * mode in the order given, 2^(N-1) blocks (v = 0, 1, ...) of I_mode x R
 * doubles, row-major.  CP_MIXED_BF16X3 on a dense tensor with
 * 2^(N-1) * (R rounded up to 4) <= 256 runs one tensor-core launch for all
 * listed modes (the line search's pass); otherwise one MTTKRP per variant.
 * Asynchronous. */
cp_status cp_mttkrp_variants(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, const double* d,
                             const int* modes, int nmodes, double* out, cp_precision prec);

/* Dimension-tree MTTKRPs of a 3-way dense tensor (no counterpart in the
 * paper; an exact regrouping of the index sum of Eq. Gn): one pass over T
 * forms W = T x_c A^(c), W[i_a, i_b, r] = sum_{i_c} T[...] A^(c)[i_c, r],
 * for `contracted` c = 0 or 2, and the MTTKRPs of the two other modes a < b
 * follow from W: M^(a)[i, r] = sum_j W[i, j, r] A^(b)[j, r] and
 * M^(b)[j, r] = sum_i W[i, j, r] A^(a)[i, r].  out: M^(a) (I_a x R) then
 * M^(b) (I_b x R), row-major doubles.  CP_MIXED_BF16X3 only (W on the
 * tensor cores with bf16x3 split products and FP32 accumulation; the two
 * contractions with FP32 copies of the factors, FP32 sums);
 * CP_ERR_UNSUPPORTED otherwise.  Asynchronous. */
cp_status cp_mttkrp_dimtree(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, int contracted,
                            double* out, cp_precision prec);

/* FP64 dense MTTKRP that allocates no device memory (no counterpart in the
 * paper; it exists for callers that cannot allocate while they run: code that
 * enqueues work inside a stream capture it does not own, serving loops with a
 * fixed memory budget in which cudaMalloc may stall or fail, or programs
 * whose device memory is owned by another allocator).  Same arguments and
 * result as cp_mttkrp with CP_FP64 on a dense tensor (t must be dense; t and
 * ctx are created beforehand).  The split-K partial sums go to one 8 MiB
 * scratch array inside the library, which every GPU that loads the library
 * holds until the process exits.  Rejected with CP_ERR_SHAPE when
 * I_mode * R * 8 bytes exceeds that scratch.  The first call on a device
 * looks up the scratch's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  All calls share the one scratch
 * array: calls that may overlap on the GPU (other streams, other contexts on
 * the same device) race and must be serialised by the caller.  The scratch
 * needs no clearing: every call overwrites the part it reads.  Asynchronous. */
cp_status cp_mttkrp_noalloc(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, int mode,
                            double* out);

/* Objective and gradient (Eq. fA, Eq. Gn):
 *   f = 1/2 (||T||^2 - 2 <T, A_R> + sum_{r,s} Gamma[r,s]),
 *   G^(n) = -M^(n) + A^(n) Gammabar^(n),
 * with Gamma, Gammabar^(n) the Hadamard products of the factor Grams (Eq.
 * Gamma).  f: one device double; g: P device doubles or NULL.  All sums of
 * f are FP64.  Asynchronous. */
cp_status cp_fg(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, double* f,
                double* g, cp_precision prec);

/* One ALS iteration M(u) (Section 2.3, Eq. foopt): for n = 1..N,
 * A^(n) <- M^(n) (Gammabar^(n))^{-1} with the factors of modes < n already
 * updated (block Gauss-Seidel); the SPD R x R matrix is inverted by
 * Gauss-Jordan elimination without pivoting, which fails exactly when a
 * Cholesky factorisation would.  If a pivot is not positive, one retry with
 * Gammabar + 1e-12 tr/R I; then CP_ERR_NOT_SPD is recorded (reported by the
 * next sync).  If
 * `normalize` is non-zero the result is normalised as cp_normalize does.
 * u is updated in place.  Asynchronous. */
cp_status cp_als_sweep(cp_ctx* ctx, const cp_tensor* t, int R, double* u, int normalize,
                       cp_precision prec);

/* Normalisation and reordering (Section 2.3): every column of every factor
 * is scaled to norm lambda_r^(1/N), lambda_r = prod_n ||a_r^(n)||, and the
 * terms are stably ordered by decreasing lambda_r.  A term with a zero column
 * gets lambda_r = 0 and is left unscaled.  If g (same layout) is given it is
 * rescaled exactly to the gradient at the normalised point (column r of mode
 * n divided by the scale of that column) and permuted alike.  lambda: R
 * doubles (sorted) or NULL.  Asynchronous. */
cp_status cp_normalize(cp_ctx* ctx, int N, const int64_t* dims, int R, double* u, double* g,
                       double* lambda);

/* ------------------------------------------------------------------ N-GMRES */

/* N-GMRES Step II (Section 2.1, Eq. accel, Eq. linearize, Eq. normal): with
 * p_j = gbar - G_j, solve (P^T P + delta I) alpha = -P^T gbar (SPD; by
 * Gauss-Jordan elimination without pivoting),
 * delta = eps * max_j (P^T P)_jj (alpha = 0 if that maximum is 0), and form
 * uhat = ubar + sum_j alpha_j (ubar - U_j).
 * U, G: m x Pn row-major (window iterates and their gradients, any order);
 * ubar, gbar, uhat: Pn doubles; alpha: m doubles (may be NULL).
 * 1 <= m <= 64.  Asynchronous. */
cp_status ngmres_step(cp_ctx* ctx, int64_t Pn, int m, const double* U, const double* G,
                      const double* ubar, const double* gbar, double eps, double* uhat,
                      double* alpha);

/* Line-search parameters (Section 2.4 and More & Thuente 1994).
 * Defaults: ftol 1e-4, gtol 1e-2, xtol 1e-15, stpmin 1e-15, stpmax 1e15,
 * stp0 1, maxfev 20. */
typedef struct {
  double ftol, gtol, xtol, stpmin, stpmax, stp0;
  int maxfev;
} cp_ls_opts;

void cp_ls_opts_default(cp_ls_opts* o);

/* More-Thuente line search on phi(beta) = f(x0 + beta d), phi'(beta) =
 * g(x0 + beta d)^T d (Step III, Eq. linesearch).  phi is a polynomial of
 * degree 2N in beta (the model is multilinear in the factors); its
 * coefficients come from one MTTKRP pass (the last mode against the 2^(N-1)
 * mixes of x0's and d's factors) and factor Grams, and every trial evaluates
 * phi and phi' from them; f and g are then evaluated with cp_fg at the final
 * point.  x0, g0, d: device (P).  f0 = f(x0) and g0 are accepted for
 * interface stability; the search starts from phi(0) and phi'(0) of the
 * polynomial, equal to f0 and g0^T d up to rounding.  On return
 * x = x0 + stp d and f, g are evaluated there (x, g device; f, stp, nfev,
 * info host; nfev counts trials).  info as in More-Thuente: 1 strong Wolfe
 * met, 2 xtol, 3 maxfev, 4 stpmin, 5 stpmax, 6 rounding; and 7 when a trial's
 * phi or phi' is not finite (the search stops at that trial); if
 * phi'(0) >= 0 returns CP_ERR_LINESEARCH.  Synchronous. */
cp_status linesearch(cp_ctx* ctx, const cp_tensor* t, int R, const double* x0, double f0,
                     const double* g0, const double* d, const cp_ls_opts* opts, double* x,
                     double* f, double* g, double* stp, int* nfev, int* info,
                     cp_precision prec);

/* ---------------------------------------------------------------- the solve */

typedef struct {
  int R;               /* rank                                                   */
  int w;               /* N-GMRES window (Section 2.4: 20)                       */
  int maxit;           /* iteration limit                                        */
  double tol;          /* stop when ||g||_2 / P < tol                            */
  double eps;          /* delta = eps * max diag(P^T P) (Section 2.4: 1e-12)     */
  cp_precision prec;   /* precision of MTTKRP in the iterations                  */
  int polish;          /* mixed precision: finish with FP64 iterations until the */
                       /* FP64 gradient meets tol (1 = on)                       */
  double mixed_tol_factor; /* mixed phase stops at tol * factor before polishing */
  cp_ls_opts ls;
  int mixed_maxfev;    /* mixed precision phase: at most this many trials    */
                       /* per line search when > 0 (default 0: ls.maxfev)     */
  int dimtree;         /* 3-way dense tensors in the mixed phase: the sweep's */
                       /* M^(2), M^(3) from W = T x_1 A^(1), and M^(1), M^(2) */
                       /* at ubar from T x_3 A^(3) (see cp_mttkrp_dimtree):  */
                       /* 1 on, 0 off, -1 (default) when prod(dims) >= 2^21  */
  int mixed_stall;     /* mixed phase: hand over to the FP64 phase after this */
                       /* many iterations without a new smallest ||g||         */
                       /* (<= 0: the default, 800)                            */
  int mixed_min_entries; /* dense tensors with fewer entries run CP_MIXED_BF16X3 */
                         /* solves in FP64 (0: the default, 4096; -1: never)   */
} cp_solve_opts;

typedef struct {
  int iters, fg_evals, als_sweeps, restarts, ls_failures, converged;
  int mixed_iters, fp64_iters;
  double f, gnorm_over_P, normT2;
  double t_total_s;
  int ls_trials;       /* line-search trials: evaluations of phi and phi' on  */
                       /* the line polynomial, summed over all searches       */
} cp_solve_report;

void cp_solve_opts_default(cp_solve_opts* o, int R);

/* N-GMRES optimisation algorithm (Algorithm 1; Steps I-III of Section 2.1;
 * window start-up of Section 2.1; restart rule and delta I of Section 2.1):
 *   u0 <- normalise(u0); window {(u0, g(u0))};
 *   repeat: ubar = normalise(ALS(u_i)); uhat = ngmres(window; ubar);
 *           uhat <- normalise(uhat); d = uhat - ubar; s = g(ubar)^T d;
 *           s >= 0: restart (u_{i+1} = ubar, window {(ubar, g(ubar))});
 *           else u_{i+1} = normalise(ubar + beta* d) by the line search;
 *           push (u_{i+1}, g(u_{i+1})) keeping the last w;
 *   until ||g(u_i)||_2 / P < tol or maxit.
 * u: P doubles, host or device; initial guess in, solution out.  rep: host,
 * may be NULL.  Synchronous.  Returns CP_ERR_MAXIT if tol was not met. */
cp_status cp_solve(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts* opts, double* u,
                   cp_solve_report* rep);

/* ------------------------------------------------- batching and serving */

/* Solve nreq independent problems at once (host-side batching of
 * Algorithm 1): every problem runs its own device-resident solve on its own
 * stream, so their iterations overlap on the GPU.  tensors[i], opts[i], u[i]
 * (host or device, in: initial guess, out: solution) as for cp_solve; reps
 * (may be NULL) receives nreq reports.  Returns the first failing status
 * (CP_ERR_MAXIT if a problem did not meet its tol).  Synchronous. */
cp_status cp_solve_batch(cp_ctx* ctx, int nreq, const cp_tensor* const* tensors,
                         const cp_solve_opts* opts, double* const* u, cp_solve_report* reps);

/* Many small 3-way dense decompositions in one persistent launch (Algorithm 1
 * for every request; Steps I-III as for cp_solve).  Each thread-block
 * cluster of `cluster` CTAs (1, 2, 4 or 8; 0 picks one per request from its
 * size) runs the whole solve of one request at a time, with cluster barriers
 * between the dependent steps and no host round trip per iteration, and then
 * takes the next request from a device queue.
 * Requests: tensors[i] dense, N = 3, every side <= 256, I_n R <= 8192,
 * R <= 32, w <= 32 (CP_ERR_UNSUPPORTED otherwise).  opts[i].prec CP_FP64:
 * FP64 throughout; any mixed precision: a phase with FP32 products and FP32
 * sums over at most a few hundred terms on the CUDA cores (partial sums,
 * Grams, solves, window least squares, f and the line search in FP64), then
 * with opts[i].polish the FP64 phase to tol; the mixed phase ends at
 * tol * mixed_tol_factor or after mixed_stall iterations without a new
 * smallest ||g|| (as for cp_solve).  u[i] (host or device, P doubles): the
 * initial guess in, the solution out; reps (may be NULL): nreq reports.
 * Returns the first failing status (CP_ERR_MAXIT if a request did not meet
 * its tol).  Synchronous. */
cp_status cp_solve_many(cp_ctx* ctx, int nreq, const cp_tensor* const* tensors, const cp_solve_opts* opts,
                        double* const* u, cp_solve_report* reps, int cluster);

/* Length of cp_solve_many's launches on this context (default 0.5 s): a
 * cluster that has run this long finishes its current iteration, leaves its
 * request's state in device memory and stops; the next launch resumes it
 * (results are the same whatever the length).  CP_ERR_ARG unless
 * 0 < seconds <= 3600. */
cp_status cp_many_set_round(cp_ctx* ctx, double seconds);

/* The cluster size cp_solve_many uses for a request when given 0: the size
 * chosen for its bucket (ceil log2 of its entries, ceil log2 R, FP64 or
 * mixed).  The first request of a bucket is timed for a few iterations with
 * each size, 1, 2, 4 and 8 CTAs (the request itself, from u0, in scratch
 * buffers); among the sizes within 1.5x of the fastest, the one with the
 * least SM time per iteration (CTAs x time) is kept for the rest of the
 * process.  u0: host or device (P doubles).
 * Synchronous.  CP_ERR_UNSUPPORTED as for cp_solve_many. */
cp_status cp_many_plan(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts* opts, const double* u0, int* cluster);

/* Request server (continuous batching).  Requests (dense tensors, each with
 * its own shape, rank, tolerance and precision) wait in arrival order and are
 * admitted while one of `max_active` slots is free and the sum of the device
 * footprints of the running requests stays within hbm_budget_bytes.  Each
 * admitted request keeps its tensor, factors, N-GMRES window and line-search
 * state on the device; requests that fit the cluster engine (see
 * cp_server_set_engine) share its persistent launches (up to `max_active` of
 * them), the others run on a slot of their own (`max_active` slots, each its
 * own stream); requests that arrive while others run are admitted as slots and
 * memory free up.  A worker thread inside the server admits, polls and
 * retires requests. */
typedef struct cp_server cp_server;

cp_status cp_server_create(cp_ctx* ctx, size_t hbm_budget_bytes, int max_active, cp_server** out);

/* Submit a dense request: data (host, row-major, prod(dims) elements of
 * dtype) and u0 (host, P doubles) are copied at submission; the solution is
 * written to the host array u_out (P doubles), which must stay valid until
 * the request is done.  CP_ERR_BUSY if the request alone exceeds the budget. */
cp_status cp_server_submit(cp_server* s, int N, const int64_t* dims, cp_dtype dtype, const void* data,
                           const cp_solve_opts* opts, const double* u0, double* u_out,
                           uint64_t* req_id);

/* done: 1 once the request finished (or was cancelled); then req_status,
 * rep and latency_s (submission to completion) are filled (each may be NULL). */
cp_status cp_server_poll(cp_server* s, uint64_t req_id, int* done, cp_status* req_status,
                         cp_solve_report* rep, double* latency_s);

/* Cancel a request that is still waiting (CP_ERR_ARG otherwise). */
cp_status cp_server_cancel(cp_server* s, uint64_t req_id);

/* Wait until no request is waiting or running; CP_ERR_TIMEOUT after timeout_s. */
cp_status cp_server_drain(cp_server* s, double timeout_s);

/* p50/p99 latency (nearest rank) of finished requests, finished requests per
 * second since the first submission, number finished, peak admitted footprint.
 * Any output may be NULL. */
cp_status cp_server_stats(cp_server* s, double* p50_s, double* p99_s, double* solves_per_s, int* completed,
                          size_t* peak_bytes);

/* Route requests that fit cp_solve_many's limits (3-way dense, sides <= 256,
 * I_n R <= 8192, R <= 32, w <= 32) and have at most max_work entries x R
 * (max_work / 64 for CP_FP64 requests; max_work <= 0: no such limit) to the
 * cluster engine (on = 1: one
 * persistent launch per round of about 10 ms runs every such running
 * request, each on a thread-block cluster of the size chosen for its bucket,
 * see cp_many_plan), the others to a graph slot of their own (tensor-core
 * MTTKRPs over the whole GPU); on = 0 sends every request to a graph slot.
 * An engine round uses at most max_ctas CTAs (each takes a whole SM;
 * <= 0: as many as fit), leaving the rest to the graph slots.  Default: on,
 * max_work = 2^26, no CTA limit.  Applies to requests admitted from then on
 * (the CTA limit to the next round).  CP_ERR_UNSUPPORTED when the engine
 * could not be set up on this device. */
cp_status cp_server_set_engine(cp_server* s, int on, long long max_work, int max_ctas);

/* Stop the worker after the running requests finish; free everything. */
void cp_server_destroy(cp_server* s);

#ifdef __cplusplus
}
#endif

#endif /* CP_GB300_H */
