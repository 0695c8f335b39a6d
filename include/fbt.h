/*
 * fbt.h - C ABI of the GB300 Fisher-BT library (libfbt.so).
 *
 * Exact Gaussian log-likelihood, score and expected Fisher information of a zero-mean Matern
 * random field, and the Fisher-BT maximiser built on them (Hong, Abdulah, Genton & Sun,
 * "Fisher Scoring for Exact Matern Covariance Estimation through Stable Smoothness
 * Optimization", arXiv 2601.11437).
 *
 * Model (Sec. 2.1): theta = (sigma^2, alpha, nu), all > 0;
 *   C(h; theta) = sigma^2 / (2^(nu-1) Gamma(nu)) (h/alpha)^nu K_nu(h/alpha),
 *   Sigma_ij = C(||s_i - s_j||; theta), plus a diagonal jitter delta (the paper has none):
 *   Sigma = sigma^2 (R + delta I), R the Matern correlation, so that d Sigma / d sigma^2 =
 *   Sigma / sigma^2 exactly (the premise of Algorithm 3, Step 2).
 *   l(theta) = -n/2 log(2 pi) - 1/2 log det Sigma - 1/2 z^T Sigma^-1 z               (Eq. 1)
 *   l_i      = -1/2 tr(Sigma^-1 Sigma_i) + 1/2 z^T Sigma^-1 Sigma_i Sigma^-1 z          (Eq. 2)
 *   I_ij     =  1/2 tr(Sigma^-1 Sigma_i Sigma^-1 Sigma_j)                              (Eq. 3)
 *
 * Conventions
 *   - Every entry point returns an fbt_status (0 = success); fbt_strerror() names it.
 *   - All floating point is IEEE binary64.  Arrays passed in are read, never retained: the
 *     context copies what it needs.  Outputs are caller-allocated host arrays.
 *   - Pointers marked "host or device" are host pointers unless the matching *_on_device flag
 *     is non-zero, in which case they are device pointers on the context's device.
 *   - A context is not thread safe; use one context per host thread.  All device work of a
 *     context runs on the CUDA stream given at creation (NULL = legacy default stream), and
 *     every entry point that returns numbers synchronises that stream before returning.
 *   - The device work of every evaluation runs in this library's CUDA kernels (sm_103a).  No
 *     CPU fallback exists: without a usable GPU, fbt_create returns FBT_ERR_CUDA.
 */
#ifndef FBT_H
#define FBT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FBT_OK = 0,
    FBT_ERR_DOMAIN = 1,   /* a theta_i <= 0 or non-finite: l is -inf, nothing is computed      */
    FBT_ERR_NOT_PD = 2,   /* a Cholesky pivot was <= 0 or not finite: loglik = -inf, the score */
                          /* and Fisher outputs are left untouched                             */
    FBT_ERR_BESSEL = 3,   /* a generated covariance entry was not finite                        */
    FBT_ERR_TIMEOUT = 4,  /* a bounded device wait expired                                      */
    FBT_ERR_CUDA = 5,     /* a CUDA runtime call failed (message: fbt_last_cuda_error)          */
    FBT_ERR_OOM = 6,      /* device memory could not be obtained or the workspace is too small */
    FBT_ERR_ARG = 7,      /* invalid argument (NULL pointer, n < 1, unsupported option)         */
    FBT_ERR_STATE = 8     /* fisher_bt_step on a state that is not running                      */
} fbt_status;

/* Options of a context.  fbt_default_opts() fills the defaults. */
typedef struct {
    double jitter;        /* delta of Sigma = sigma^2 (R + delta I); default 1e-8                 */
    int nb;               /* tile size: 64 or 128 (0 = default 128)                                */
    int reorder;          /* 1 (default): Z-order (Morton) reordering of the locations; results  */
                          /* are permutation invariant, the reordering groups near locations     */
    int with_derivatives; /* 1 (default): workspace for mle_eval; 0: mle_loglik only             */
    int device;           /* CUDA device ordinal; default 0                                        */
    int precision;        /* arithmetic of the tile updates: FBT_PREC_FP64 (default, FP64 DFMA),  */
                          /* FBT_PREC_FP64_EMULATED (FP64-accurate products on the BF16 tensor     */
                          /* cores by 8-bit slicing) or FBT_PREC_MIXED (per tile product 7, 3 or 1 */
                          /* digit planes, FP64 / FP32 / BF16-class, chosen from the operand tiles' */
                          /* largest entries against mixed_tol); the last two need nb = 128.       */
                          /* Diagonal-tile Cholesky, inverses, generation, solves of the field,   */
                          /* the log-determinant and the final reductions stay FP64 throughout.   */
    double mixed_tol;     /* FBT_PREC_MIXED: tau = mixed_tol * sigma^2; a tile product over K =   */
                          /* 128 whose operand entries are below 2^ea, 2^eb uses 1 plane when      */
                          /* 2^(ea+eb) < tau / 4, 3 planes when 2^(ea+eb) < 2^13 tau, is skipped   */
                          /* when 2^(ea+eb) < tau / 2^8 (each keeps the product within tau / 2);   */
                          /* default 1e-12                                                         */
} fbt_opts;

enum { FBT_PREC_FP64 = 0, FBT_PREC_FP64_EMULATED = 1, FBT_PREC_MIXED = 2 };

void fbt_default_opts(fbt_opts* opts);

typedef struct fbt_ctx fbt_ctx;   /* opaque: owns the device copies of locations and field,  */
                                  /* the tile workspace and the per-evaluation scratch        */

/* Device bytes the workspace of a context for n locations needs (0 on invalid input). */
size_t fbt_workspace_bytes(long long n, const fbt_opts* opts);

/*
 * Create a context for n locations and one observed field.
 *   locs      n x 2 row-major (x_i, y_i), host or device (locs_on_device)
 *   z         n values, host or device (z_on_device)
 *   workspace device memory of at least fbt_workspace_bytes(n, opts) bytes, 256-byte aligned,
 *             owned by the caller and kept alive until fbt_destroy; NULL = the library
 *             allocates (and frees) it itself with cudaMalloc
 *   stream    a cudaStream_t on opts->device, or NULL
 * Locations and field are copied to the device, put in Z-order (Morton order of the
 * locations; l, the score and the Fisher matrix are invariant under any reordering of Eq. 1-3)
 * and padded to whole tiles.  On failure *out is NULL.
 */
fbt_status fbt_create(fbt_ctx** out, const double* locs, int locs_on_device,
                      const double* z, int z_on_device, long long n,
                      const fbt_opts* opts, void* workspace, size_t workspace_bytes,
                      void* stream);

/* Replace the observed field (n values, host or device); locations and workspace are kept. */
fbt_status fbt_set_field(fbt_ctx* ctx, const double* z, int z_on_device);

/*
 * Algorithm 2 (Sec. 2.2): l(theta) for theta = (sigma^2, alpha, nu).
 * Covariance generation, tiled Cholesky, log-determinant 2 sum log L_ii, Y = L^-1 z, Y^T Y.
 * FBT_ERR_DOMAIN / FBT_ERR_NOT_PD set *loglik = -inf.
 */
fbt_status mle_loglik(fbt_ctx* ctx, const double theta[3], double* loglik);

/*
 * Algorithm 3 (Sec. 2.2): l(theta), score[3] = grad l (Eq. 2), fisher[9] = I(theta) (Eq. 3,
 * row-major, symmetric).  Requires with_derivatives.  Sigma_alpha and Sigma_nu come from the
 * partials of the Matern function (Sec. 2.2 and Supp. A); tr(Sigma^-1 Sigma_i Sigma^-1 Sigma_j)
 * is evaluated as the Frobenius product <B_i, B_j> of B_i = L^-1 Sigma_i L^-T, which equals
 * the trace of Eq. 3 (the role Eq. 4 plays in the paper).
 */
fbt_status mle_eval(fbt_ctx* ctx, const double theta[3], double* loglik,
                    double score[3], double fisher[9]);

/*
 * l(theta) and its gradient by the adjoint (trace) form of Eq. 2,
 *   dl/dtheta_i = 1/2 <w w^T - Sigma^-1, Sigma_i>_F,  w = Sigma^-1 z,
 * with Sigma^-1 = L^-T L^-1 formed from the Cholesky factor and the partials Sigma_alpha,
 * Sigma_nu regenerated entry by entry inside the reduction (never stored); dl/dsigma^2 by
 * Algorithm 3, Step 2.  About n^3 flops against 7 n^3 / 3 for mle_eval, which also yields the
 * Fisher information.  Requires with_derivatives, nb = 128 and precision
 * FBT_PREC_FP64_EMULATED or FBT_PREC_MIXED (FBT_ERR_ARG otherwise).  Reuses the factor of a
 * preceding evaluation at the same theta.
 */
fbt_status mle_loglik_grad(fbt_ctx* ctx, const double theta[3], double* loglik, double grad[3]);

/* Options of the Fisher-BT driver (Algorithm 1, Sec. 2.1); fbt_default_bt_opts() fills the
 * paper's values: armijo_c 0.001, rho 0.5, slack 0.001, grad_tol 0.001, max_ll_calls 60,
 * max_grad_calls 20, nm_ftol 1e-9 (plus nm_max_calls 1000, max_halvings 64 as guards).
 * polish_step (default 1e-4; not in the paper) applies to fisher_bt_run on an FBT_PREC_MIXED
 * context whose tolerance is above 0: the run iterates with the mixed tile products until the
 * Fisher direction is small, max_i |phi_i / theta_i| <= polish_step, the last line search
 * halved phi four times or more, or the stopping rule or the shift rule holds on a mixed
 * evaluation; it then switches the context to all digit planes
 * (FP64-accurate products), repeats the Fisher scoring iteration at the current theta and
 * continues Algorithm 1 there, so that the paper's stopping rule is judged on FP64-accurate
 * values.  The context's tolerance is restored when the run returns.  polish_step < 0 turns the
 * switch off (the whole run in mixed precision). */
typedef struct {
    double armijo_c, rho, slack, grad_tol, nm_ftol;
    int max_ll_calls, max_grad_calls, nm_max_calls, max_halvings;
    double polish_step;
} fbt_bt_opts;

void fbt_default_bt_opts(fbt_bt_opts* opts);

enum { FBT_RUNNING = 0, FBT_CONVERGED = 1, FBT_SHIFT = 2, FBT_DONE_NM = 3, FBT_FAILED = -1 };

/* State of a Fisher-BT run (Algorithm 1): theta^(t), phi^(t) = I^-1 grad l, l, grad l, I at
 * theta^(t), the call counters of the shift rule, the accepted-step count and the state;
 * halvings of the last line search; polish_iter: the accepted-step count at which a mixed run
 * switched to FP64-accurate products (-1: no switch), theta_mixed: theta at that switch. */
typedef struct {
    double theta[3], phi[3], loglik, score[3], fisher[9];
    int n_ll, n_grad, iter, state, halvings, polish_iter;
    double theta_mixed[3];
} fbt_state;

/*
 * Start Algorithm 1: theta0 given (non-NULL), else the best of the nine L9 candidates of
 * Table 1 built from theta_lo and theta_hi; then one Fisher scoring iteration.
 */
fbt_status fisher_bt_start(fbt_ctx* ctx, const double* theta0, const double* theta_lo,
                           const double* theta_hi, const fbt_bt_opts* bt, fbt_state* st);

/*
 * One accepted Fisher-BT step (Algorithm 1's loop body): halve phi until the relaxed Armijo
 * condition (Eq. 5 with c = 0.001 and slack 0.001) holds, evaluating mle_loglik on the host's
 * behalf for each candidate; theta <- theta + phi; one Fisher scoring iteration (mle_eval).
 * Sets st->state to FBT_CONVERGED (||grad l||_2 <= grad_tol) or FBT_SHIFT (call limits exceeded
 * or I not positive definite).  FBT_ERR_STATE if st->state != FBT_RUNNING.
 */
fbt_status fisher_bt_step(fbt_ctx* ctx, fbt_state* st, const fbt_bt_opts* bt);

/* Algorithm 1 end to end, including the Nelder-Mead fallback and its final Fisher evaluation. */
fbt_status fisher_bt_run(fbt_ctx* ctx, const double* theta0, const double* theta_lo,
                         const double* theta_hi, const fbt_bt_opts* bt, fbt_state* out);

/*
 * Many independent fields (one context each, same device; a context may appear once).  A pool
 * of nthreads host threads (<= 0: FBT_BATCH_DEFAULT_THREADS) drives the fields, largest first,
 * each thread on its own CUDA stream, ordered after and before each context's own stream, so
 * that the fields' kernels overlap on the GPU.  Nothing is exchanged between fields.  Every
 * call returns when all fields are done: FBT_OK, or the first hard error (CUDA, OOM, TIMEOUT,
 * ARG, STATE) of any field; the per-field statuses are in status[] either way.
 */
#define FBT_BATCH_DEFAULT_THREADS 16
enum { FBT_BATCH_LOGLIK = 0, FBT_BATCH_EVAL = 1 };

/* k candidates per field: thetas[(f k + j) 3 + d]; with FBT_BATCH_EVAL, out[(f k + j) 13 + ...]
 * = (l, score[3], fisher[9]) as mle_eval, else out[f k + j] = l as mle_loglik; status[f k + j]
 * is that evaluation's status. */
fbt_status mle_eval_batch(fbt_ctx* const* ctxs, int nfields, const double* thetas, int k, int flags,
                          double* out, int* status, int nthreads);

/* fisher_bt_start / fisher_bt_step / fisher_bt_run per field (theta0s, theta_lo, theta_hi: 3 per
 * field, or NULL as in fisher_bt_start); fisher_bt_step_batch leaves fields whose state is not
 * FBT_RUNNING untouched (status FBT_OK). */
fbt_status fisher_bt_start_batch(fbt_ctx* const* ctxs, int nfields, const double* theta0s,
                                 const double* theta_lo, const double* theta_hi, const fbt_bt_opts* bt,
                                 fbt_state* states, int* status, int nthreads);
fbt_status fisher_bt_step_batch(fbt_ctx* const* ctxs, int nfields, fbt_state* states,
                                const fbt_bt_opts* bt, int* status, int nthreads);
fbt_status fisher_bt_run_batch(fbt_ctx* const* ctxs, int nfields, const double* theta0s,
                               const double* theta_lo, const double* theta_hi, const fbt_bt_opts* bt,
                               fbt_state* states, int* status, int nthreads);

/*
 * Autotuners (not in the paper; they choose how the work is run, never what it computes).
 *
 * fbt_tune_batch_threads: times one batched Algorithm 2 pass (mle_eval_batch, l only) over the
 * given fields (thetas: 3 per field) for each candidate host-thread count, after two untimed
 * passes (direct launches, then graph capture), and returns the fastest count in *best and
 * each candidate's wall-clock seconds in seconds[ncand].  Many concurrent streams only overlap
 * on the GPU when the process allows enough hardware queues (CUDA_DEVICE_MAX_CONNECTIONS, an
 * environment variable read when the CUDA context is created; the default is 8).
 *
 * fbt_autotune: for a field of n locations (host arrays, as fbt_create), chooses the faster of
 * the two FP64-accurate configurations, FBT_PREC_FP64 with nb = 64 (FP64 DFMA tiles) and
 * FBT_PREC_FP64_EMULATED with nb = 128 (tensor-core tiles), by timing `reps` Algorithm 3
 * evaluations of each at theta on temporary contexts (after two untimed ones).  opts->precision
 * must be one of the two; on return opts->precision and opts->nb hold the choice and
 * seconds[2] the mean seconds per evaluation of (FP64 nb 64, emulated nb 128).  The choice is
 * cached per device and size band (n rounded up to a power of two): a later call in the band
 * returns it without measuring (*cached = 1; cached may be NULL).
 */
fbt_status fbt_tune_batch_threads(fbt_ctx* const* ctxs, int nfields, const double* thetas, const int* candidates,
                                  int ncand, int* best, double* seconds);
fbt_status fbt_autotune(const double* locs, const double* z, long long n, const double theta[3], int reps,
                        fbt_opts* opts, double seconds[2], int* cached);

/*
 * Graph replay of evaluations (default on).  The launch sequence of an evaluation depends only on
 * its kind (Algorithm 2 with or without kept partials; Algorithm 3 fresh, reusing the factor,
 * or reusing factor and partials), not on theta, which reaches the device through a buffer the
 * sequence itself fills.  The second evaluation of a kind captures its sequence as a CUDA graph;
 * later ones replay it with one launch.  Results are bitwise those of direct launches.  Not
 * used for FBT_PREC_MIXED with a tolerance above 0 (its plane thresholds depend on sigma^2) or
 * while profiling.
 * fbt_set_graphs(ctx, 0) switches to direct launches (and drops the captured graphs).
 */
fbt_status fbt_set_graphs(fbt_ctx* ctx, int enable);
/* Number of evaluation kinds currently replayed from a captured graph (0 .. 5). */
int fbt_graph_count(fbt_ctx* ctx);

/* FBT_PREC_MIXED contexts: set the tolerance of the digit-plane choice (as fbt_opts.mixed_tol;
 * 0 keeps all 7 planes, the FP64-accurate products of FBT_PREC_FP64_EMULATED, bitwise), read it
 * back (-1 for a NULL context), and read (optionally reset) the tile-product tasks counted per
 * tier since creation: counts[0] skipped (every entry below the tolerance), counts[1] 1 plane,
 * counts[2] 3 planes, counts[3] 7 planes.  FBT_ERR_ARG on other contexts or tol outside [0, 1). */
fbt_status fbt_set_mixed_tol(fbt_ctx* ctx, double tol);
double fbt_get_mixed_tol(fbt_ctx* ctx);
fbt_status fbt_mixed_counts(fbt_ctx* ctx, long long counts[4], int reset);

/* Iteration limit of every mbarrier wait in the tensor-core tile-update kernel (test hook; <= 0
 * restores the default of 2^26 tries).  A wait that runs out makes the kernel stop issuing work,
 * wait for the copies and tensor-core operations it already issued, free its tensor memory and
 * return; the evaluation then fails with FBT_ERR_TIMEOUT and the context stays usable. */
fbt_status fbt_set_spin_budget(fbt_ctx* ctx, long long iterations);

/* Per-kernel statistics, recorded with CUDA events on the context's stream while enabled. */
typedef struct {
    const char* name;     /* kernel family                                                    */
    long long launches;   /* launches recorded                                                */
    double ms;            /* summed device time of those launches                             */
    double flops;         /* algorithmic floating-point operations of those launches          */
    double bytes;         /* algorithmic DRAM bytes of those launches                         */
} fbt_kernel_stat;

/* Enable (1) or disable (0) per-kernel event timing; enabling clears the counters. */
fbt_status fbt_profile(fbt_ctx* ctx, int enable);
/* Copy up to cap entries of the statistics into out; *count receives the number of families. */
fbt_status fbt_profile_read(fbt_ctx* ctx, fbt_kernel_stat* out, int cap, int* count);
/* Number of this library's kernel launches since creation (or the last reset). */
long long fbt_launch_count(fbt_ctx* ctx, int reset);

/* Bytes this context has copied host-to-device and device-to-host since creation (or the last
 * reset), inputs and results included; either pointer may be NULL. */
fbt_status fbt_transfer_bytes(fbt_ctx* ctx, long long* h2d, long long* d2h, int reset);

/* Number of mle_eval calls that reused the Cholesky factor left by the previous evaluation at
 * the same theta (the Fisher iteration at the point the line search accepted, Algorithm 1): the
 * factor of Sigma(theta) is kept in the context after every successful evaluation, and an
 * mle_eval at an identical theta generates only the partials instead of Sigma and its factor. */
long long fbt_factor_reuses(fbt_ctx* ctx);

/* Geometry of a context: padded size, tile size, tile count per side. */
fbt_status fbt_geometry(fbt_ctx* ctx, long long* n, long long* n_pad, int* nb, int* tiles);

/* Copy the lower-tile slab (which = 0: Sigma or its Cholesky factor, 1: Sigma_alpha or B_alpha,
 * 2: Sigma_nu or B_nu, whichever the last call left there) to a host or device buffer of
 * tiles*(tiles+1)/2 * nb*nb doubles (fbt_geometry).  Tile (i, j), i >= j, starts at
 * (j*tiles - j*(j-1)/2 + i - j) * nb*nb and is column-major inside.  Test hook. */
fbt_status fbt_copy_slab(fbt_ctx* ctx, int which, double* dst, int dst_on_device);
/* Permutation applied to the locations: perm[i] = caller index of reordered point i. */
fbt_status fbt_copy_perm(fbt_ctx* ctx, long long* perm);
/* Generate Sigma, Sigma_alpha, Sigma_nu at theta into the slabs without factorising (test hook). */
fbt_status fbt_generate(fbt_ctx* ctx, const double theta[3], int with_derivatives);

/*
 * Allocation-free log-likelihood for small problems.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory at the time they need l(theta),
 * for example a process whose GPU memory another framework's allocator has already reserved,
 * or a latency-critical loop that must not enter the CUDA allocator (cudaMalloc and cudaFree
 * may synchronise the device).
 *
 * Computes the same l(theta) as mle_loglik (Algorithm 2, tile size 64, Z-order reordering) for
 * n <= FBT_NOALLOC_MAX_N locations.  All scratch lives in one file-scope device array of
 * 5 MiB inside libfbt.so, which every GPU that loads the library holds until the process exits;
 * nothing is allocated or freed by this call (no cudaMalloc, cudaFree or allocating library
 * routine).
 *   locs, z           n x 2 row-major locations and n field values: device pointers on the
 *                     current device if inputs_on_device != 0, else host pointers
 *   theta, jitter     as for mle_loglik and fbt_opts.jitter (host values)
 *   loglik            host pointer receiving l(theta) (-inf on FBT_ERR_DOMAIN / FBT_ERR_NOT_PD)
 *   stream            cudaStream_t on the current device, or NULL; the call synchronises it
 * Returns FBT_ERR_ARG for n < 1, n > FBT_NOALLOC_MAX_N, NULL pointers or a bad jitter.
 * Every call looks up the array's device address in the current context (the lookup allocates
 * nothing, and it stays valid after the primary context is reset and created again); make the
 * first call on a device before any stream capture.  Every call uses the
 * same array and leaves its contents behind for the next; calls whose device work overlaps
 * (two host threads, or two streams not ordered with each other) race on it and must be
 * serialised by the caller.
 */
#define FBT_NOALLOC_MAX_N 1024
long long fbt_noalloc_max_n(void);
fbt_status fbt_loglik_noalloc(const double* locs, const double* z, int inputs_on_device, long long n,
                              const double theta[3], double jitter, double* loglik, void* stream);

void fbt_destroy(fbt_ctx* ctx);
const char* fbt_strerror(int status);
const char* fbt_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FBT_H */
