/*
 * apc.h -- C ABI of the GB300 (sm_103a) Accelerated Projection-based
 * Consensus (APC) solver for A x = b.
 *
 * Method (Azizan-Ruhi, Lahouti, Avestimehr, Hassibi, 2017): the N equations
 * are split into m contiguous row blocks [A_i, b_i] (Sec. 2).  Each block
 * keeps an iterate x_i; the master keeps xbar.  One iteration is Eq. (cons):
 *     x_i(t+1)  = x_i(t) + gamma * P_i (xbar(t) - x_i(t))            (cons1)
 *     xbar(t+1) = (eta/m) sum_i x_i(t+1) + (1 - eta) xbar(t)         (cons2)
 * with P_i = I - A_i^T (A_i A_i^T)^{-1} A_i the projector onto the nullspace
 * of A_i (Sec. 3.1), applied through an orthonormal basis Q_i of the row
 * space of A_i (Sec. 3.3, "e.g. using QR factorization").
 *
 * Conventions for every entry point:
 *   - Return value: APC_OK (0) or a negative APC_ERR_* code; the text of the
 *     last error of a context is available from apc_last_error().
 *   - Pointers named *_dev are CUDA device pointers; *_host are host pointers.
 *     The caller owns every buffer it passes; nothing is retained after a call
 *     returns except what apc_setup() copies into the context.
 *   - Matrices are row-major with an explicit leading dimension (in elements).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; entry points that return host values
 *     synchronise that stream before returning.
 *   - One context belongs to one device (the device current at apc_setup).
 *     Calls on one context must not overlap.
 */
#ifndef APC_H
#define APC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define APC_OK                  0
#define APC_ERR_INVALID_ARG    -1  /* bad size, pointer, offsets or option     */
#define APC_ERR_SINGULAR_BLOCK -2  /* A_i A_i^T not positive definite (Sec.3.1)*/
#define APC_ERR_NONFINITE      -3  /* NaN/Inf in an input or an iterate        */
#define APC_ERR_PARAMS         -4  /* (gamma, eta) outside the set S (Thm. 1)  */
#define APC_ERR_NOT_CONVERGED  -5  /* max_iters reached before the tolerance   */
#define APC_ERR_DIVERGED       -6  /* residual grew by > 1e8 over its start    */
#define APC_ERR_LAUNCH         -7  /* persistent grid cannot be co-resident    */
#define APC_ERR_TIMEOUT        -8  /* a device-side wait ran out of time       */
#define APC_ERR_CUDA           -9  /* a CUDA runtime call failed               */
#define APC_ERR_UNSUPPORTED   -10  /* a size outside what the kernels handle   */
#define APC_ERR_NOMEM         -11  /* device allocation failed                 */

/* Arithmetic of the iteration.  The setup (QR of the blocks) and the
 * refinement residual are FP64 in every mode. */
#define APC_F64  0   /* Q_i FP64, iterates FP64                            */
#define APC_F32  1   /* Q_i FP32, iterates FP32                            */
#define APC_BF16 2   /* Q_i BF16, iterates and accumulation FP32           */

typedef struct apc_ctx apc_ctx;

typedef struct apc_options {
    int32_t precision;      /* APC_F64 / APC_F32 / APC_BF16                   */
    int32_t cluster_size;   /* CTAs sharing one row range, 1..8; 0 = automatic */
    int32_t workers_per_warp; /* 1, 2 or 4 (FP32/BF16) blocks per warp; 0 = automatic */
    double  timeout_s;      /* limit of every device-side wait; 0 = 2 s       */
    int32_t rows_per_group; /* rows of Q per pipeline step, 1 or 2; 0 = automatic */
} apc_options;

typedef struct apc_stats {
    int64_t iterations;     /* APC iterations run (all sweeps)                */
    int32_t sweeps;         /* refinement sweeps (1 without refinement)       */
    double  rel_residual;   /* final ||b - A x||_2 / ||b||_2, FP64            */
    double  seconds;        /* wall time of the solve on the host clock       */
    int64_t residual_checks; /* FP64 residuals ||b - A x|| computed (one sweep over A each) */
    int64_t monitor_checks;  /* free monitor checks (apc_monitor), FP32/FP64 contexts */
} apc_stats;

/* apc_setup -- partition [A, b] into m row blocks and factor each block.
 * Sec. 2 (partition) and Sec. 3.3 (QR).  For block i (rows
 * row_offsets_host[i] .. row_offsets_host[i+1]-1) the rows are scaled to unit
 * length (this leaves P_i unchanged) and A_i^T = Q_i R_i is computed by
 * Cholesky QR in FP64: two passes, or one for an FP32 / BF16 context whose
 * first pass is already orthonormal far below the stored rounding (see
 * apc_setup_report).  Q_i is then stored in the precision of
 * opt->precision.  A copy of A and b (FP64) is kept for FP64 residuals.
 *   A_dev  : N x n, row-major, leading dimension lda >= n, FP64, device.
 *   b_dev  : N, FP64, device.
 *   N >= n >= 1; row_offsets_host: m+1 strictly increasing int64 with
 *   offsets[0] = 0 and offsets[m] = N; every block has 1..256 rows and
 *   at most n rows (a block of n rows of a square system is the whole
 *   system: P_1 = 0).  m <= 256.
 * Errors: INVALID_ARG, SINGULAR_BLOCK (block index in apc_last_error),
 * NONFINITE, NOMEM, CUDA, UNSUPPORTED.  On error *out is NULL. */
int apc_setup(apc_ctx **out, const double *A_dev, int64_t N, int64_t n, int64_t lda,
              const double *b_dev, const int64_t *row_offsets_host, int32_t m,
              const apc_options *opt, void *stream);

/* apc_setup_rows -- apc_setup for a partition whose blocks are arbitrary
 * (not necessarily contiguous) sets of rows (Sec. 2 only asks that the
 * equations be split among the machines).  Block i holds rows
 * row_index_host[row_offsets_host[i] .. row_offsets_host[i+1]-1] of [A, b],
 * in that order; row_index_host (N int64, host) must list every row 0..N-1
 * exactly once.  The rows are gathered once into the blocked order; the
 * context keeps the permutation, so right-hand sides passed later
 * (apc_reset, apc_residual) are given in the caller's row order and row-space
 * results (apc_residual's residual vector, apc_backward's dL/db) come back in
 * it.  Other arguments, limits and errors as apc_setup (INVALID_ARG also when
 * row_index is not a permutation). */
int apc_setup_rows(apc_ctx **out, const double *A_dev, int64_t N, int64_t n, int64_t lda, const double *b_dev,
                   const int64_t *row_index_host, const int64_t *row_offsets_host, int32_t m,
                   const apc_options *opt, void *stream);

/* apc_optimal_params -- Theorem 1: from mu_min, mu_max of
 * X = (1/m) sum_i A_i^T (A_i A_i^T)^{-1} A_i return the optimal rate
 * rho = (sqrt(kappa)-1)/(sqrt(kappa)+1) and (gamma*, eta*), the roots of
 * z^2 - (s + 1 - rho^2) z + s with s = 4/(sqrt(mu_max)+sqrt(mu_min))^2,
 * gamma the smaller one (S requires gamma in [0, 2]).  Pure host arithmetic.
 * Errors: INVALID_ARG unless 0 < mu_min <= mu_max <= 1. */
int apc_optimal_params(double mu_min, double mu_max, double *gamma, double *eta, double *rho);

/* apc_spectral_bounds -- estimates of mu_min and mu_max, the extreme
 * eigenvalues of X = (1/m) sum_i Q_i Q_i^T (Eq. 3), from `steps` (1..4096)
 * steps of the Lanczos process on X started from a pseudo-random vector
 * (splitmix64 stream of `seed`).  Each step applies X once, as two passes of
 * the iteration kernel over the stored bases (in the context's precision:
 * BF16 bases give the eigenvalues of the BF16 X); the Lanczos vectors and the
 * recurrence are FP64, and the extreme eigenvalues of the k x k tridiagonal
 * matrix (the Ritz values) are found by bisection on the host.  Ritz values
 * lie inside the spectrum and approach its ends from inside:
 * mu_min <= *mu_min_host and *mu_max_host <= mu_max.  Theorem 1 needs an
 * enclosing interval for a guaranteed rate: mu_max <= 1 always holds (X is a
 * mean of orthogonal projectors), and the estimate of mu_min should be
 * lowered by the caller's margin.  Uses the context's iteration state (a
 * later apc_iterate needs apc_reset).  Errors: INVALID_ARG, NONFINITE,
 * NOMEM, TIMEOUT, CUDA. */
int apc_spectral_bounds(apc_ctx *ctx, int32_t steps, uint64_t seed, double *mu_min_host, double *mu_max_host,
                        void *stream);

/* apc_hb_optimal_params -- step size and momentum of the heavy-ball method
 * on the system preconditioned as in Sec. 6 (each block premultiplied by
 * (A_i A_i^T)^{-1/2}, so that C^T C = m X): with the spectrum of m X in
 * [m mu_min, m mu_max], alpha = 4 / (sqrt(m mu_max) + sqrt(m mu_min))^2,
 * beta = rho^2, rho = (sqrt(kappa) - 1) / (sqrt(kappa) + 1), the rate Sec. 4.3
 * quotes for D-HBM and Sec. 6 for its preconditioned form (the same as APC's).
 * Pure host arithmetic.  Errors: INVALID_ARG unless 0 < mu_min <= mu_max <= 1
 * and m >= 1. */
int apc_hb_optimal_params(double mu_min, double mu_max, int32_t m, double *alpha, double *beta, double *rho);

/* apc_reset -- Algorithm 1 initialisation for right-hand side rhs_dev
 * (FP64, N, device; NULL = the b given to apc_setup): x_i(0) is the
 * least-norm solution A_i^T (A_i A_i^T)^{-1} b_i of block i and
 * xbar(0) = (1/m) sum_i x_i(0).  Resets the iteration counter. */
int apc_reset(apc_ctx *ctx, const double *rhs_dev, void *stream);

/* apc_iterate -- run `iters` iterations of Eq. (cons) from the current state
 * in one persistent launch (one grid-wide barrier per iteration).  Requires
 * 0 < gamma < 2 (Theorem 1's S; the (m-1)n eigenvalues 1 - gamma of App. A)
 * else APC_ERR_PARAMS.  Errors: TIMEOUT, LAUNCH, CUDA. */
int apc_iterate(apc_ctx *ctx, double gamma, double eta, int64_t iters, void *stream);

/* apc_get_xbar -- copy xbar (n values) to x_dev as FP64 (device). */
int apc_get_xbar(apc_ctx *ctx, double *x_dev, void *stream);

/* apc_get_x -- copy the machines' iterates x_i (m x n, row i = x_i, FP64,
 * device, leading dimension ldx >= n) to x_dev.  For tests and checkpoints. */
int apc_get_x(apc_ctx *ctx, double *x_dev, int64_t ldx, void *stream);

/* apc_get_basis -- copy the orthonormal basis Q_i of block i (Sec. 3.3; the
 * columns span the row space of A_i, so P_i = I - Q_i Q_i^T) to Q_dev as an
 * n x p_i FP64 row-major matrix with leading dimension ldq >= p_i.  The
 * values are those the iteration uses (after rounding to its precision). */
int apc_get_basis(apc_ctx *ctx, int32_t block, double *Q_dev, int64_t ldq, void *stream);

/* apc_residual -- FP64 relative residual ||r - A x||_2 / ||r||_2 of x_dev
 * (FP64, n, device) against rhs_dev (NULL = the stored b).  If resid_dev is
 * not NULL the residual vector r - A x (N, FP64) is written there. */
int apc_residual(apc_ctx *ctx, const double *x_dev, const double *rhs_dev,
                 double *resid_dev, double *rel_residual_host, void *stream);

/* apc_residual_noalloc -- the FP64 relative residual ||rhs - A x||_2 / ||rhs||_2
 * (and, if resid_dev is not NULL, the vector rhs - A x), computed without
 * allocating any device memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate at the moment they need the
 * check (a framework that has reserved all device memory for its own pool, or
 * a latency-critical path where cudaMalloc's implicit synchronisation is not
 * acceptable).  It takes no context: the caller passes every input and output.
 *   A_dev: N x n FP64 row-major, leading dimension lda >= n (device);
 *   x_dev: n FP64; rhs_dev: N FP64; resid_dev: N FP64 or NULL (device);
 *   rel_residual_host: result (host).  Synchronises `stream`.
 * Working memory is a fixed array inside the library (about 512 KiB, held on
 * every GPU that loads the library until the process exits), which limits
 * N to 1,048,576 rows: larger N returns APC_ERR_UNSUPPORTED.  All calls share
 * that array, so calls that overlap on the GPU (different streams or host
 * threads on one device) race and may return wrong results.  The first call
 * on a device looks up the array's address with that device current, and so
 * does the first call after that device's context was reset
 * (cudaDeviceReset): the array may move when the library's code is loaded
 * again.  Make that first call before any stream capture.  Errors: INVALID_ARG, UNSUPPORTED, CUDA (text in
 * apc_last_error(NULL)). */
int apc_residual_noalloc(const double *A_dev, int64_t lda, int64_t N, int64_t n, const double *x_dev,
                         const double *rhs_dev, double *resid_dev, double *rel_residual_host, void *stream);

/* apc_monitor -- the free residual monitor: an estimate of
 * ||r - A xbar||_2 / ||r||_2 for the current xbar and the right-hand side r of
 * the last apc_reset, without reading A.  Block i's residual is
 * A_i xbar - r_i = D_i^{-1} R_i'^T (Q_i^T xbar - c_i), with (D_i A_i)^T = Q_i R_i'
 * (row scaling D_i, two Cholesky factors) and c_i = R_i'^{-T} D_i r_i; because
 * every x_i solves A_i x = r_i (the invariant of App. A),
 * Q_i^T xbar - c_i = Q_i^T (xbar - x_i) = z_i, the coefficients the iteration
 * kernel already holds for its next pass.  So the estimate costs a p_i x p_i
 * product per block.  Its error is set by the precision of the stored bases
 * and of z: about 1e-6 of ||r|| with FP32 bases, 1e-13 with FP64, and near
 * 4e-3 with BF16 bases (their rounding moves Q_i^T xbar by that much).
 * Synchronises `stream`.  Errors: INVALID_ARG (no forward state: call
 * apc_reset first), CUDA. */
int apc_monitor(apc_ctx *ctx, double *rel_residual_host, void *stream);

/* apc_solve -- run Algorithm 1 from the least-norm initialisation until the
 * FP64 relative residual ||b - A xbar|| / ||b|| <= tol, checking every
 * `check_every` iterations, or max_iters iterations.  FP32 and FP64 contexts
 * check with the free monitor (apc_monitor) and compute the FP64 residual
 * (a sweep over A) only when the monitor reaches tol, every eighth check and
 * at the end; BF16 contexts check with the FP64 residual.  With refine != 0
 * the iteration runs as the inner solver of FP64 iterative refinement:
 * x <- x + delta, where delta is the APC solution of A delta = b - A x,
 * stopped when its residual (monitor, or FP64 for BF16) is below 1e-4 of
 * ||b - A x|| or stagnates: it fell less than twofold over the iterations in
 * which the best rate the parameters allow, sqrt|(gamma-1)(eta-1)| (Eq. 5;
 * rho of Theorem 1), would make it fall tenfold (at least one check
 * interval).  One FP64 residual per sweep.  The solution (FP64,
 * n) goes to x_dev.  Errors: NOT_CONVERGED (x_dev still holds the last
 * iterate), DIVERGED, PARAMS, TIMEOUT, CUDA. */
int apc_solve(apc_ctx *ctx, double gamma, double eta, double tol, int64_t max_iters,
              int64_t check_every, int32_t refine, double *x_dev, apc_stats *stats,
              void *stream);

/* apc_backward -- reverse-mode sweep through T unrolled iterations.
 * The forward map is b -> xbar(T): least-norm x_i(0), xbar(0) = mean, then T
 * applications of Eq. (cons) with (gamma, eta) (apc_reset + apc_iterate).  It
 * is linear in b, so its transpose needs no forward state.  Given
 * g_dev = dL/dxbar(T) (FP64, n, device) this computes db_dev = dL/db (FP64, N,
 * device) by the transposed step (P_i is symmetric, Sec. 3.1): with
 * mu_i = lambda_i + (eta/m) lbar,
 *   lambda_i <- (1 - gamma) mu_i + gamma Q_i Q_i^T mu_i,
 *   lbar     <- (1 - eta) lbar + gamma sum_i (mu_i - Q_i Q_i^T mu_i),
 * from lambda_i = 0, lbar = g, then db_i = (A_i^+)^T (lambda_i + lbar/m).
 * Uses the context's iteration state (a later apc_iterate needs apc_reset).
 * Errors: PARAMS (gamma outside (0, 2)), INVALID_ARG, TIMEOUT, CUDA. */
int apc_backward(apc_ctx *ctx, const double *g_dev, int64_t T, double gamma, double eta, double *db_dev,
                 void *stream);

/* apc_solve_rhs -- apc_solve for k right-hand sides in one call: column j of
 * B_dev (N x k FP64, row-major, ldb >= k, caller's row order; device) is
 * solved to the tolerance (or max_iters) exactly as apc_solve solves b, one
 * column after another (each is the context's right-hand side for its solve;
 * the b of apc_setup is put back at the end), and its solution goes to column
 * j of X_dev (n x k FP64, ldx >= k; device).  stats (may be NULL) sums
 * iterations, checks and seconds over the columns and holds the largest
 * final relative residual and sweep count.  Errors: as apc_solve
 * (NOT_CONVERGED if any column missed the tolerance; the others are still
 * solved), NOMEM. */
int apc_solve_rhs(apc_ctx *ctx, const double *B_dev, int64_t k, int64_t ldb, double gamma, double eta, double tol,
                  int64_t max_iters, int64_t check_every, int32_t refine, double *X_dev, int64_t ldx, apc_stats *stats,
                  void *stream);

/* apc_backward_params -- apc_backward plus the derivatives of L with respect
 * to gamma and eta.  The paper prints no formula for these; they are the
 * reverse-mode derivative of Eq. (cons): with mu_i = lambda_i + (eta/m) lbar at
 * step t+1 and the forward states x_i(t), xbar(t),
 *   dL/dgamma = sum_t sum_i <mu_i(t+1), P_i (xbar(t) - x_i(t))>
 *             = (1/gamma) sum_t sum_i <mu_i(t+1), x_i(t+1) - x_i(t)>,
 *   dL/deta   = sum_t <lbar(t+1), (1/m) sum_i x_i(t+1) - xbar(t)>.
 * These need the forward trajectory, which (unlike dL/db) depends on b:
 *   b_dev      : N, FP64, device, caller's row order; NULL = the b of apc_setup.
 *   ckpt_every : the forward states are kept every ckpt_every iterations
 *                (0 = 20) and recomputed from there, one segment at a time,
 *                during the reverse sweep: device memory for ceil(T/ckpt_every)
 *                checkpoints and ckpt_every + 1 states (each m n + n values),
 *                allocated and freed by the call, and ~T more forward steps.
 *   db_dev     : as apc_backward.  dgamma_host, deta_host: host doubles.
 * Uses the context's iteration state (a later apc_iterate needs apc_reset).
 * Errors: PARAMS, INVALID_ARG, NOMEM, TIMEOUT, CUDA. */
int apc_backward_params(apc_ctx *ctx, const double *g_dev, const double *b_dev, int64_t T, double gamma,
                        double eta, int32_t ckpt_every, double *db_dev, double *dgamma_host, double *deta_host,
                        void *stream);

/* apc_forward_rhs -- the forward map of apc_backward for k right-hand sides
 * in one call: for each column b_j of B (N x k FP64, row-major, leading
 * dimension ldb >= k, caller's row order; device), x_i(0) the least-norm
 * solution of block i, xbar(0) their mean, then T iterations with
 * (gamma, eta); xbar_j(T) goes to column j of X (n x k FP64, ldx >= k;
 * device).  Eq. (cons) is column-wise (Sec. 3.1, Algorithm 1), so the columns
 * share every read of the bases:
 *   - BF16 context of a square system with contiguous blocks and 2 <= k <= 32:
 *     the k columns run together on the tensor cores in the form of App. A,
 *     z_i = Q_i^T xbar - c_i, x_i <- x_i + gamma (xbar - x_i - Q_i z_i) (equal to
 *     Eq. (cons) in exact arithmetic; see apc_batch.h), one persistent launch
 *     for the T iterations, on a one-system batch that the context builds on
 *     the first such call (set-up cost and memory of apc_batch_setup; rebuilt
 *     when k changes; it also uses the iteration state);
 *   - any other context: the columns one after another through the
 *     iteration kernel (apc_reset, apc_iterate), in this one call.
 * Uses the context's iteration state (a later apc_iterate needs apc_reset).
 * Errors: PARAMS (gamma outside (0, 2)), INVALID_ARG, NOMEM, TIMEOUT, CUDA. */
int apc_forward_rhs(apc_ctx *ctx, const double *B_dev, int64_t k, int64_t ldb, int64_t T, double gamma, double eta,
                    double *X_dev, int64_t ldx, void *stream);

/* apc_backward_rhs -- apc_backward for k columns in one call: G_dev holds
 * dL/dxbar_j(T) (n x k FP64, ldg >= k; device) and DB_dev receives dL/dB
 * (N x k FP64, lddb >= k, caller's row order; device) for the map of
 * apc_forward_rhs with the same context, T, gamma and eta.  On the tensor-core
 * form the sweep is the exact transpose of that form's steps (every machine's
 * adjoint is one shared vector there, so a step is two GEMMs over the packed
 * bases, like the forward), one persistent launch for the T steps; otherwise
 * the columns go one after another through apc_backward.  Uses the context's
 * iteration state.  Errors: as apc_forward_rhs. */
int apc_backward_rhs(apc_ctx *ctx, const double *G_dev, int64_t k, int64_t ldg, int64_t T, double gamma, double eta,
                     double *DB_dev, int64_t lddb, void *stream);

/* apc_set_deterministic -- with on != 0, later launches of the iteration
 * kernel sum the clusters' partial products z_i' = sum_j Q_i[j,:]^T (...) in a
 * fixed order (each cluster stores its partial; after a grid-wide barrier
 * the partials are added cluster by cluster) instead of with floating-point
 * atomics, whose order varies from run to run.  A context's trajectory is
 * then the same bit for bit on every run with the same launch configuration,
 * at the cost of one more grid-wide barrier per iteration and a buffer of
 * clusters x m x width values (allocated on the first call).  on = 0 returns
 * to atomics.  Errors: INVALID_ARG, NOMEM. */
int apc_set_deterministic(apc_ctx *ctx, int32_t on);

/* apc_state_bytes / apc_export_state / apc_import_state -- checkpoint and
 * resume of the iteration state: the machines' iterates x_i, xbar, the
 * coefficients z of the next pass (all three rotating buffers), the pass
 * counter and ||r||^2 of the last reset, behind a header that records the
 * problem's shape and precision.  apc_state_bytes gives the size of the host
 * buffer; export copies the state into it (synchronises `stream`); import
 * loads a state exported from a context of the same shape (n, N, m, block
 * width) and precision, and a later apc_iterate continues from it exactly
 * where the exporting context stood (bit for bit in deterministic mode).
 * Errors: INVALID_ARG (buffer too short, another shape, not a state), CUDA. */
int apc_state_bytes(const apc_ctx *ctx, size_t *bytes);
int apc_export_state(apc_ctx *ctx, void *host_buf, size_t bytes, void *stream);
int apc_import_state(apc_ctx *ctx, const void *host_buf, size_t bytes, void *stream);

/* apc_set_test_hooks -- failure injection for tests, on the host side of a
 * device wait: every grid barrier of later launches waits for
 * grid_barrier_skew arrivals more than the grid has (0 = normal), and every
 * device-side wait gives up after timeout_s seconds.  With a positive skew a
 * launch of two or more iterations runs out of time at its first barrier,
 * returns cleanly and apc_iterate reports APC_ERR_TIMEOUT; the context stays
 * usable (apc_reset, then iterate).  Errors: INVALID_ARG. */
int apc_set_test_hooks(apc_ctx *ctx, int32_t grid_barrier_skew, double timeout_s);

/* apc_setup_report -- how the blocks were factored: the number of Cholesky-QR
 * passes (2 for FP64 contexts; 1 for FP32 / BF16 contexts when the first
 * pass's basis was probed orthonormal to below 1e-11 / 1e-8, far under the
 * rounding of the stored basis, else 2) and that probe's largest value over
 * the blocks, ||Q_i^T Q_i v - v|| / ||v|| for a fixed +-1 vector v (-1 when not
 * probed).  Either pointer may be NULL.  Errors: INVALID_ARG. */
int apc_setup_report(const apc_ctx *ctx, int32_t *qr_passes, double *orth_probe);

/* apc_context_info -- sizes chosen at setup: padded block width, cluster
 * size, number of clusters, bytes of Q and rows of Q per pipeline step.  Any
 * pointer may be NULL. */
int apc_context_info(const apc_ctx *ctx, int64_t *n, int64_t *N, int32_t *m, int32_t *width,
                     int32_t *cluster_size, int32_t *clusters, int64_t *q_bytes, int32_t *rows_per_group);

/* apc_last_error -- text of the last error on ctx (or of the last failed
 * apc_setup when ctx is NULL).  Valid until the next call on ctx. */
const char *apc_last_error(const apc_ctx *ctx);

/* apc_destroy -- free the context and its device buffers.  NULL is a no-op. */
void apc_destroy(apc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* APC_H */
