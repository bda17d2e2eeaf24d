/*
 * apc_batch.h -- C ABI of the batched APC solver: many independent systems
 * A_s X_s = B_s (s = 0 .. nsys-1), each square (n_s x n_s) with its own
 * uneven row partition and k <= 32 right-hand sides, advanced together by one
 * persistent kernel on the tensor cores.
 *
 * Method per system (Azizan-Ruhi, Lahouti, Avestimehr, Hassibi, 2017): the
 * rows are split into m_s contiguous blocks (Sec. 2), each block keeps an
 * iterate x_i (n x k) and the master keeps xbar (n x k).  One iteration is
 *     z_i  = Q_i^T xbar - c_i,
 *     x_i <- x_i + gamma_s (xbar - x_i - Q_i z_i)                  (cons1)
 *     xbar <- (eta_s/m_s) sum_i x_i + (1 - eta_s) xbar              (cons2)
 * where Q_i is an orthonormal basis of the row space of A_i (Sec. 3.3) and
 * c_i = R_i^{-T} b_i the coordinates of every solution of A_i x = b_i in it,
 * so that Q_i z_i = Q_i Q_i^T (xbar - x_i) = (I - P_i)(xbar - x_i): this is
 * Eq. (cons1) in the form used in App. A (Eq. (e_i(t+1)), which relies on
 * A_i x_i = b_i).  Initialisation (Algorithm 1): x_i(0) = Q_i c_i, the
 * least-norm solution of A_i x = b_i, and xbar(0) their mean.
 *
 * Arithmetic: set-up in FP64 (Cholesky QR per block, as apc_setup); Q_i is
 * stored in BF16; the iterates are FP32, the master's estimate double-float,
 * and products accumulate in FP32 on the tensor cores.
 *
 * Conventions are those of apc.h: APC_OK or a negative APC_ERR_* code; *_dev
 * pointers are device memory, *_host host memory; the caller owns every
 * buffer it passes; `stream` is a cudaStream_t passed as void*; a batch
 * belongs to the device current at apc_batch_setup; calls on one batch must
 * not overlap.  Matrices are row-major.
 */
#ifndef APC_BATCH_H
#define APC_BATCH_H

#include "apc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct apc_batch apc_batch;

/* apc_batch_setup -- partition and factor every system (Sec. 2, Sec. 3.3) and
 * form the least-norm coordinates c_i of every right-hand side.
 *   n_host[s], m_host[s] : size and number of row blocks of system s.
 *   row_offsets_host     : the systems' offsets one after another, m_s + 1
 *                          int64 each (0 = first, n_s = last), blocks of 1..256
 *                          rows and fewer rows than n_s, m_s <= 256.
 *   A_dev_host[s]        : host array of device pointers, A_s n_s x n_s FP64,
 *                          leading dimension n_s.
 *   B_dev_host[s]        : host array of device pointers, B_s n_s x k FP64,
 *                          leading dimension k.  Copied.
 *   k                    : right-hand sides per system, 1..32.
 *   opt                  : NULL or precision APC_BF16 (the only one) and the
 *                          limit of every device-side wait (0 = 2 s).
 * Errors: INVALID_ARG, UNSUPPORTED (k, precision), SINGULAR_BLOCK, NONFINITE,
 * NOMEM, LAUNCH, CUDA; the text names the system.  On error *out is NULL. */
int apc_batch_setup(apc_batch **out, int32_t nsys, const int64_t *n_host, const int32_t *m_host,
                    const int64_t *row_offsets_host, const double *const *A_dev_host,
                    const double *const *B_dev_host, int32_t k, const apc_options *opt, void *stream);

/* apc_batch_set_params -- (gamma_s, eta_s) per system, host arrays of nsys
 * (Theorem 1 gives the optimal pair from the extreme eigenvalues of X_s, see
 * apc_optimal_params).  Synchronous: the parameters are copied to the device
 * with a blocking copy, which waits for the device's earlier work.  Errors:
 * PARAMS unless 0 < gamma_s < 2 and eta_s is finite (nothing is changed
 * then), INVALID_ARG, CUDA. */
int apc_batch_set_params(apc_batch *b, const double *gamma_host, const double *eta_host);

/* apc_batch_set_hb_params -- switch later apc_batch_iterate calls to the
 * distributed heavy-ball method on the preconditioned system of Sec. 6
 * (C_i = (A_i A_i^T)^{-1/2} A_i, d_i = (A_i A_i^T)^{-1/2} b_i; any orthonormal
 * basis of the row space gives the same gradient, so the stored Q_i and c_i
 * serve): per system
 *     zeta <- beta zeta + sum_i Q_i (Q_i^T x - c_i),   x <- x - alpha zeta
 * (the D-HBM update of Sec. 4.3), with x the master's estimate
 * (apc_batch_get_xbar) and zeta = 0 after apc_batch_reset.  alpha_host and
 * beta_host hold one value per system (see apc_hb_optimal_params).
 * apc_batch_set_params switches back to APC.  Synchronous, like
 * apc_batch_set_params.  Errors: PARAMS unless alpha > 0 and 0 <= beta < 1
 * (nothing is changed then), INVALID_ARG, CUDA. */
int apc_batch_set_hb_params(apc_batch *b, const double *alpha_host, const double *beta_host);

/* apc_batch_reset -- Algorithm 1 initialisation of every system (and a zero
 * heavy-ball momentum).  With
 * B_dev_host non-NULL the right-hand sides are replaced first (same layout
 * as in apc_batch_setup).  Errors: INVALID_ARG, TIMEOUT, CUDA. */
int apc_batch_reset(apc_batch *b, const double *const *B_dev_host, void *stream);

/* apc_batch_iterate -- `iters` iterations of every system in one persistent
 * launch, replayed from a CUDA graph captured once per iteration count.
 * Synchronises the stream to read the device error flag.  Errors: PARAMS
 * (no apc_batch_set_params yet), INVALID_ARG (no reset yet, iters < 0),
 * TIMEOUT, CUDA. */
int apc_batch_iterate(apc_batch *b, int64_t iters, void *stream);

/* apc_batch_forward -- apc_batch_reset with B_dev_host (or the stored
 * right-hand sides when NULL), T iterations, and each system's xbar(T) into
 * X_dev_host[s] (n_s x k FP64, leading dimension k; device), in one call.
 * Errors: as apc_batch_reset and apc_batch_iterate (PARAMS also when the
 * batch is set to heavy ball). */
int apc_batch_forward(apc_batch *b, const double *const *B_dev_host, int64_t T, double *const *X_dev_host,
                      void *stream);

/* apc_batch_backward -- reverse-mode sweep through the map of
 * apc_batch_forward, B_s -> xbar_s(T), for every system at once: given
 * G_dev_host[s] = dL/dxbar_s(T) (n_s x k FP64, leading dimension k; device)
 * it writes dL/dB_s to DB_dev_host[s] (same layout).  The map is linear.  Its
 * step (App. A form above) transposes, with lam_i the adjoint of x_i and lbar
 * that of xbar, mu_i = lam_i + (eta/m) lbar, to
 *     lam_i <- (1 - gamma) mu_i,  lbar <- (1 - eta) lbar + gamma sum_i P_i mu_i,
 *     dL/dc_i += gamma Q_i^T mu_i,
 * from lam_i = 0, lbar = G; all lam_i stay equal (one vector ell), so a step
 * is v = Q^T mu over the packed basis (sweep B) and sum_i Q_i v_i (sweep A),
 * both on the tensor cores, in one persistent launch for the T steps.  The
 * initialisation adds dL/dc_i += Q_i^T (ell + lbar/m), and
 * dL/db_i = R_i^{-1} dL/dc_i (c_i = R_i^{-T} b_i).  Uses the iteration state
 * (a later apc_batch_iterate needs apc_batch_reset).  Errors: PARAMS (no APC
 * parameters set, or heavy ball), INVALID_ARG, NOMEM, TIMEOUT, CUDA. */
int apc_batch_backward(apc_batch *b, const double *const *G_dev_host, int64_t T, double *const *DB_dev_host,
                       void *stream);

/* apc_batch_set_tiles -- the shape of the persistent kernel's work units:
 *   rows_a   rows of every system per sweep-A unit (128 or 256; a unit
 *            streams the packed basis of those rows and the machines' iterates);
 *   cols_b   packed columns per sweep-B unit (128, 256 or 512; a unit streams
 *            all rows of those columns);
 *   prefetch the sweep-A L2 prefetch distance in windows / machines (0..8);
 *   l2       the L2 policy of the bulk copies (0 evict-first: operands
 *            streamed once per sweep; 1 normal; 2 evict-last);
 *   split_a, split_b  parts per unit (1, 2, 4 or 8): a sweep-A unit's
 *            machines, a sweep-B unit's rows are shared out among that many
 *            CTAs, whose partial row sums / products are added in part order
 *            by the last part to finish (buffers of split x k x n values per
 *            system are allocated on first use).
 * Smaller and split units give more units to the 152 SMs (a single large
 * system), larger ones fewer unit boundaries (many systems).  For a given
 * split, results do not depend on the other choices (each row and column is
 * computed by the same arithmetic in the same order); a split changes the
 * order of two sums (the machines' row sums, the rows of Q^T xbar'), which
 * moves results at the level of FP32 rounding.  Default 256 / 512 / 2 / 0 /
 * 1 / 1.  Synchronises the device.
 * apc_batch_get_tiles -- the current choices (any pointer may be NULL).
 * Errors: INVALID_ARG, NOMEM, CUDA. */
int apc_batch_set_tiles(apc_batch *b, int32_t rows_a, int32_t cols_b, int32_t prefetch, int32_t l2, int32_t split_a,
                        int32_t split_b);
int apc_batch_get_tiles(const apc_batch *b, int32_t *rows_a, int32_t *cols_b, int32_t *prefetch, int32_t *l2,
                        int32_t *split_a, int32_t *split_b);

/* apc_batch_autotune -- the project's tile tuner: times `reps` launches of
 * `iters` iterations (CUDA events on `stream`) for every unit shape of
 * {256, 128} x {512, 256, 128} with every split {1, 2, 4, 8} x {1, 2, 4, 8}
 * (the current prefetch distance and L2 policy; a sweep is split only when
 * the shape gives it fewer than twice as many units as the grid has CTAs),
 * then the other prefetch
 * distances {0, 1, 2, 4} and then the other L2 policies on the fastest so
 * far, keeps the fastest of all, writes it to tiles_out[6] (the arguments of apc_batch_set_tiles in
 * order; may be NULL) with its time per iteration, and the time of the
 * choices set before the call (ms_default).  Needs apc_batch_set_params and
 * apc_batch_reset first; it advances the iteration state, so apc_batch_reset
 * must follow.  Errors: INVALID_ARG, NOMEM, TIMEOUT, CUDA (the previous
 * choices are then restored). */
int apc_batch_autotune(apc_batch *b, int64_t iters, int32_t reps, int32_t *tiles_out, double *ms_best,
                       double *ms_default, void *stream);

/* apc_batch_get_xbar -- the master's estimate of system s as FP64,
 * n_s x k row-major with leading dimension ldx >= k, into X_dev.
 * apc_batch_get_x -- the iterate x_i of machine `worker` of system s, same
 * layout.  Errors: INVALID_ARG, CUDA. */
int apc_batch_get_xbar(apc_batch *b, int32_t sys, double *X_dev, int64_t ldx, void *stream);
int apc_batch_get_x(apc_batch *b, int32_t sys, int32_t worker, double *X_dev, int64_t ldx, void *stream);

/* apc_batch_set_test_hooks -- failure injection for tests, as
 * apc_set_test_hooks: every wait of one CTA on the others' work in later
 * launches (the grid barrier after the initialisation, and a unit's wait for
 * the units of its system that write its inputs) waits for grid_barrier_skew
 * arrivals more than there will be, and every device-side wait gives up
 * after timeout_s seconds (0 = 2 s).  A launch then returns
 * APC_ERR_TIMEOUT and the batch stays usable (reset, then iterate).
 * Errors: INVALID_ARG. */
int apc_batch_set_test_hooks(apc_batch *b, int32_t grid_barrier_skew, double timeout_s);

/* apc_batch_info -- sizes: systems, right-hand sides, bytes of the packed
 * BF16 bases, bytes of the machines' iterates, CTAs of the persistent grid
 * and the work units of its two sweeps.  Any pointer may be NULL. */
int apc_batch_info(const apc_batch *b, int32_t *nsys, int32_t *k, int64_t *q_bytes, int64_t *state_bytes,
                   int32_t *grid, int32_t *units_a, int32_t *units_b);

/* apc_batch_last_error -- text of the last error on b (or of the last failed
 * apc_batch_setup when b is NULL). */
const char *apc_batch_last_error(const apc_batch *b);

/* apc_batch_destroy -- free the batch and its device buffers.  NULL is a no-op. */
void apc_batch_destroy(apc_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* APC_BATCH_H */
