// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace apc {

// What one pass of the persistent kernel computes per row j (see apc_iter.cu).
enum PassMode : int {
    MODE_APC = 0,        // Eq. (cons): x_i += gamma P_i (xbar - x_i); momentum average
    MODE_INIT = 1,       // least-norm x_i(0) = Q_i c_i, xbar(0) = mean
    MODE_ADJ = 2,        // transpose of one step of Eq. (cons) (reverse sweep)
    MODE_ADJ_SEED = 3,   // start of the reverse sweep: lambda_i = 0, lbar = g
    MODE_ADJ_FINAL = 4,  // v_i = Q_i^T (lambda_i + lbar/m) at the end of the sweep
    MODE_POWER = 5,      // v <- X v with X = (1/m) sum_i Q_i Q_i^T (Eq. 3)
};

struct IterArgs {
    const void *Q;      // [n][m][P] in the iteration precision
    void *xw;           // [n][m] machines' iterates (TS)
    double *xbar;       // [n] master estimate (always FP64)
    void *zbuf;         // 3 x [m][P] (TS): z_i = Q_i^T(...) for the next pass
    uint32_t *bar;      // grid barrier counter (zeroed before each launch)
    int *err;           // device error word (0 = ok)
    int64_t n;
    int32_t m, P;
    int32_t cs;         // cluster size (CTAs sharing a row range)
    int32_t nw;         // element warps per CTA
    int32_t wpw;        // workers per element warp (1, 2 or 4); worker slots per CTA = nw * wpw
    int32_t rg;         // rows of Q per pipeline step (1 or 2); 2 * rg control warps
    int32_t stages;     // TMA ring depth
    int32_t mode;
    int64_t rows_per_cluster;
    int64_t t0;         // global pass counter at launch (z buffer rotation)
    int64_t iters;      // passes in this launch
    double gamma, eta, inv_m;
    // FP32 splits (hi + lo) of gamma, eta/m and 1 - eta for the FP32 / BF16 path
    float g_hi, g_lo, em_hi, em_lo, e1_hi, e1_lo;
    uint64_t timeout_ns;
    uint32_t barrier_skew;  // test hook: extra arrivals the grid barrier waits for (0 in use)
    // Deterministic reduction (det != 0): each cluster stores its partial z'
    // into zpart[cluster][m][P] (TS) and, after a grid barrier, the partials
    // are summed in cluster order into the z buffer, in place of atomics.
    void *zpart;
    int32_t det;
};

// Device error word values.
enum DevErr : int { DEV_OK = 0, DEV_TIMEOUT_TMA = 1, DEV_TIMEOUT_XCHG = 2, DEV_TIMEOUT_GRID = 3 };

// Launch the persistent iteration kernel.  Returns cudaSuccess or the launch
// error; `clusters` is the grid size in clusters (all co-resident).
cudaError_t launch_iter(int precision, int cpl, const IterArgs &a, int clusters, size_t smem,
                        cudaStream_t s);
// Maximum number of co-resident clusters for a configuration (0 on failure).
int iter_max_clusters(int precision, int cpl, int wpw, int cs, int nw, int rg, size_t smem);
// Minimum ring depth: four stages are in use at a time.
constexpr int kMinStages = 5;
// Dynamic shared memory of one CTA: `slots` worker slots, `stages` ring stages.
size_t iter_smem_bytes(int precision, int P, int slots, int stages, int64_t rows_per_cluster, int rg);
constexpr int kMaxRowsPerGroup = 2;  // rows of Q per pipeline step: 1 or 2
constexpr int kMaxElemWarps = 16;  // warps streaming Q per CTA of the iteration kernel
constexpr int kCtlWarps = 2 * kMaxRowsPerGroup;  // control warps per CTA (at most): per row of
                                   // a group, one for the master's update and one for the
                                   // machines' update
constexpr int kProducerWarps = 1;  // issues the TMA copies of the Q ring
constexpr int kMaxThreads = (kMaxElemWarps + kCtlWarps + kProducerWarps) * 32;

// Kernel entry points, one translation unit per Q precision.
void *iter_kernel_f64(int cpl, int wpw, bool apc, int rg);
void *iter_kernel_f32(int cpl, int wpw, bool apc, int rg);
void *iter_kernel_bf16(int cpl, int wpw, bool apc, int rg);
// ... and with the deterministic reduction (IterArgs::det)
void *iter_kernel_f64_det(int cpl, int wpw, bool apc, int rg);
void *iter_kernel_f32_det(int cpl, int wpw, bool apc, int rg);
void *iter_kernel_bf16_det(int cpl, int wpw, bool apc, int rg);

// ---- setup (FP64) -----------------------------------------------------------
cudaError_t launch_rownorm(const double *A, int64_t lda, int64_t N, int64_t n, double *dinv, int *err,
                           cudaStream_t s);
// G_b = (D X_b)(D X_b)^T for each block b; X rows of block b start at
// X + row_start[b]*ldx; D = dinv (NULL = identity).  G is [m][P][P].
cudaError_t launch_gram(const double *X, int64_t ldx, const int64_t *row_start_dev, const int32_t *p_dev,
                        const double *dinv, int m, int P, int64_t n, double *G, cudaStream_t s);
// In place: G_b = R_b^T R_b (upper R_b over G_b), Rinv_b = R_b^{-1}.  err[0]
// receives 1 + (first singular block) when a pivot is below pivot_tol.
cudaError_t launch_chol(double *G, double *Rinv, const int32_t *p_dev, int m, int P, double pivot_tol,
                        int *err, cudaStream_t s);
// QT_b[c][j] = sum_{r<=c} Rinv_b[r][c] d_r X_b[r][j]  (QT is [m][P][n]).
cudaError_t launch_qt(const double *X, int64_t ldx, const int64_t *row_start_dev, const int32_t *p_dev,
                      const double *dinv, const double *Rinv, int m, int P, int64_t n, double *QT,
                      cudaStream_t s);
// Q[j][b][c] = (TQ) QT_b[c][j]
cudaError_t launch_pack(const double *QT, int m, int P, int64_t n, int precision, void *Q, cudaStream_t s);
// c_b = Rinv2_b^T Rinv1_b^T (d .* rhs_b), written as TS into z[b][P] (zero padded).
cudaError_t launch_csolve(const double *rhs, const int64_t *row_start_dev, const int32_t *p_dev,
                          const double *dinv, const double *Rinv1, const double *Rinv2, int m, int P,
                          int precision, void *z, cudaStream_t s);
// db_b = d .* (Rinv1_b (Rinv2_b v_b)) with v read from z[b][P] (TS).
cudaError_t launch_bsolve(const void *z, const int64_t *row_start_dev, const int32_t *p_dev,
                          const double *dinv, const double *Rinv1, const double *Rinv2, int m, int P,
                          int precision, double *db, cudaStream_t s);
// sums[0] += sum_b ||D_b^{-1} R1_b^T R2_b^T z_b||^2 (z: TS [m][P], the state's
// precision: 0 = FP64, 1 = FP32; R1, R2 the Cholesky factors [m][P][P]).
cudaError_t launch_monitor(const void *z, int precision, const int64_t *row_start_dev, const int32_t *p_dev,
                           const double *dinv, const double *R1, const double *R2, int m, int P, double *sums,
                           cudaStream_t s);
// sums[0] += ||v||^2 (FP64).
cudaError_t launch_sumsq(const double *v, int64_t count, double *sums, cudaStream_t s);
// out = rhs - A x (FP64); sums[0] += ||out||^2, sums[1] += ||rhs||^2.
cudaError_t launch_residual(const double *A, int64_t lda, int64_t N, int64_t n, const double *x,
                            const double *rhs, double *out, double *sums, cudaStream_t s);
// Conversions between the state type and FP64.
cudaError_t launch_to_f64(const void *src, int precision, int64_t count, double *dst, cudaStream_t s);
cudaError_t launch_from_f64(const double *src, int precision, int64_t count, void *dst, cudaStream_t s);
// x_i rows of the [n][m] state into an m x n FP64 matrix (ld >= n).
cudaError_t launch_unpack_x(const void *xw, int precision, int64_t n, int m, double *out, int64_t ld,
                            cudaStream_t s);
// out[j*ldq + c] = Q[j][b][c] for c < p (FP64), one block b.
cudaError_t launch_get_basis(const void *Q, int precision, int64_t n, int m, int P, int b, int p, double *out,
                             int64_t ldq, cudaStream_t s);
cudaError_t launch_axpy_f64(double *y, const double *x, double a, int64_t count, cudaStream_t s);
// acc[0] += sum (lam + em lbar) . (x1 - x0) over the [n][m] states,
// acc[1] += lbar . (mean_i x1 - xb0)   (precision: 0 = FP64 states, 1 = FP32)
cudaError_t launch_adj_dots(const void *lam, const double *lbar, const void *x1, const void *x0, const double *xb0,
                            int64_t n, int m, double em, int precision, double *acc, cudaStream_t s);
cudaError_t launch_gather_rows(const double *A, int64_t lda, int64_t N, int64_t n, const int64_t *perm,
                               double *out, cudaStream_t s);
// gather (scatter = 0): out[k] = v[perm[k]];  scatter (1): out[perm[k]] = v[k]
cudaError_t launch_permute_vec(const double *v, const int64_t *perm, int64_t N, int scatter, double *out,
                               cudaStream_t s);
// flags[0] |= 1 if any of v[0..count) is not finite.
cudaError_t launch_check_finite(const double *v, int64_t count, int *flag, cudaStream_t s);

}  // namespace apc
