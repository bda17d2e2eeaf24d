// The solver context (include/apc.h's opaque apc_ctx), shared by the
// translation units that implement the C ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

struct apc_ctx {
    int device = 0;
    int precision = APC_F32;
    int64_t N = 0, n = 0;
    int m = 0, P = 0, cpl = 0;
    std::vector<int64_t> offs;
    int64_t *d_rowstart = nullptr;   // block b starts at row offs[b]
    int32_t *d_p = nullptr;          // rows per block
    double *A = nullptr, *b = nullptr, *dinv = nullptr;
    double *Rinv1 = nullptr, *Rinv2 = nullptr;
    double *R1 = nullptr, *R2 = nullptr;  // the two Cholesky factors (free residual monitor)
    void *Q = nullptr;
    void *xw = nullptr, *zbuf = nullptr;
    double *xbar = nullptr;  // master estimate, FP64 in every mode
    uint32_t *bar = nullptr;
    int *err = nullptr;
    double *sums = nullptr, *xtmp = nullptr, *rtmp = nullptr, *xacc = nullptr, *rhs = nullptr;
    int cs = 1, nw = 1, wpw = 1, rg = 2, stages = 2, clusters = 1;
    int64_t rows_per_cluster = 1;
    size_t smem = 0;
    int64_t t = 0;   // global pass counter (z buffer rotation)
    double timeout_s = 2.0;
    uint32_t test_barrier_skew = 0;
    size_t q_bytes = 0;
    int qr_passes = 2;          // Cholesky-QR passes taken at set-up (1 or 2)
    double orth_probe = -1.0;   // the first pass's probed departure from orthogonality (-1: not probed)
    void *zpart = nullptr;      // deterministic reduction: per-cluster partial z' [clusters][m][P]
    int det = 0;
    int64_t *d_perm = nullptr;  // apc_setup_rows: row k of the blocked system is row d_perm[k] of the caller's
    // k right-hand sides at once (apc_forward_rhs / apc_backward_rhs on a BF16
    // square context): a one-system batch on the tensor cores, built on first use
    struct apc_batch *mrhs = nullptr;
    int mrhs_k = 0;
    double mrhs_gamma = 0.0, mrhs_eta = 0.0;  // the parameters last uploaded to mrhs
    bool mrhs_params_set = false;
    double *mrhs_in = nullptr, *mrhs_out = nullptr;  // n x k staging, leading dimension k
    std::string last_error;
};

namespace apc {
// Frees what apc_forward_rhs / apc_backward_rhs built (apc_batch.cu).
void destroy_multi_rhs(apc_ctx *c);
// Device element sizes of Q and of the iteration state for a precision.
inline size_t q_elem_bytes(int precision) { return precision == 0 ? 8 : (precision == 1 ? 4 : 2); }
inline size_t s_elem_bytes(int precision) { return precision == 0 ? 8 : 4; }
}  // namespace apc
