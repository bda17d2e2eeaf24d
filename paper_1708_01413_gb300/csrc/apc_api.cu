// C ABI of the APC solver (include/apc.h): context set-up, the solve loop
// with optional FP64 iterative refinement, and residual checks.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <utility>
#include <vector>

#include "../../include/apc.h"
#include "apc_ctx.h"
#include "apc_internal.h"

using namespace apc;

namespace apc {
// Departure from orthogonality of each block's basis from a Cholesky-QR pass
// (QT: [m][P][n] FP64, Q_b = QT_b^T) along a fixed +-1 vector: err[b] =
// ||Q_b^T Q_b v - v|| / ||v||.  Y: m x n FP64 scratch (apc_setup.cu).
cudaError_t launch_orth_probe(const double *QT, const int32_t *p_dev, int m, int P, int64_t n, double *Y, double *err,
                              cudaStream_t s);
// R_b = I for every block ([m][P][P], zero padding).
cudaError_t launch_identity(double *R, const int32_t *p_dev, int m, int P, cudaStream_t s);
}  // namespace apc


namespace {

thread_local std::string g_setup_error;

int fail(apc_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->last_error = buf;
    else g_setup_error = buf;
    return code;
}

#define CK(ctx, call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail((ctx), APC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

size_t q_elem_size(int precision) { return precision == APC_F64 ? 8 : (precision == APC_F32 ? 4 : 2); }
size_t s_elem_size(int precision) { return precision == APC_F64 ? 8 : 4; }
int state_prec(int precision) { return precision == APC_F64 ? 0 : 1; }

template <typename T>
int dalloc(apc_ctx *ctx, T **p, size_t bytes) {
    if (cudaMalloc(reinterpret_cast<void **>(p), bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, APC_ERR_NOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    return APC_OK;
}

void free_all(apc_ctx *c) {
    void *ps[] = {c->d_rowstart, c->d_p, c->A, c->b, c->dinv, c->Rinv1, c->Rinv2, c->R1, c->R2, c->Q, c->xw,
                  c->xbar, c->zbuf, c->bar, c->err, c->sums, c->xtmp, c->rtmp, c->xacc, c->rhs, c->d_perm,
                  c->zpart};
    for (void *p : ps)
        if (p) cudaFree(p);
}

// Pick cluster size, rows per pipeline step, workers per warp, warps per CTA,
// ring depth and grid for the iteration kernel.  Every CTA of a cluster gets
// W = ceil(m / cs) worker slots; a stage holds R rows of W * P elements of Q.
int configure(apc_ctx *c, int cs_request, int wpw_request, int rg_request) {
    int dev_sms = 0;
    CK(c, cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device));
    int smem_optin = 0;
    CK(c, cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    const size_t qsz = q_elem_size(c->precision);
    const size_t budget = size_t(smem_optin) - 2 * 1024;
    // The smallest cluster whose CTAs hold at most 32 worker slots each: fewer
    // CTAs per row range means fewer cluster exchanges per row and more work
    // per pipeline step (sizes need not be powers of two; 8 is the portable
    // maximum).  At one cluster size two rows per step are preferred; one row
    // per step halves the stages, which lets FP32 Q (twice the bytes of BF16)
    // use the same cluster size as BF16 with a full ring.
    for (int cs = 1; cs <= 8; ++cs) {
        if (cs_request > 0 && cs != cs_request) continue;
        for (int R = kMaxRowsPerGroup; R >= 1; --R) {
            if (rg_request > 0 && R != rg_request) continue;
            const int W0 = (c->m + cs - 1) / cs;
            // Four workers per element warp (8 element warps for 32 slots) when
            // the CTA has at least 16: each warp's fixed cost per step (waits,
            // barrier, addressing) is shared by more workers, and the control
            // warps compete with fewer warps for issue slots.
            const int wpw = wpw_request > 0 ? wpw_request
                                            : (c->precision != APC_F64 && W0 >= 16) ? 4 : (W0 >= 2 ? 2 : 1);
            if (wpw != 1 && wpw != 2 && wpw != 4) continue;
            if (wpw == 4 && c->precision == APC_F64) continue;
            const int nw = (W0 + wpw - 1) / wpw;
            const int W = nw * wpw;  // worker slots per CTA
            if (W > 32 || nw > kMaxElemWarps || (cs - 1) * W >= c->m) continue;
            const size_t stage = size_t(R) * W * c->P * qsz;
            // clusters that fit with the smallest ring, then the deepest ring that fits
            int64_t clusters = std::min<int64_t>(std::max(1, dev_sms / cs), (c->n + R - 1) / R);
            int stages = 0;
            size_t smem = 0;
            bool ok = false;
            for (int pass = 0; pass < 4 && !ok; ++pass) {
                const int64_t rpc = (c->n + clusters - 1) / clusters;
                const size_t fixed = iter_smem_bytes(c->precision, c->P, W, 0, rpc, R);
                if (fixed + size_t(kMinStages) * stage > budget) break;
                stages = int(std::min<size_t>(6, (budget - fixed) / stage));
                smem = iter_smem_bytes(c->precision, c->P, W, stages, rpc, R);
                const int maxc = iter_max_clusters(c->precision, c->cpl, wpw, cs, nw, R, smem);
                if (maxc <= 0) break;
                if (maxc >= clusters) ok = true;
                else clusters = maxc;
            }
            if (!ok) continue;
            c->cs = cs;
            c->rg = R;
            c->wpw = wpw;
            c->nw = nw;
            c->stages = stages;
            c->clusters = int(clusters);
            c->rows_per_cluster = (c->n + clusters - 1) / clusters;
            c->smem = smem;
            return APC_OK;
        }
    }
    return fail(c, APC_ERR_UNSUPPORTED,
                "no launch configuration fits m=%d blocks of width %d, n=%lld (requested cs=%d wpw=%d rows=%d)", c->m,
                c->P, (long long)c->n, cs_request, wpw_request, rg_request);
}

// Device-side wait that timed out, if any (then cleared): APC_OK or TIMEOUT.
// Synchronises the stream.
int check_device_error(apc_ctx *c, cudaStream_t s) {
    int herr = 0;
    CK(c, cudaMemcpyAsync(&herr, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    if (herr != 0) {
        cudaMemsetAsync(c->err, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
        static const char *what[] = {"", "TMA stage", "cluster exchange", "grid barrier"};
        return fail(c, APC_ERR_TIMEOUT, "device wait timed out (%s)", what[herr >= 1 && herr <= 3 ? herr : 0]);
    }
    return APC_OK;
}

// `iters` passes of the iteration kernel in `mode`.  With check (the public
// calls) the stream is synchronised after each launch and a device-side
// timeout is reported at once; without it the launches only queue (a caller
// that runs many short passes, the Lanczos process, checks once at its end
// with check_device_error; every wait in the kernel is bounded, so passes
// after a timed-out one still end).
int run_pass(apc_ctx *c, int mode, double gamma, double eta, int64_t iters, cudaStream_t s, bool check = true) {
    const int64_t chunk_max = 1 << 20;
    while (iters > 0) {
        const int64_t it = std::min(iters, chunk_max);
        IterArgs a = {};
        a.Q = c->Q;
        a.xw = c->xw;
        a.xbar = c->xbar;
        a.zbuf = c->zbuf;
        a.bar = c->bar;
        a.err = c->err;
        a.n = c->n;
        a.m = c->m;
        a.P = c->P;
        a.cs = c->cs;
        a.nw = c->nw;
        a.wpw = c->wpw;
        a.rg = c->rg;
        a.stages = c->stages;
        a.mode = mode;
        a.rows_per_cluster = c->rows_per_cluster;
        a.t0 = c->t;
        a.iters = it;
        a.gamma = gamma;
        a.eta = eta;
        a.inv_m = 1.0 / c->m;
        auto split = [](double v, float &hi, float &lo) {
            hi = float(v);
            lo = float(v - double(hi));
        };
        split(gamma, a.g_hi, a.g_lo);
        split(eta / c->m, a.em_hi, a.em_lo);
        split(1.0 - eta, a.e1_hi, a.e1_lo);
        a.timeout_ns = uint64_t(c->timeout_s * 1e9);
        a.barrier_skew = c->test_barrier_skew;
        a.zpart = c->zpart;
        a.det = c->det;
        CK(c, cudaMemsetAsync(c->bar, 0, sizeof(uint32_t), s));
        cudaError_t e = launch_iter(c->precision, c->cpl, a, c->clusters, c->smem, s);
        if (e != cudaSuccess) return fail(c, APC_ERR_LAUNCH, "iteration kernel launch failed: %s", cudaGetErrorString(e));
        c->t += it;
        iters -= it;
        if (check) {
            const int rc = check_device_error(c, s);
            if (rc != APC_OK) return rc;
        }
    }
    return APC_OK;
}

// Free residual monitor of the current xbar: sqrt(sum_b ||D^{-1} R'^T z_b||^2) /
// ||rhs|| with z the coefficients of the next pass (see launch_monitor) and
// rhs the right-hand side of the last reset.
int monitor(apc_ctx *c, double *rel, cudaStream_t s) {
    if (c->t == 0) return fail(c, APC_ERR_INVALID_ARG, "no forward iteration state (apc_reset first)");
    const size_t ssz = s_elem_size(c->precision);
    const void *z = static_cast<const char *>(c->zbuf) + ssz * size_t(c->t % 3) * c->m * c->P;
    CK(c, cudaMemsetAsync(c->sums + 3, 0, sizeof(double), s));
    CK(c, launch_monitor(z, state_prec(c->precision), c->d_rowstart, c->d_p, c->dinv, c->R1, c->R2, c->m, c->P,
                         c->sums + 3, s));
    double h[2];
    CK(c, cudaMemcpyAsync(h, c->sums + 2, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    *rel = h[0] > 0 ? std::sqrt(h[1] / h[0]) : std::sqrt(h[1]);
    return APC_OK;
}

int residual(apc_ctx *c, const double *x, const double *rhs, double *out, double *rel, cudaStream_t s) {
    CK(c, cudaMemsetAsync(c->sums, 0, 2 * sizeof(double), s));
    CK(c, launch_residual(c->A, c->n, c->N, c->n, x, rhs, out, c->sums, s));
    double h[2];
    CK(c, cudaMemcpyAsync(h, c->sums, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    *rel = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return APC_OK;
}

}  // namespace

namespace {
int reset_blocked(apc_ctx *c, const double *rhs_dev, cudaStream_t s);
}

namespace apc {
// Error text for entry points that have no context (read by apc_last_error(NULL)).
void set_global_error_text(const char *msg) { g_setup_error = msg; }
// `iters` passes of the iteration kernel in `mode` (used by apc_spectral.cu)
int pass(apc_ctx *c, int mode, double gamma, double eta, int64_t iters, cudaStream_t s) {
    return run_pass(c, mode, gamma, eta, iters, s);
}
int pass_queued(apc_ctx *c, int mode, double gamma, double eta, int64_t iters, cudaStream_t s) {
    return run_pass(c, mode, gamma, eta, iters, s, false);
}
int device_error(apc_ctx *c, cudaStream_t s) { return check_device_error(c, s); }
}  // namespace apc

extern "C" {

int apc_setup_rows(apc_ctx **out, const double *A_dev, int64_t N, int64_t n, int64_t lda, const double *b_dev,
                   const int64_t *row_index_host, const int64_t *row_offsets_host, int32_t m, const apc_options *opt,
                   void *stream) {
    if (!out) return fail(nullptr, APC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!A_dev || !b_dev || !row_index_host || !row_offsets_host || N < 1 || n < 1 || lda < n)
        return fail(nullptr, APC_ERR_INVALID_ARG, "apc_setup_rows: NULL argument or bad size");
    // row_index must list every row exactly once
    std::vector<char> seen(size_t(N), 0);
    for (int64_t k = 0; k < N; ++k) {
        const int64_t r = row_index_host[k];
        if (r < 0 || r >= N || seen[size_t(r)])
            return fail(nullptr, APC_ERR_INVALID_ARG, "apc_setup_rows: row_index is not a permutation of 0..N-1");
        seen[size_t(r)] = 1;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t *d_perm = nullptr;
    double *Ag = nullptr, *bg = nullptr;
    auto release = [&]() {
        if (d_perm) cudaFree(d_perm);
        if (Ag) cudaFree(Ag);
        if (bg) cudaFree(bg);
    };
    if (cudaMalloc(&d_perm, sizeof(int64_t) * N) != cudaSuccess || cudaMalloc(&Ag, sizeof(double) * N * n) != cudaSuccess ||
        cudaMalloc(&bg, sizeof(double) * N) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(nullptr, APC_ERR_NOMEM, "apc_setup_rows: cudaMalloc failed");
    }
    if (cudaMemcpyAsync(d_perm, row_index_host, sizeof(int64_t) * N, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        launch_gather_rows(A_dev, lda, N, n, d_perm, Ag, s) != cudaSuccess ||
        launch_permute_vec(b_dev, d_perm, N, 0, bg, s) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(nullptr, APC_ERR_CUDA, "apc_setup_rows: gather failed");
    }
    // the blocked system's rows are contiguous: factor it as usual (its copy of A
    // and b, in the blocked order, serves the residuals)
    const int rc = apc_setup(out, Ag, N, n, n, bg, row_offsets_host, m, opt, stream);
    cudaStreamSynchronize(s);
    cudaFree(Ag);
    cudaFree(bg);
    Ag = bg = nullptr;
    if (rc != APC_OK) {
        release();
        return rc;
    }
    (*out)->d_perm = d_perm;
    return APC_OK;
}

int apc_hb_optimal_params(double mu_min, double mu_max, int32_t m, double *alpha, double *beta, double *rho) {
    if (!(mu_min > 0.0) || !(mu_min <= mu_max) || !(mu_max <= 1.0 + 1e-12) || m < 1 || !alpha || !beta || !rho)
        return fail(nullptr, APC_ERR_INVALID_ARG, "need 0 < mu_min <= mu_max <= 1, m >= 1 and non-NULL outputs");
    // Hessian of the preconditioned least squares: C^T C = m X, spectrum [m mu_min, m mu_max]
    const double a = std::sqrt(m * mu_max), c = std::sqrt(m * mu_min);
    *alpha = 4.0 / ((a + c) * (a + c));
    *rho = (a - c) / (a + c);
    *beta = (*rho) * (*rho);
    return APC_OK;
}

int apc_optimal_params(double mu_min, double mu_max, double *gamma, double *eta, double *rho) {
    if (!(mu_min > 0.0) || !(mu_min <= mu_max) || !(mu_max <= 1.0 + 1e-12))
        return fail(nullptr, APC_ERR_INVALID_ARG, "need 0 < mu_min <= mu_max <= 1 (got %g, %g)", mu_min, mu_max);
    const double smin = std::sqrt(mu_min), smax = std::sqrt(std::min(mu_max, 1.0));
    const double s = 4.0 / ((smax + smin) * (smax + smin));
    const double r = (smax - smin) / (smax + smin);
    const double tr = s + 1.0 - r * r;
    const double disc = std::max(tr * tr - 4.0 * s, 0.0);
    if (gamma) *gamma = (tr - std::sqrt(disc)) / 2.0;
    if (eta) *eta = (tr + std::sqrt(disc)) / 2.0;
    if (rho) *rho = r;
    return APC_OK;
}

int apc_setup(apc_ctx **out, const double *A_dev, int64_t N, int64_t n, int64_t lda, const double *b_dev,
              const int64_t *row_offsets_host, int32_t m, const apc_options *opt, void *stream) {
    if (!out) return fail(nullptr, APC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!A_dev || !b_dev || !row_offsets_host) return fail(nullptr, APC_ERR_INVALID_ARG, "NULL input pointer");
    if (n < 1 || N < n || lda < n) return fail(nullptr, APC_ERR_INVALID_ARG, "need N >= n >= 1 and lda >= n");
    if (m < 1 || m > 256) return fail(nullptr, APC_ERR_UNSUPPORTED, "m=%d outside 1..256", m);
    const int precision = opt ? opt->precision : APC_F32;
    if (precision < APC_F64 || precision > APC_BF16) return fail(nullptr, APC_ERR_INVALID_ARG, "bad precision");
    if (opt && (opt->rows_per_group < 0 || opt->rows_per_group > 2))
        return fail(nullptr, APC_ERR_INVALID_ARG, "rows_per_group=%d: 0 (automatic), 1 or 2", opt->rows_per_group);
    if (row_offsets_host[0] != 0 || row_offsets_host[m] != N)
        return fail(nullptr, APC_ERR_INVALID_ARG, "row_offsets must start at 0 and end at N");
    int64_t pmax = 0;
    for (int i = 0; i < m; ++i) {
        const int64_t p = row_offsets_host[i + 1] - row_offsets_host[i];
        if (p < 1) return fail(nullptr, APC_ERR_INVALID_ARG, "block %d is empty or offsets decrease", i);
        if (p > n) return fail(nullptr, APC_ERR_SINGULAR_BLOCK, "block %d has %lld rows > n", i, (long long)p);
        pmax = std::max(pmax, p);
    }
    if (pmax > 256) return fail(nullptr, APC_ERR_UNSUPPORTED, "block of %lld rows; at most 256", (long long)pmax);

    apc_ctx *c = new apc_ctx();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto bail = [&](int code) {
        g_setup_error = c->last_error;
        free_all(c);
        delete c;
        return code;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        fail(c, APC_ERR_CUDA, "no CUDA device");
        return bail(APC_ERR_CUDA);
    }
    c->precision = precision;
    c->N = N;
    c->n = n;
    c->m = m;
    c->P = pmax <= 64 ? 64 : pmax <= 128 ? 128 : 256;
    c->cpl = c->P / 32;
    c->timeout_s = (opt && opt->timeout_s > 0) ? opt->timeout_s : 2.0;
    c->offs.assign(row_offsets_host, row_offsets_host + m + 1);
    const size_t P = c->P;
    int rc;
#define ALLOC(ptr, bytes) \
    if ((rc = dalloc(c, &(ptr), (bytes))) != APC_OK) return bail(rc)
    ALLOC(c->d_rowstart, sizeof(int64_t) * m);
    ALLOC(c->d_p, sizeof(int32_t) * m);
    ALLOC(c->A, sizeof(double) * N * n);
    ALLOC(c->b, sizeof(double) * N);
    ALLOC(c->dinv, sizeof(double) * N);
    ALLOC(c->Rinv1, sizeof(double) * m * P * P);
    ALLOC(c->Rinv2, sizeof(double) * m * P * P);
    ALLOC(c->R1, sizeof(double) * m * P * P);
    ALLOC(c->R2, sizeof(double) * m * P * P);
    ALLOC(c->err, sizeof(int) * 4);
    ALLOC(c->bar, sizeof(uint32_t) * 4);
    ALLOC(c->sums, sizeof(double) * 4);
    ALLOC(c->xtmp, sizeof(double) * n);
    ALLOC(c->xacc, sizeof(double) * n);
    ALLOC(c->rtmp, sizeof(double) * N);
    ALLOC(c->rhs, sizeof(double) * N);
    std::vector<int64_t> rs(m);
    std::vector<int32_t> pc(m);
    for (int i = 0; i < m; ++i) {
        rs[i] = row_offsets_host[i];
        pc[i] = int32_t(row_offsets_host[i + 1] - row_offsets_host[i]);
    }
#define CKB(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            fail(c, APC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));             \
            return bail(APC_ERR_CUDA);                                                         \
        }                                                                                      \
    } while (0)
    CKB(cudaMemcpyAsync(c->d_rowstart, rs.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    CKB(cudaMemcpyAsync(c->d_p, pc.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    CKB(cudaMemcpy2DAsync(c->A, sizeof(double) * n, A_dev, sizeof(double) * lda, sizeof(double) * n, N,
                          cudaMemcpyDeviceToDevice, s));
    CKB(cudaMemcpyAsync(c->b, b_dev, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    CKB(cudaMemsetAsync(c->err, 0, sizeof(int) * 4, s));

    // non-finite inputs
    CKB(launch_check_finite(c->A, N * n, c->err + 1, s));
    CKB(launch_check_finite(c->b, N, c->err + 1, s));
    CKB(launch_rownorm(c->A, n, N, n, c->dinv, c->err, s));
    int herr[4];
    CKB(cudaMemcpyAsync(herr, c->err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    CKB(cudaStreamSynchronize(s));
    if (herr[1]) {
        fail(c, APC_ERR_NONFINITE, "A or b holds NaN or Inf");
        return bail(APC_ERR_NONFINITE);
    }
    if (herr[0]) {
        fail(c, APC_ERR_SINGULAR_BLOCK, "A has a zero row");
        return bail(APC_ERR_SINGULAR_BLOCK);
    }

    // two passes of Cholesky QR in FP64 (scratch freed at the end)
    double *G = nullptr, *QT1 = nullptr, *QT2 = nullptr;
    int64_t *rs2 = nullptr;
    auto free_scratch = [&]() {
        if (G) cudaFree(G);
        if (QT1) cudaFree(QT1);
        if (QT2) cudaFree(QT2);
        if (rs2) cudaFree(rs2);
    };
    auto bail2 = [&](int code) {
        free_scratch();
        return bail(code);
    };
    if (dalloc(c, &G, sizeof(double) * m * P * P) || dalloc(c, &QT1, sizeof(double) * m * P * n) ||
        dalloc(c, &QT2, sizeof(double) * m * P * n) || dalloc(c, &rs2, sizeof(int64_t) * m))
        return bail2(APC_ERR_NOMEM);
    for (int i = 0; i < m; ++i) rs[i] = int64_t(i) * P;
#define CKB2(call)                                                                             \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            fail(c, APC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));             \
            return bail2(APC_ERR_CUDA);                                                        \
        }                                                                                      \
    } while (0)
    CKB2(cudaMemcpyAsync(rs2, rs.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    CKB2(cudaMemsetAsync(G, 0, sizeof(double) * m * P * P, s));
    CKB2(launch_gram(c->A, n, c->d_rowstart, c->d_p, c->dinv, m, int(P), n, G, s));
    CKB2(launch_chol(G, c->Rinv1, c->d_p, m, int(P), 1e-14, c->err + 2, s));
    CKB2(cudaMemcpyAsync(c->R1, G, sizeof(double) * m * P * P, cudaMemcpyDeviceToDevice, s));
    CKB2(launch_qt(c->A, n, c->d_rowstart, c->d_p, c->dinv, c->Rinv1, m, int(P), n, QT1, s));
    // The second pass restores orthogonality lost to rounding in the first
    // (about u kappa(A_i)^2).  FP64 contexts always take it.  FP32 and BF16
    // contexts store Q rounded to 2^-24 or 2^-9, so a first pass whose basis
    // is orthonormal to far below that is kept: a probe measures
    // ||Q_i^T Q_i v - v|| / ||v|| for every block (two reads of the basis,
    // against p_i + 1 for a second pass) and the pass is left out when the
    // largest is below 1e-11 (FP32) or 1e-8 (BF16).
    bool second_pass = true;
    c->orth_probe = -1.0;
    if (precision != APC_F64) {
        CKB2(launch_orth_probe(QT1, c->d_p, m, int(P), n, QT2, G, s));
        std::vector<double> perr(m);
        CKB2(cudaMemcpyAsync(perr.data(), G, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
        CKB2(cudaStreamSynchronize(s));
        double worst = 0.0;
        for (double e : perr) worst = std::isfinite(e) ? std::max(worst, e) : 1e300;
        c->orth_probe = worst;
        second_pass = !(worst <= (precision == APC_F32 ? 1e-11 : 1e-8));
    }
    if (second_pass) {
        CKB2(cudaMemsetAsync(G, 0, sizeof(double) * m * P * P, s));
        CKB2(launch_gram(QT1, n, rs2, c->d_p, nullptr, m, int(P), n, G, s));
        CKB2(launch_chol(G, c->Rinv2, c->d_p, m, int(P), 1e-14, c->err + 3, s));
        CKB2(cudaMemcpyAsync(c->R2, G, sizeof(double) * m * P * P, cudaMemcpyDeviceToDevice, s));
        CKB2(launch_qt(QT1, n, rs2, c->d_p, nullptr, c->Rinv2, m, int(P), n, QT2, s));
    } else {
        CKB2(launch_identity(c->Rinv2, c->d_p, m, int(P), s));
        CKB2(launch_identity(c->R2, c->d_p, m, int(P), s));
    }
    c->qr_passes = second_pass ? 2 : 1;
    c->q_bytes = size_t(n) * m * P * q_elem_size(precision);
    if (dalloc(c, &c->Q, c->q_bytes)) return bail2(APC_ERR_NOMEM);
    CKB2(launch_pack(second_pass ? QT2 : QT1, m, int(P), n, precision, c->Q, s));
    CKB2(cudaMemcpyAsync(herr, c->err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    CKB2(cudaStreamSynchronize(s));
    free_scratch();
    G = QT1 = QT2 = nullptr;
    rs2 = nullptr;
    if (herr[2] || herr[3]) {
        const int blk = (herr[2] ? herr[2] : herr[3]) - 1;
        fail(c, APC_ERR_SINGULAR_BLOCK, "block %d: A_i A_i^T is numerically singular (Cholesky pivot)", blk);
        return bail(APC_ERR_SINGULAR_BLOCK);
    }

    const size_t ssz = s_elem_size(precision);
    ALLOC(c->xw, ssz * n * m);
    ALLOC(c->xbar, sizeof(double) * n);
    ALLOC(c->zbuf, ssz * 3 * m * P);
    CKB(cudaMemsetAsync(c->xw, 0, ssz * n * m, s));
    CKB(cudaMemsetAsync(c->xbar, 0, sizeof(double) * n, s));
    CKB(cudaMemsetAsync(c->zbuf, 0, ssz * 3 * m * P, s));
    CKB(cudaMemsetAsync(c->err, 0, sizeof(int) * 4, s));
    if ((rc = configure(c, opt ? opt->cluster_size : 0, opt ? opt->workers_per_warp : 0,
                        opt ? opt->rows_per_group : 0)) != APC_OK)
        return bail(rc);
    CKB(cudaStreamSynchronize(s));
    *out = c;
    return APC_OK;
#undef ALLOC
#undef CKB
#undef CKB2
}

int apc_reset(apc_ctx *c, const double *rhs_dev, void *stream) {
    if (!c) return fail(nullptr, APC_ERR_INVALID_ARG, "NULL context");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (rhs_dev && c->d_perm) {  // caller's row order -> the blocked order
        CK(c, launch_permute_vec(rhs_dev, c->d_perm, c->N, 0, c->rtmp, s));
        rhs_dev = c->rtmp;
    }
    return reset_blocked(c, rhs_dev, s);
}

}  // extern "C"

namespace {
// apc_reset with the right-hand side already in the blocked row order
int reset_blocked(apc_ctx *c, const double *rhs_dev, cudaStream_t s) {
    const size_t ssz = s_elem_size(c->precision);
    const double *rhs = rhs_dev ? rhs_dev : c->b;
    CK(c, cudaMemsetAsync(c->zbuf, 0, ssz * 3 * c->m * c->P, s));
    CK(c, cudaMemsetAsync(c->xbar, 0, sizeof(double) * c->n, s));
    CK(c, launch_csolve(rhs, c->d_rowstart, c->d_p, c->dinv, c->Rinv1, c->Rinv2, c->m, c->P,
                        state_prec(c->precision), c->zbuf, s));
    CK(c, cudaMemsetAsync(c->sums + 2, 0, sizeof(double), s));  // ||rhs||^2 for the monitor
    CK(c, launch_sumsq(rhs, c->N, c->sums + 2, s));
    c->t = 0;
    return run_pass(c, MODE_INIT, 1.0, 1.0, 1, s);
}
}  // namespace

extern "C" {

int apc_iterate(apc_ctx *c, double gamma, double eta, int64_t iters, void *stream) {
    if (!c) return fail(nullptr, APC_ERR_INVALID_ARG, "NULL context");
    if (!(gamma > 0.0 && gamma < 2.0) || !std::isfinite(eta))
        return fail(c, APC_ERR_PARAMS, "gamma=%g must lie in (0, 2) and eta must be finite", gamma);
    if (iters < 0) return fail(c, APC_ERR_INVALID_ARG, "iters < 0");
    if (iters == 0) return APC_OK;
    if (c->t == 0) return fail(c, APC_ERR_INVALID_ARG, "apc_reset must precede apc_iterate");
    return run_pass(c, MODE_APC, gamma, eta, iters, static_cast<cudaStream_t>(stream));
}

int apc_get_xbar(apc_ctx *c, double *x_dev, void *stream) {
    if (!c || !x_dev) return fail(c, APC_ERR_INVALID_ARG, "NULL argument");
    CK(c, cudaMemcpyAsync(x_dev, c->xbar, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
    return APC_OK;
}

int apc_get_x(apc_ctx *c, double *x_dev, int64_t ldx, void *stream) {
    if (!c || !x_dev || ldx < c->n) return fail(c, APC_ERR_INVALID_ARG, "bad argument");
    CK(c, launch_unpack_x(c->xw, state_prec(c->precision), c->n, c->m, x_dev, ldx, static_cast<cudaStream_t>(stream)));
    return APC_OK;
}

int apc_get_basis(apc_ctx *c, int32_t block, double *Q_dev, int64_t ldq, void *stream) {
    if (!c || !Q_dev || block < 0 || block >= c->m) return fail(c, APC_ERR_INVALID_ARG, "bad argument");
    const int p = int(c->offs[block + 1] - c->offs[block]);
    if (ldq < p) return fail(c, APC_ERR_INVALID_ARG, "ldq < p_i");
    CK(c, launch_get_basis(c->Q, c->precision, c->n, c->m, c->P, block, p, Q_dev, ldq,
                           static_cast<cudaStream_t>(stream)));
    return APC_OK;
}

int apc_residual(apc_ctx *c, const double *x_dev, const double *rhs_dev, double *resid_dev, double *rel_host,
                 void *stream) {
    if (!c || !x_dev || !rel_host) return fail(c, APC_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!c->d_perm)
        return residual(c, x_dev, rhs_dev ? rhs_dev : c->b, resid_dev ? resid_dev : c->rtmp, rel_host, s);
    // rows were regrouped by apc_setup_rows: work in the blocked order, return
    // the residual vector in the caller's order
    if (rhs_dev) CK(c, launch_permute_vec(rhs_dev, c->d_perm, c->N, 0, c->rhs, s));
    const int rc = residual(c, x_dev, rhs_dev ? c->rhs : c->b, c->rtmp, rel_host, s);
    if (rc != APC_OK) return rc;
    if (resid_dev) CK(c, launch_permute_vec(c->rtmp, c->d_perm, c->N, 1, resid_dev, s));
    return APC_OK;
}

int apc_monitor(apc_ctx *c, double *rel_residual_host, void *stream) {
    if (!c || !rel_residual_host) return fail(c, APC_ERR_INVALID_ARG, "NULL argument");
    return monitor(c, rel_residual_host, static_cast<cudaStream_t>(stream));
}

int apc_solve(apc_ctx *c, double gamma, double eta, double tol, int64_t max_iters, int64_t check_every,
              int32_t refine, double *x_dev, apc_stats *stats, void *stream) {
    if (!c || !x_dev) return fail(c, APC_ERR_INVALID_ARG, "NULL argument");
    if (!(gamma > 0.0 && gamma < 2.0)) return fail(c, APC_ERR_PARAMS, "gamma=%g must lie in (0, 2)", gamma);
    if (check_every <= 0) check_every = 100;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const auto t_start = std::chrono::steady_clock::now();
    int64_t iters = 0, rchecks = 0, mchecks = 0;
    int sweeps = 0;
    double rel = 0.0;
    int rc = APC_OK;
    // The free monitor (R'^T z, the invariant of App. A) equals the residual to
    // the precision of the stored bases: FP64 and FP32 contexts use it for the
    // checks between FP64 residuals; BF16 bases (relative error 2^-9) would put
    // its error near 4e-3 of ||b||, so BF16 checks stay FP64 residuals.
    const bool use_monitor = c->precision != APC_BF16;
    const int kFullEvery = 8;  // an FP64 residual at least every 8 monitor checks
    if (!refine) {
        sweeps = 1;
        if ((rc = reset_blocked(c, nullptr, s)) != APC_OK) return rc;
        CK(c, cudaMemcpyAsync(x_dev, c->xbar, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
        if ((rc = residual(c, x_dev, c->b, c->rtmp, &rel, s)) != APC_OK) return rc;
        ++rchecks;
        const double rel0 = rel;
        bool exact = true;  // rel is an FP64 residual of the current xbar (copied to x_dev)
        int since_full = 0;
        rc = APC_ERR_NOT_CONVERGED;
        while (iters < max_iters) {
            if (rel <= tol && exact) { rc = APC_OK; break; }
            const int64_t k = std::min(check_every, max_iters - iters);
            int r2 = run_pass(c, MODE_APC, gamma, eta, k, s);
            if (r2 != APC_OK) return r2;
            iters += k;
            bool full = !use_monitor || iters >= max_iters;
            if (!full) {
                if ((r2 = monitor(c, &rel, s)) != APC_OK) return r2;
                ++mchecks;
                exact = false;
                full = rel <= tol || !std::isfinite(rel) || ++since_full >= kFullEvery;
            }
            if (full) {
                CK(c, cudaMemcpyAsync(x_dev, c->xbar, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
                if ((r2 = residual(c, x_dev, c->b, c->rtmp, &rel, s)) != APC_OK) return r2;
                ++rchecks;
                exact = true;
                since_full = 0;
            }
            if (!std::isfinite(rel)) { rc = fail(c, APC_ERR_NONFINITE, "iterate became non-finite"); break; }
            if (rel > 1e8 * std::max(rel0, 1e-300)) { rc = fail(c, APC_ERR_DIVERGED, "residual grew to %g", rel); break; }
        }
        if (!exact) {
            CK(c, cudaMemcpyAsync(x_dev, c->xbar, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
            if ((rc = residual(c, x_dev, c->b, c->rtmp, &rel, s)) != APC_OK) return rc;
            ++rchecks;
        }
        if (rc == APC_OK || rc == APC_ERR_NOT_CONVERGED) {
            if (rel <= tol) rc = APC_OK;
            else rc = fail(c, APC_ERR_NOT_CONVERGED, "relative residual %g > tol %g after %lld iterations", rel,
                           tol, (long long)iters);
        }
    } else {
        // FP64 iterative refinement: x <- x + delta, A delta ~= r = b - A x by APC
        CK(c, cudaMemsetAsync(c->xacc, 0, sizeof(double) * c->n, s));
        CK(c, cudaMemcpyAsync(c->rhs, c->b, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, s));
        if ((rc = residual(c, c->xacc, c->b, c->rhs, &rel, s)) != APC_OK) return rc;
        ++rchecks;
        rc = APC_ERR_NOT_CONVERGED;
        const int max_sweeps = 64;
        const double best_rate = std::sqrt(std::fabs((gamma - 1.0) * (eta - 1.0)));
        int64_t window = 64 * check_every;
        if (best_rate > 0.0 && best_rate < 1.0)
            window = std::min(window, std::max(check_every, int64_t(std::ceil(std::log(0.1) / std::log(best_rate)))));
        else if (best_rate == 0.0)
            window = check_every;
        std::deque<std::pair<int64_t, double>> hist;  // (iterations, inner residual) of the sweep's checks
        while (iters < max_iters && sweeps < max_sweeps) {
            if (rel <= tol) { rc = APC_OK; break; }
            ++sweeps;
            int r2 = reset_blocked(c, c->rhs, s);
            if (r2 != APC_OK) return r2;
            double inner = 1.0;
            // inner APC on A delta = r; stop when its residual (relative to r)
            // is below 1e-4, stagnates, or suffices for the outer tolerance.
            // "Stagnates": less than a halving over the window in which the
            // parameters' best rate, sqrt|(gamma-1)(eta-1)| (the modulus of the
            // complex roots of Eq. 5; rho itself for Theorem 1's parameters),
            // promises a tenfold drop.  A fixed window would call the slow but
            // steady progress at kappa(X) ~ 1e5 (rho^50 ~ 0.87) a stall and
            // restart the momentum every few checks.
            const int64_t sweep_start = iters;
            hist.clear();
            hist.push_back({iters, inner});
            while (iters < max_iters) {
                const int64_t k = std::min(check_every, max_iters - iters);
                if ((r2 = run_pass(c, MODE_APC, gamma, eta, k, s)) != APC_OK) return r2;
                iters += k;
                if (use_monitor) {
                    if ((r2 = monitor(c, &inner, s)) != APC_OK) return r2;
                    ++mchecks;
                } else {
                    CK(c, cudaMemcpyAsync(c->xtmp, c->xbar, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
                    if ((r2 = residual(c, c->xtmp, c->rhs, c->rtmp, &inner, s)) != APC_OK) return r2;
                    ++rchecks;
                }
                if (!std::isfinite(inner)) return fail(c, APC_ERR_NONFINITE, "inner iterate became non-finite");
                if (inner > 1e8) return fail(c, APC_ERR_DIVERGED, "inner residual grew to %g", inner);
                // the latest check at least `window` iterations back (older
                // ones are no longer needed)
                while (hist.size() >= 2 && iters - hist[1].first >= window) hist.pop_front();
                const double back = (!hist.empty() && iters - hist.front().first >= window) ? hist.front().second : -1.0;
                hist.push_back({iters, inner});
                const bool stalled = back > 0.0 && inner > 0.5 * back && inner < 0.5 && iters - sweep_start >= window;
                if (inner <= 1e-4 || stalled || rel * inner <= 0.5 * tol) break;
            }
            CK(c, cudaMemcpyAsync(c->xtmp, c->xbar, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
            CK(c, launch_axpy_f64(c->xacc, c->xtmp, 1.0, c->n, s));
            if ((r2 = residual(c, c->xacc, c->b, c->rhs, &rel, s)) != APC_OK) return r2;
            ++rchecks;
            if (!std::isfinite(rel)) return fail(c, APC_ERR_NONFINITE, "refined iterate became non-finite");
        }
        CK(c, cudaMemcpyAsync(x_dev, c->xacc, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
        CK(c, cudaStreamSynchronize(s));
        if (rel <= tol) rc = APC_OK;
        else rc = fail(c, APC_ERR_NOT_CONVERGED, "relative residual %g > tol %g after %d sweeps", rel, tol, sweeps);
    }
    if (stats) {
        stats->iterations = iters;
        stats->sweeps = sweeps;
        stats->rel_residual = rel;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        stats->residual_checks = rchecks;
        stats->monitor_checks = mchecks;
    }
    return rc;
}

int apc_solve_rhs(apc_ctx *c, const double *B_dev, int64_t k, int64_t ldb, double gamma, double eta, double tol,
                  int64_t max_iters, int64_t check_every, int32_t refine, double *X_dev, int64_t ldx, apc_stats *stats,
                  void *stream) {
    if (!c || !B_dev || !X_dev || k < 1 || ldb < k || ldx < k)
        return fail(c, APC_ERR_INVALID_ARG, "apc_solve_rhs: bad pointer, k or leading dimension");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the columns one after another through apc_solve, each as the context's
    // right-hand side (the stored b is set aside and put back)
    double *bsave = nullptr, *xcol = nullptr;
    if (cudaMalloc(&bsave, sizeof(double) * c->N) != cudaSuccess ||
        cudaMalloc(&xcol, sizeof(double) * c->n) != cudaSuccess) {
        cudaGetLastError();
        if (bsave) cudaFree(bsave);
        return fail(c, APC_ERR_NOMEM, "apc_solve_rhs: staging buffers");
    }
    apc_stats total = {};
    int rc = APC_OK, worst = APC_OK;
    if (cudaMemcpyAsync(bsave, c->b, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        rc = fail(c, APC_ERR_CUDA, "apc_solve_rhs: copy of b failed");
    for (int64_t j = 0; rc == APC_OK && j < k; ++j) {
        cudaError_t e = cudaMemcpy2DAsync(c->rhs, sizeof(double), B_dev + j, sizeof(double) * ldb, sizeof(double), c->N,
                                          cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && c->d_perm) e = launch_permute_vec(c->rhs, c->d_perm, c->N, 0, c->b, s);
        else if (e == cudaSuccess) e = cudaMemcpyAsync(c->b, c->rhs, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { rc = fail(c, APC_ERR_CUDA, "apc_solve_rhs: column copy failed"); break; }
        apc_stats st = {};
        const int r = apc_solve(c, gamma, eta, tol, max_iters, check_every, refine, xcol, &st, stream);
        if (r != APC_OK && r != APC_ERR_NOT_CONVERGED) { rc = r; break; }
        if (r != APC_OK) worst = r;
        if (cudaMemcpy2DAsync(X_dev + j, sizeof(double) * ldx, xcol, sizeof(double), sizeof(double), c->n,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            rc = fail(c, APC_ERR_CUDA, "apc_solve_rhs: solution copy failed");
            break;
        }
        total.iterations += st.iterations;
        total.sweeps = std::max(total.sweeps, st.sweeps);
        total.rel_residual = std::max(total.rel_residual, st.rel_residual);
        total.seconds += st.seconds;
        total.residual_checks += st.residual_checks;
        total.monitor_checks += st.monitor_checks;
    }
    const std::string msg = c->last_error;
    cudaMemcpyAsync(c->b, bsave, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    cudaFree(bsave);
    cudaFree(xcol);
    c->last_error = msg;
    if (stats) *stats = total;
    return rc != APC_OK ? rc : worst;
}

int apc_backward(apc_ctx *c, const double *g_dev, int64_t T, double gamma, double eta, double *db_dev,
                 void *stream) {
    if (!c || !g_dev || !db_dev || T < 0) return fail(c, APC_ERR_INVALID_ARG, "bad argument");
    if (!(gamma > 0.0 && gamma < 2.0) || !std::isfinite(eta))
        return fail(c, APC_ERR_PARAMS, "gamma=%g must lie in (0, 2) and eta must be finite", gamma);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t ssz = s_elem_size(c->precision);
    // lambda_i = 0, lbar = g, z buffers cleared
    CK(c, cudaMemsetAsync(c->xw, 0, ssz * c->n * c->m, s));
    CK(c, cudaMemsetAsync(c->zbuf, 0, ssz * 3 * c->m * c->P, s));
    CK(c, cudaMemcpyAsync(c->xbar, g_dev, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
    c->t = 0;
    int rc;
    // z = Q_i^T mu_i(T) with mu_i(T) = (eta/m) g
    if ((rc = run_pass(c, MODE_ADJ_SEED, gamma, eta, 1, s)) != APC_OK) return rc;
    if ((rc = run_pass(c, MODE_ADJ, gamma, eta, T, s)) != APC_OK) return rc;
    // v_i = Q_i^T (lambda_i(0) + lbar(0)/m)
    if ((rc = run_pass(c, MODE_ADJ_FINAL, gamma, eta, 1, s)) != APC_OK) return rc;
    const void *v = static_cast<const char *>(c->zbuf) + ssz * size_t(c->t % 3) * c->m * c->P;
    CK(c, launch_bsolve(v, c->d_rowstart, c->d_p, c->dinv, c->Rinv1, c->Rinv2, c->m, c->P, state_prec(c->precision),
                        c->d_perm ? c->rtmp : db_dev, s));
    if (c->d_perm) CK(c, launch_permute_vec(c->rtmp, c->d_perm, c->N, 1, db_dev, s));  // caller's row order
    c->t = 0;  // the iteration state now holds the reverse sweep: apc_iterate needs apc_reset
    return APC_OK;
}

int apc_backward_params(apc_ctx *c, const double *g_dev, const double *b_dev, int64_t T, double gamma, double eta,
                        int32_t ckpt_every, double *db_dev, double *dgamma_host, double *deta_host, void *stream) {
    if (!c || !g_dev || !db_dev || !dgamma_host || !deta_host || T < 0 || ckpt_every < 0)
        return fail(c, APC_ERR_INVALID_ARG, "bad argument");
    if (!(gamma > 0.0 && gamma < 2.0) || !std::isfinite(eta))
        return fail(c, APC_ERR_PARAMS, "gamma=%g must lie in (0, 2) and eta must be finite", gamma);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t C = std::max<int64_t>(1, std::min<int64_t>(ckpt_every > 0 ? ckpt_every : 20, std::max<int64_t>(T, 1)));
    const int64_t nseg = (T + C - 1) / C;
    const size_t ssz = s_elem_size(c->precision);
    const size_t xs = ssz * size_t(c->n) * c->m, xbs = sizeof(double) * size_t(c->n);
    const size_t zs = ssz * 3 * size_t(c->m) * c->P, st = xs + xbs + zs;
    char *ck = nullptr, *seg = nullptr, *save = nullptr;
    double *acc = nullptr;
    std::vector<int64_t> ck_t(size_t(std::max<int64_t>(nseg, 1)), 0);
    auto release = [&]() {
        cudaFree(ck);
        cudaFree(seg);
        cudaFree(save);
        cudaFree(acc);
    };
    if (cudaMalloc(&ck, st * size_t(std::max<int64_t>(nseg, 1))) != cudaSuccess ||
        cudaMalloc(&seg, (xs + xbs) * size_t(C + 1)) != cudaSuccess || cudaMalloc(&save, st) != cudaSuccess ||
        cudaMalloc(&acc, 2 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(c, APC_ERR_NOMEM, "apc_backward_params: cannot allocate %lld checkpoints",
                    (long long)nseg);
    }
    // copies of the iteration state (machines' iterates, master, z buffers, pass counter)
    auto put = [&](char *dst) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, c->xw, xs, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst + xs, c->xbar, xbs, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst + xs + xbs, c->zbuf, zs, cudaMemcpyDeviceToDevice, s);
        return e;
    };
    auto get = [&](const char *src) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(c->xw, src, xs, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->xbar, src + xs, xbs, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->zbuf, src + xs + xbs, zs, cudaMemcpyDeviceToDevice, s);
        return e;
    };
    auto seg_state = [&](int64_t j) { return seg + size_t(j) * (xs + xbs); };
    auto keep = [&](int64_t j) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(seg_state(j), c->xw, xs, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(seg_state(j) + xs, c->xbar, xbs, cudaMemcpyDeviceToDevice, s);
        return e;
    };
    int rc = APC_OK;
    auto body = [&]() -> int {
        int r;
        // forward from the least-norm start, a checkpoint every C iterations
        const double *rhs = b_dev;
        if (b_dev && c->d_perm) {
            CK(c, launch_permute_vec(b_dev, c->d_perm, c->N, 0, c->rtmp, s));
            rhs = c->rtmp;
        }
        if ((r = reset_blocked(c, rhs, s)) != APC_OK) return r;
        for (int64_t k = 0; k < nseg; ++k) {
            CK(c, put(ck + size_t(k) * st));
            ck_t[size_t(k)] = c->t;
            if (k + 1 < nseg && (r = run_pass(c, MODE_APC, gamma, eta, C, s)) != APC_OK) return r;
        }
        // reverse sweep (apc_backward), one transposed step at a time
        CK(c, cudaMemsetAsync(c->xw, 0, xs, s));
        CK(c, cudaMemsetAsync(c->zbuf, 0, zs, s));
        CK(c, cudaMemcpyAsync(c->xbar, g_dev, xbs, cudaMemcpyDeviceToDevice, s));
        CK(c, cudaMemsetAsync(acc, 0, 2 * sizeof(double), s));
        c->t = 0;
        if ((r = run_pass(c, MODE_ADJ_SEED, gamma, eta, 1, s)) != APC_OK) return r;
        for (int64_t k = nseg - 1; k >= 0; --k) {
            const int64_t t0 = k * C, len = std::min(T, t0 + C) - t0;
            // forward states t0 .. t0 + len from the checkpoint, the reverse state set aside
            CK(c, put(save));
            const int64_t t_adj = c->t;
            CK(c, get(ck + size_t(k) * st));
            c->t = ck_t[size_t(k)];
            CK(c, keep(0));
            for (int64_t j = 1; j <= len; ++j) {
                if ((r = run_pass(c, MODE_APC, gamma, eta, 1, s)) != APC_OK) return r;
                CK(c, keep(j));
            }
            CK(c, get(save));
            c->t = t_adj;
            for (int64_t j = len - 1; j >= 0; --j) {
                // lambda_i(t+1), lbar(t+1) are the state before the transposed step for t = t0 + j
                CK(c, launch_adj_dots(c->xw, c->xbar, seg_state(j + 1), seg_state(j), reinterpret_cast<const double *>(
                                          seg_state(j) + xs), c->n, c->m, eta / c->m, state_prec(c->precision), acc, s));
                if ((r = run_pass(c, MODE_ADJ, gamma, eta, 1, s)) != APC_OK) return r;
            }
        }
        // v_i = Q_i^T (lambda_i(0) + lbar(0)/m), db_i = (A_i^+)^T-part as in apc_backward
        if ((r = run_pass(c, MODE_ADJ_FINAL, gamma, eta, 1, s)) != APC_OK) return r;
        const void *v = static_cast<const char *>(c->zbuf) + ssz * size_t(c->t % 3) * c->m * c->P;
        CK(c, launch_bsolve(v, c->d_rowstart, c->d_p, c->dinv, c->Rinv1, c->Rinv2, c->m, c->P,
                            state_prec(c->precision), c->d_perm ? c->rtmp : db_dev, s));
        if (c->d_perm) CK(c, launch_permute_vec(c->rtmp, c->d_perm, c->N, 1, db_dev, s));
        double h[2];
        CK(c, cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(c, cudaStreamSynchronize(s));
        *dgamma_host = h[0] / gamma;
        *deta_host = h[1];
        return APC_OK;
    };
    rc = body();
    cudaStreamSynchronize(s);
    release();
    c->t = 0;  // the iteration state now holds the reverse sweep: apc_iterate needs apc_reset
    return rc;
}

int apc_set_deterministic(apc_ctx *c, int32_t on) {
    if (!c) return fail(nullptr, APC_ERR_INVALID_ARG, "NULL context");
    if (on && !c->zpart) {
        const size_t bytes = s_elem_size(c->precision) * size_t(c->clusters) * c->m * c->P;
        if (cudaMalloc(&c->zpart, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->zpart = nullptr;
            return fail(c, APC_ERR_NOMEM, "cudaMalloc of %zu bytes (per-cluster partial sums) failed", bytes);
        }
    }
    c->det = on ? 1 : 0;
    return APC_OK;
}

namespace {
// Header of an exported iteration state (apc_export_state).
struct StateHeader {
    uint64_t magic;
    uint32_t version;
    int32_t precision;
    int64_t n, N;
    int32_t m, P;
    int64_t t;
    uint64_t payload;
    double rhs_norm2;  // ||rhs||^2 of the last reset (the monitor's denominator)
};
constexpr uint64_t kStateMagic = 0x4554415453435041ull;  // "APCSTATE"

size_t state_payload(const apc_ctx *c) {
    const size_t ssz = s_elem_size(c->precision);
    return ssz * size_t(c->n) * c->m + sizeof(double) * size_t(c->n) + ssz * 3 * size_t(c->m) * c->P;
}
}  // namespace

int apc_state_bytes(const apc_ctx *c, size_t *bytes) {
    if (!c || !bytes) return APC_ERR_INVALID_ARG;
    *bytes = sizeof(StateHeader) + state_payload(c);
    return APC_OK;
}

int apc_export_state(apc_ctx *c, void *host_buf, size_t bytes, void *stream) {
    if (!c || !host_buf) return fail(c, APC_ERR_INVALID_ARG, "NULL argument");
    const size_t need = sizeof(StateHeader) + state_payload(c);
    if (bytes < need) return fail(c, APC_ERR_INVALID_ARG, "buffer of %zu bytes; the state needs %zu", bytes, need);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StateHeader h = {kStateMagic, 1u, c->precision, c->n, c->N, c->m, c->P, c->t, state_payload(c), 0.0};
    CK(c, cudaMemcpyAsync(&h.rhs_norm2, c->sums + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    char *p = static_cast<char *>(host_buf);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const size_t ssz = s_elem_size(c->precision);
    const size_t bx = ssz * size_t(c->n) * c->m, bb = sizeof(double) * size_t(c->n), bz = ssz * 3 * size_t(c->m) * c->P;
    CK(c, cudaMemcpyAsync(p, c->xw, bx, cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(p + bx, c->xbar, bb, cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(p + bx + bb, c->zbuf, bz, cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    return APC_OK;
}

int apc_import_state(apc_ctx *c, const void *host_buf, size_t bytes, void *stream) {
    if (!c || !host_buf) return fail(c, APC_ERR_INVALID_ARG, "NULL argument");
    StateHeader h;
    if (bytes < sizeof(h)) return fail(c, APC_ERR_INVALID_ARG, "buffer shorter than the state header");
    std::memcpy(&h, host_buf, sizeof(h));
    if (h.magic != kStateMagic || h.version != 1u)
        return fail(c, APC_ERR_INVALID_ARG, "not an exported APC state (magic or version)");
    if (h.precision != c->precision || h.n != c->n || h.N != c->N || h.m != c->m || h.P != c->P ||
        h.payload != state_payload(c))
        return fail(c, APC_ERR_INVALID_ARG, "the state belongs to another problem shape or precision");
    if (bytes < sizeof(h) + h.payload) return fail(c, APC_ERR_INVALID_ARG, "buffer shorter than the state");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const char *p = static_cast<const char *>(host_buf) + sizeof(h);
    const size_t ssz = s_elem_size(c->precision);
    const size_t bx = ssz * size_t(c->n) * c->m, bb = sizeof(double) * size_t(c->n), bz = ssz * 3 * size_t(c->m) * c->P;
    CK(c, cudaMemcpyAsync(c->xw, p, bx, cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(c->xbar, p + bx, bb, cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(c->zbuf, p + bx + bb, bz, cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(c->sums + 2, &h.rhs_norm2, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(c, cudaStreamSynchronize(s));
    c->t = h.t;
    return APC_OK;
}

int apc_set_test_hooks(apc_ctx *c, int32_t grid_barrier_skew, double timeout_s) {
    if (!c || grid_barrier_skew < 0 || !(timeout_s > 0.0)) return fail(c, APC_ERR_INVALID_ARG, "bad argument");
    c->test_barrier_skew = uint32_t(grid_barrier_skew);
    c->timeout_s = timeout_s;
    return APC_OK;
}

int apc_setup_report(const apc_ctx *c, int32_t *qr_passes, double *orth_probe) {
    if (!c) return APC_ERR_INVALID_ARG;
    if (qr_passes) *qr_passes = c->qr_passes;
    if (orth_probe) *orth_probe = c->orth_probe;
    return APC_OK;
}

int apc_context_info(const apc_ctx *c, int64_t *n, int64_t *N, int32_t *m, int32_t *width, int32_t *cluster_size,
                     int32_t *clusters, int64_t *q_bytes, int32_t *rows_per_group) {
    if (!c) return APC_ERR_INVALID_ARG;
    if (n) *n = c->n;
    if (N) *N = c->N;
    if (m) *m = c->m;
    if (width) *width = c->P;
    if (cluster_size) *cluster_size = c->cs;
    if (clusters) *clusters = c->clusters;
    if (q_bytes) *q_bytes = int64_t(c->q_bytes);
    if (rows_per_group) *rows_per_group = c->rg;
    return APC_OK;
}

const char *apc_last_error(const apc_ctx *c) { return c ? c->last_error.c_str() : g_setup_error.c_str(); }

void apc_destroy(apc_ctx *c) {
    if (!c) return;
    apc::destroy_multi_rhs(c);
    free_all(c);
    delete c;
}

}  // extern "C"
