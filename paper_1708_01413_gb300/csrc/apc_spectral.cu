// Estimates of the extreme eigenvalues of X = (1/m) sum_i Q_i Q_i^T (Eq. 3),
// the inputs of Theorem 1's optimal (gamma, eta), by the Lanczos process.
//
// Each Lanczos step needs one product X v.  The iteration kernel computes it
// in two passes over Q: a seed pass (z_i = Q_i^T v, xbar unchanged) and a
// power pass (xbar = (1/m) sum_i Q_i z_i).  The Lanczos vectors, the
// three-term recurrence and the dot products are FP64 on the device, and so
// are its scalars (alpha_j, beta_j): the steps queue on the stream without a
// host round trip, and the host reads the tridiagonal at the end; every
// new vector is re-orthogonalised against all previous ones (two classical
// Gram-Schmidt passes), without which the smallest Ritz value stalls percents
// above mu_min.  The k x k tridiagonal matrix stays on the host, where
// Sturm-sequence bisection gives its extreme eigenvalues (the Ritz values).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/apc.h"
#include "apc_ctx.h"
#include "apc_internal.h"

namespace apc {
int pass(apc_ctx *c, int mode, double gamma, double eta, int64_t iters, cudaStream_t s);  // apc_api.cu
// the same without a synchronisation after the launch, and the deferred check
int pass_queued(apc_ctx *c, int mode, double gamma, double eta, int64_t iters, cudaStream_t s);
int device_error(apc_ctx *c, cudaStream_t s);
}

namespace {

constexpr int kDotBlocks = 512, kDotThreads = 256;

__global__ void dot_partial_kernel(const double *a, const double *b, int64_t n, double *partial) {
    __shared__ double sh[kDotThreads];
    double s = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        s = fma(a[i], b[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = kDotThreads / 2; k > 0; k >>= 1) {
        if (int(threadIdx.x) < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void dot_final_kernel(const double *partial, int nb, double *out) {
    __shared__ double sh[kDotThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = kDotThreads / 2; k > 0; k >>= 1) {
        if (int(threadIdx.x) < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// w <- w - alpha v - beta vp, alpha = *alpha_d and beta = sqrt(*ww_prev)
// (the previous step's norm; 0 at the first step): the scalars stay on the
// device, so the steps queue without a host round trip
__global__ void three_term_kernel(double *w, const double *v, const double *vp, const double *alpha_d,
                                  const double *ww_prev, int64_t n) {
    const double alpha = *alpha_d, beta = ww_prev ? sqrt(*ww_prev) : 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        w[i] = w[i] - alpha * v[i] - beta * vp[i];
}

// h[j] = V_j . w for j < k (one block per j)
__global__ void gemv_t_kernel(const double *V, int64_t n, const double *w, double *h) {
    __shared__ double sh[kDotThreads];
    const double *Vj = V + size_t(blockIdx.x) * n;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(Vj[i], w[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = kDotThreads / 2; k > 0; k >>= 1) {
        if (int(threadIdx.x) < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) h[blockIdx.x] = sh[0];
}

// w <- w - sum_{j < k} h[j] V_j
__global__ void gemv_sub_kernel(const double *V, int k, int64_t n, const double *h, double *w) {
    extern __shared__ double hs[];
    for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = h[j];
    __syncthreads();
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = fma(V[size_t(j) * n + i], hs[j], s);
        w[i] -= s;
    }
}

// dst <- s * src
__global__ void scale_kernel(double *dst, const double *src, double s, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = s * src[i];
}

// The next Lanczos vector: dst <- src / b with b = sqrt(*ww), or zero at a
// breakdown (b <= 1e-14 max(1, |alpha|)); the steps after a breakdown then
// stay zero and the host drops them
__global__ void normalise_kernel(double *dst, const double *src, const double *ww, const double *alpha_d, int64_t n) {
    const double b = sqrt(*ww);
    const double s = (b <= 1e-14 * fmax(1.0, fabs(*alpha_d)) || !(b == b)) ? 0.0 : 1.0 / b;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = s * src[i];
}

// Number of eigenvalues of the symmetric tridiagonal (alpha, beta) below x
// (Sturm sequence of the LDL^T pivots).
int count_below(const std::vector<double> &alpha, const std::vector<double> &beta, double x) {
    int cnt = 0;
    double d = 1.0;
    for (size_t i = 0; i < alpha.size(); ++i) {
        const double b2 = i ? beta[i] * beta[i] : 0.0;
        d = alpha[i] - x - (i ? b2 / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// The j-th smallest eigenvalue (0-based) of the tridiagonal, by bisection.
double kth_eigenvalue(const std::vector<double> &alpha, const std::vector<double> &beta, int j) {
    double lo = 1e300, hi = -1e300;
    for (size_t i = 0; i < alpha.size(); ++i) {  // Gershgorin interval
        const double r = (i ? std::fabs(beta[i]) : 0.0) + (i + 1 < alpha.size() ? std::fabs(beta[i + 1]) : 0.0);
        lo = std::min(lo, alpha[i] - r);
        hi = std::max(hi, alpha[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-17 * std::max(1.0, std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (count_below(alpha, beta, mid) > j)
            hi = mid;
        else
            lo = mid;
    }
    return 0.5 * (lo + hi);
}

int sfail(apc_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->last_error = buf;
    return code;
}

struct DevBuf {
    double *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace

extern "C" int apc_spectral_bounds(apc_ctx *c, int32_t steps, uint64_t seed, double *mu_min_host,
                                   double *mu_max_host, void *stream) {
    if (!c || !mu_min_host || !mu_max_host) return sfail(c, APC_ERR_INVALID_ARG, "NULL argument");
    if (steps < 1 || steps > 4096) return sfail(c, APC_ERR_INVALID_ARG, "steps=%d outside 1..4096", steps);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = c->n;
    DevBuf V, w, scratch, h, ab;
    if (cudaMalloc(&V.p, sizeof(double) * n * steps) != cudaSuccess ||
        cudaMalloc(&w.p, sizeof(double) * n) != cudaSuccess || cudaMalloc(&h.p, sizeof(double) * steps) != cudaSuccess ||
        cudaMalloc(&scratch.p, sizeof(double) * (kDotBlocks + 2)) != cudaSuccess ||
        cudaMalloc(&ab.p, sizeof(double) * 2 * steps) != cudaSuccess) {
        cudaGetLastError();
        return sfail(c, APC_ERR_NOMEM, "cudaMalloc failed");
    }
    const unsigned grid = unsigned(std::min<int64_t>((n + kDotThreads - 1) / kDotThreads, kDotBlocks));
    auto dot = [&](const double *a, const double *b, double *out) -> int {
        dot_partial_kernel<<<grid, kDotThreads, 0, s>>>(a, b, n, scratch.p);
        dot_final_kernel<<<1, kDotThreads, 0, s>>>(scratch.p, int(grid), scratch.p + kDotBlocks);
        if (cudaMemcpyAsync(out, scratch.p + kDotBlocks, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return sfail(c, APC_ERR_CUDA, "dot product failed: %s", cudaGetErrorString(cudaGetLastError()));
        return APC_OK;
    };
    // the same into device memory, no host round trip
    auto dot_dev = [&](const double *a, const double *b, double *out_dev) {
        dot_partial_kernel<<<grid, kDotThreads, 0, s>>>(a, b, n, scratch.p);
        dot_final_kernel<<<1, kDotThreads, 0, s>>>(scratch.p, int(grid), out_dev);
    };
    double *alpha_d = ab.p, *ww_d = ab.p + steps;  // per step: v . Xv and the squared norm of the new w
    // start vector: splitmix64 stream of the seed, uniform in [-1, 1)
    std::vector<double> hv(n);
    uint64_t st = seed;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        hv[i] = double(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    if (cudaMemcpyAsync(w.p, hv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return sfail(c, APC_ERR_CUDA, "copy of the start vector failed");
    double nn = 0.0;
    int rc;
    if ((rc = dot(w.p, w.p, &nn)) != APC_OK) return rc;
    scale_kernel<<<grid, kDotThreads, 0, s>>>(V.p, w.p, 1.0 / std::sqrt(nn), n);
    const size_t sub_smem = sizeof(double) * steps;
    for (int j = 0; j < steps; ++j) {
        const double *v = V.p + size_t(j) * n, *vp = j ? V.p + size_t(j - 1) * n : V.p;
        // w = X v: seed pass (z_i = Q_i^T v, since eta/m = 1) then power pass
        if (cudaMemcpyAsync(c->xbar, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return sfail(c, APC_ERR_CUDA, "copy failed");
        if ((rc = apc::pass_queued(c, apc::MODE_ADJ_SEED, 1.0, double(c->m), 1, s)) != APC_OK) return rc;
        if ((rc = apc::pass_queued(c, apc::MODE_POWER, 1.0, double(c->m), 1, s)) != APC_OK) return rc;
        if (cudaMemcpyAsync(w.p, c->xbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return sfail(c, APC_ERR_CUDA, "copy failed");
        dot_dev(v, w.p, alpha_d + j);  // alpha_j
        three_term_kernel<<<grid, kDotThreads, 0, s>>>(w.p, v, vp, alpha_d + j, j ? ww_d + (j - 1) : nullptr, n);
        // full re-orthogonalisation against V_0 .. V_j, twice
        for (int pass = 0; pass < 2; ++pass) {
            gemv_t_kernel<<<unsigned(j + 1), kDotThreads, 0, s>>>(V.p, n, w.p, h.p);
            gemv_sub_kernel<<<grid, kDotThreads, sub_smem, s>>>(V.p, j + 1, n, h.p, w.p);
        }
        dot_dev(w.p, w.p, ww_d + j);  // beta_{j+1}^2
        if (j + 1 < steps)  // V_{j+1} = w / beta_{j+1}
            normalise_kernel<<<grid, kDotThreads, 0, s>>>(V.p + size_t(j + 1) * n, w.p, ww_d + j, alpha_d + j, n);
        if (cudaGetLastError() != cudaSuccess) return sfail(c, APC_ERR_CUDA, "Lanczos launch failed");
        // a pass's wait that timed out, every 8 steps: the steps queue without a
        // host round trip in between, and a persistent fault ends the process
        // after at most 16 passes
        if ((j & 7) == 7 && (rc = apc::device_error(c, s)) != APC_OK) return rc;
    }
    // the tridiagonal on the host, cut at the first breakdown (steps after it
    // ran on a zero vector)
    std::vector<double> ah(steps), wwh(steps);
    if (cudaMemcpyAsync(ah.data(), alpha_d, sizeof(double) * steps, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(wwh.data(), ww_d, sizeof(double) * steps, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return sfail(c, APC_ERR_CUDA, "Lanczos failed");
    if ((rc = apc::device_error(c, s)) != APC_OK) return rc;  // a pass's wait that timed out
    std::vector<double> alpha, beta{0.0};
    for (int j = 0; j < steps; ++j) {
        const double a = ah[j], b = std::sqrt(wwh[j]);
        alpha.push_back(a);
        if (!std::isfinite(a) || !std::isfinite(b)) return sfail(c, APC_ERR_NONFINITE, "Lanczos step %d not finite", j);
        if (j + 1 == steps || b <= 1e-14 * std::max(1.0, std::fabs(a))) break;
        beta.push_back(b);
    }
    *mu_min_host = kth_eigenvalue(alpha, beta, 0);
    *mu_max_host = kth_eigenvalue(alpha, beta, int(alpha.size()) - 1);
    return APC_OK;
}
