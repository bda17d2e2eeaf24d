// Allocation-free variant of the FP64 residual check (apc_residual_noalloc).
//
// Who needs it: callers that may not allocate device memory at the moment
// they need a residual -- for example code running under a framework that has
// reserved all device memory for its own pool, or a latency-critical path
// where a cudaMalloc (which can synchronise the device) is not acceptable.
// Such a caller still owns and passes every input and output; the only
// working memory this entry point needs -- one pair of partial sums per
// thread block plus the final pair -- lives in the fixed-size array below,
// which is part of the library image and is held by every GPU that loads the
// library until the process exits.
//
// Consequences for callers:
//  * the array is shared by all calls: two calls that run at the same time on
//    the GPU (different streams, or different host threads on one device)
//    race on it and may return wrong results;
//  * every entry that a call reads is first written by that same call, so no
//    part of the array needs to start at zero;
//  * the first call on a device (and again the first call after the device's
//    context was reset) looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture;
//  * every call waits for its stream to finish (the result is a host value).
#include <cmath>
#include <cstdio>
#include <mutex>

#include <cuda.h>

#include "../../include/apc.h"
#include "apc_internal.h"

namespace apc {
void set_global_error_text(const char *msg);  // apc_api.cu
}

namespace {

// Rows per thread block of the partial-sum kernel and the largest number of
// blocks the static array holds: N <= 32 * 32768 = 1,048,576 rows.
constexpr int kWarps = 8, kRowsPerWarp = 4, kChunk = 2048;
constexpr int64_t kRowsPerBlock = int64_t(kWarps) * kRowsPerWarp;
constexpr int64_t kMaxBlocks = 32768;

// [0, 2*kMaxBlocks): per-block (||r||^2, ||rhs||^2); [2*kMaxBlocks, +2): totals.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxBlocks + 2];

// The array's device address, looked up once per device and context.  The
// address belongs to the module loaded into a CUDA context; after
// cudaDeviceReset the primary context is created anew, the module is loaded
// again and the array may move, so the cache is keyed by the context's
// process-unique id (cuCtxGetId), fetched through the runtime's driver entry
// points so that the library need not link the driver library.  Where those
// entry points are missing the address is looked up on every call.
struct DeviceAddress {
    bool ready = false;
    unsigned long long ctx_id = 0;
    double *ptr = nullptr;
};
constexpr int kMaxDevices = 64;
DeviceAddress g_addr[kMaxDevices];
std::mutex g_addr_mutex;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_entry_once;

// Id of the context current on this thread; false if unknown (no context yet,
// or the driver entry points are unavailable).
bool current_context_id(unsigned long long *id) {
    std::call_once(g_entry_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return false;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_noalloc_scratch for the current device and context.
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    DeviceAddress &d = g_addr[dev];
    if (d.ready && have_id && d.ctx_id == id) {
        *out = d.ptr;
        return cudaSuccess;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!have_id) have_id = current_context_id(&id);  // the lookup may have created the context
    d.ptr = static_cast<double *>(p);
    d.ctx_id = id;
    d.ready = have_id;
    *out = d.ptr;
    return cudaSuccess;
}

// out = rhs - A x for kRowsPerBlock rows per block; the block's sums of
// squares go to partials[2 * blockIdx.x + {0, 1}] (overwritten).
__global__ void __launch_bounds__(kWarps * 32) residual_partials_kernel(const double *A, int64_t lda, int64_t N,
                                                                        int64_t n, const double *x,
                                                                        const double *rhs, double *out,
                                                                        double *partials) {
    __shared__ double xs[kChunk];
    __shared__ double part[2][kWarps];
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int64_t row_base = int64_t(blockIdx.x) * kRowsPerBlock + int64_t(warp) * kRowsPerWarp;
    double acc[kRowsPerWarp];
    for (int r = 0; r < kRowsPerWarp; ++r) acc[r] = 0.0;
    for (int64_t k0 = 0; k0 < n; k0 += kChunk) {
        const int kn = int(n - k0 < kChunk ? n - k0 : kChunk);
        __syncthreads();
        for (int k = threadIdx.x; k < kn; k += blockDim.x) xs[k] = x[k0 + k];
        __syncthreads();
        for (int r = 0; r < kRowsPerWarp; ++r) {
            const int64_t row = row_base + r;
            if (row >= N) break;
            const double *a = A + row * lda + k0;
            double s = acc[r];
            for (int k = lane; k < kn; k += 32) s = fma(a[k], xs[k], s);
            acc[r] = s;
        }
    }
    double s_out = 0.0, s_rhs = 0.0;
    for (int r = 0; r < kRowsPerWarp; ++r) {
        double v = acc[r];
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        const int64_t row = row_base + r;
        if (lane == 0 && row < N) {
            const double rr = rhs[row] - v;
            if (out) out[row] = rr;
            s_out = fma(rr, rr, s_out);
            s_rhs = fma(rhs[row], rhs[row], s_rhs);
        }
    }
    if (lane == 0) {
        part[0][warp] = s_out;
        part[1][warp] = s_rhs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < kWarps; ++w) {
            a0 += part[0][w];
            a1 += part[1][w];
        }
        partials[2 * blockIdx.x] = a0;
        partials[2 * blockIdx.x + 1] = a1;
    }
}

// totals[0..1] = sums of the nblocks partial pairs, in a fixed order.
__global__ void __launch_bounds__(256) residual_totals_kernel(const double *partials, int64_t nblocks,
                                                              double *totals) {
    __shared__ double sh[2][256];
    double a0 = 0.0, a1 = 0.0;
    for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x) {
        a0 += partials[2 * b];
        a1 += partials[2 * b + 1];
    }
    sh[0][threadIdx.x] = a0;
    sh[1][threadIdx.x] = a1;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (int(threadIdx.x) < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        totals[0] = sh[0][0];
        totals[1] = sh[1][0];
    }
}

int fail(int code, const char *fmt, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b);
    apc::set_global_error_text(buf);
    return code;
}

}  // namespace

extern "C" int apc_residual_noalloc(const double *A_dev, int64_t lda, int64_t N, int64_t n, const double *x_dev,
                                    const double *rhs_dev, double *resid_dev, double *rel_residual_host,
                                    void *stream) {
    if (!A_dev || !x_dev || !rhs_dev || !rel_residual_host)
        return fail(APC_ERR_INVALID_ARG, "apc_residual_noalloc: NULL argument");
    if (n < 1 || N < 1 || lda < n) return fail(APC_ERR_INVALID_ARG, "apc_residual_noalloc: need N, n >= 1 and lda >= n");
    const int64_t nblocks = (N + kRowsPerBlock - 1) / kRowsPerBlock;
    if (nblocks > kMaxBlocks)
        return fail(APC_ERR_UNSUPPORTED,
                    "apc_residual_noalloc: N = %lld rows exceeds the static scratch limit of %lld rows",
                    (long long)N, (long long)(kMaxBlocks * kRowsPerBlock));
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return fail(APC_ERR_CUDA, "apc_residual_noalloc: cudaGetSymbolAddress failed (%lld)", (long long)e);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *partials = scratch;
    double *totals = scratch + 2 * kMaxBlocks;
    residual_partials_kernel<<<unsigned(nblocks), kWarps * 32, 0, s>>>(A_dev, lda, N, n, x_dev, rhs_dev, resid_dev,
                                                                       partials);
    residual_totals_kernel<<<1, 256, 0, s>>>(partials, nblocks, totals);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(APC_ERR_CUDA, "apc_residual_noalloc: launch failed (%lld)", (long long)e);
    double h[2];
    if ((e = cudaMemcpyAsync(h, totals, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(APC_ERR_CUDA, "apc_residual_noalloc: copy of the totals failed (%lld)", (long long)e);
    *rel_residual_host = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return APC_OK;
}
