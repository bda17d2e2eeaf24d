// Host side of the persistent iteration kernel: shared-memory sizing,
// co-residency queries and the cluster launch.
#include "apc_iter_impl.cuh"

namespace apc {

namespace {

void *kernel_for(int precision, int cpl, int wpw, bool apc, int rg, bool det = false) {
    switch (precision) {
        case 0: return det ? iter_kernel_f64_det(cpl, wpw, apc, rg) : iter_kernel_f64(cpl, wpw, apc, rg);
        case 1: return det ? iter_kernel_f32_det(cpl, wpw, apc, rg) : iter_kernel_f32(cpl, wpw, apc, rg);
        case 2: return det ? iter_kernel_bf16_det(cpl, wpw, apc, rg) : iter_kernel_bf16(cpl, wpw, apc, rg);
        default: return nullptr;
    }
}

size_t q_size(int precision) { return precision == 0 ? 8 : precision == 1 ? 4 : 2; }
size_t s_size(int precision) { return precision == 0 ? 8 : 4; }

cudaLaunchConfig_t make_config(int cs, int nw, int rg, int clusters, size_t smem, cudaStream_t s,
                               cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(clusters * cs), 1, 1);
    cfg.blockDim = dim3(unsigned((nw + 2 * rg + kProducerWarps) * 32), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(cs);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

size_t iter_smem_bytes(int precision, int P, int slots, int stages, int64_t rows_per_cluster, int rg) {
    return iterk::SmemLayout(q_size(precision), s_size(precision), slots, P, stages, rows_per_cluster, rg).total;
}

int iter_max_clusters(int precision, int cpl, int wpw, int cs, int nw, int rg, size_t smem) {
    void *k = kernel_for(precision, cpl, wpw, true, rg);
    void *k2 = kernel_for(precision, cpl, wpw, false, rg);
    if (!k || !k2) return 0;
    if (cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = make_config(cs, nw, rg, 1, smem, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_iter(int precision, int cpl, const IterArgs &a, int clusters, size_t smem, cudaStream_t s) {
    void *k = kernel_for(precision, cpl, a.wpw, a.mode == MODE_APC, a.rg, a.det != 0);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = make_config(a.cs, a.nw, a.rg, clusters, smem, s, attr);
    void *args[] = {const_cast<IterArgs *>(&a)};
    return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace apc
