// Instantiations of the persistent iteration kernel for Q stored as __nv_bfloat16,
// deterministic reduction of the clusters' partial sums (a separate
// translation unit so that the library's units compile in parallel).
#include "apc_iter_impl.cuh"

namespace apc {
void *iter_kernel_bf16_det(int cpl, int wpw, bool apc, int rg) {
    return iterk::kernel_for<__nv_bfloat16, float, true>(cpl, wpw, apc, rg);
}
}  // namespace apc
