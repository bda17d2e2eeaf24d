// Instantiations of the persistent iteration kernel for Q stored as __nv_bfloat16.
#include "apc_iter_impl.cuh"

namespace apc {
void *iter_kernel_bf16(int cpl, int wpw, bool apc, int rg) {
    return iterk::kernel_for<__nv_bfloat16, float, false>(cpl, wpw, apc, rg);
}
}  // namespace apc
