// Instantiations of the persistent iteration kernel for Q stored as float.
#include "apc_iter_impl.cuh"

namespace apc {
void *iter_kernel_f32(int cpl, int wpw, bool apc, int rg) {
    return iterk::kernel_for<float, float, false>(cpl, wpw, apc, rg);
}
}  // namespace apc
