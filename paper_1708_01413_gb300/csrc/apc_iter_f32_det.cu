// Instantiations of the persistent iteration kernel for Q stored as float,
// deterministic reduction of the clusters' partial sums (a separate
// translation unit so that the library's units compile in parallel).
#include "apc_iter_impl.cuh"

namespace apc {
void *iter_kernel_f32_det(int cpl, int wpw, bool apc, int rg) {
    return iterk::kernel_for<float, float, true>(cpl, wpw, apc, rg);
}
}  // namespace apc
