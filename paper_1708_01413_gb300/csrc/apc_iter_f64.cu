// Instantiations of the persistent iteration kernel for Q stored as double.
#include "apc_iter_impl.cuh"

namespace apc {
void *iter_kernel_f64(int cpl, int wpw, bool apc, int rg) {
    return iterk::kernel_for<double, double, false>(cpl, wpw, apc, rg);
}
}  // namespace apc
