// Two-phase engine: launcher of one pass (its own translation unit so that
// the passes compile in parallel).
#include "fx_kernels.cuh"

namespace kde {
namespace fx {

cudaError_t launch_cols_inv(const Launch& l, const ColsArgs& a) {
  if (l.cls == 0) return launch_kernel(kde_fx_cols_kernel<0, COL_INV>, l.grid, l.threads, l.smem, l.st, a);
  return launch_kernel(kde_fx_cols_kernel<1, COL_INV>, l.grid, l.threads, l.smem, l.st, a);
}

}  // namespace fx
}  // namespace kde
