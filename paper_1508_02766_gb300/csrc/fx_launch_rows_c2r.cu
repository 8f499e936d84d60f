// Two-phase engine: launcher of one pass (its own translation unit so that
// the passes compile in parallel).
#include "fx_kernels.cuh"

namespace kde {
namespace fx {

cudaError_t launch_rows_c2r(const Launch& l, const RowsArgs& a) {
  if (l.cls == 0) return launch_kernel(kde_fx_rows_c2r_kernel<0>, l.grid, l.threads, l.smem, l.st, a);
  return launch_kernel(kde_fx_rows_c2r_kernel<1>, l.grid, l.threads, l.smem, l.st, a);
}

}  // namespace fx
}  // namespace kde
