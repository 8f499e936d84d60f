// Two-phase engine: launcher of one pass (its own translation unit so that
// the passes compile in parallel).
#include "fx_kernels.cuh"

namespace kde {
namespace fx {

cudaError_t launch_rows_counts(const Launch& l, const RowsArgs& a, const long long* counts) {
  if (l.cls == 0) return launch_kernel(kde_fx_rows_fwd_kernel<0, SRC_COUNTS>, l.grid, l.threads, l.smem, l.st, a, counts, KGen<float>{});
  return launch_kernel(kde_fx_rows_fwd_kernel<1, SRC_COUNTS>, l.grid, l.threads, l.smem, l.st, a, counts, KGen<float>{});
}

}  // namespace fx
}  // namespace kde
