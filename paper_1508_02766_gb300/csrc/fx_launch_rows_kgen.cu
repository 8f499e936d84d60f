// Two-phase engine: launcher of one pass (its own translation unit so that
// the passes compile in parallel).
#include "fx_kernels.cuh"

namespace kde {
namespace fx {

cudaError_t launch_rows_kgen(const Launch& l, const RowsArgs& a, const KGen<float>& g) {
  if (l.cls == 0) return launch_kernel(kde_fx_rows_fwd_kernel<0, SRC_KGEN>, l.grid, l.threads, l.smem, l.st, a, (const long long*)nullptr, g);
  return launch_kernel(kde_fx_rows_fwd_kernel<1, SRC_KGEN>, l.grid, l.threads, l.smem, l.st, a, (const long long*)nullptr, g);
}

}  // namespace fx
}  // namespace kde
