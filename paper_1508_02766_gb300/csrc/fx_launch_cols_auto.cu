// Two-phase engine: launcher of one pass (its own translation unit so that
// the passes compile in parallel).
#include "fx3_kernels.cuh"

namespace kde {
namespace fx {

cudaError_t launch_cols_auto(const Launch& l, const ColsArgs& a) {
#define KDE_FX_KERNEL(n1, n2) kde_fx_cols_kernel<0, n1, n2, COL_AUTO>
#define KDE_FX_CASE_PAIR(n1, n2) \
  case n1 * 64 + n2:             \
    return launch_kernel(KDE_FX_KERNEL(n1, n2), l.grid, l.threads, l.smem, l.st, a);
#define KDE_FX_CASE_TRIPLE(n1, n2, n3)  \
  case n1 * 4096 + n2 * 64 + n3:       \
    return launch_kernel(kde_fx3_cols_kernel<n1, n2, n3, COL_AUTO>, l.grid, l.threads, l.smem, l.st, a);
  KDE_FX_DISPATCH(KDE_FX_KERNEL, a)
#undef KDE_FX_CASE_TRIPLE
#undef KDE_FX_CASE_PAIR
#undef KDE_FX_KERNEL
}

}  // namespace fx
}  // namespace kde

KDE_DEBUG_READER(fx_cols_auto)
