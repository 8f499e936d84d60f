// Two-phase engine: launcher of the forward slab pass (its own translation unit
// so that the passes compile in parallel).  Kernels compiled for one split
// serve plans whose last two axes share it; any other split up to 20 per
// factor takes the generic kernel.
#include "fx_slab.cuh"

namespace kde {
namespace fx {

cudaError_t launch_slab_fwd(const Launch& l, const SlabArgs& a) {
  if (a.lr.N1 == a.lc.N1 && a.lr.N2 == a.lc.N2) {
    switch (a.lr.N1 * 64 + a.lr.N2) {
#define KDE_FX_CASE_PAIR(n1, n2) \
  case n1 * 64 + n2:             \
    return launch_slab(kde_fx_slab_fwd_kernel<0, n1, n2>, l, a);
      KDE_FX_PAIRS(KDE_FX_CASE_PAIR)
#undef KDE_FX_CASE_PAIR
      default:
        break;
    }
  }
  if (a.lr.N1 > kSmallMax || a.lr.N2 > kSmallMax || a.lc.N1 > kSmallMax || a.lc.N2 > kSmallMax)
    return cudaErrorInvalidConfiguration;
  return launch_slab(kde_fx_slab_fwd_kernel<0, 0, 0>, l, a);
}

}  // namespace fx
}  // namespace kde

KDE_DEBUG_READER(fx_slab_fwd)
