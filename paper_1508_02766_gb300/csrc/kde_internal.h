// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/kde_gb300.h"

struct kde_plan_s {
  kde_plan_info info;
  double H[9];
  double Hinv[9];
  double lo[KDE_MAX_D];
  double hi[KDE_MAX_D];
  double tau;
  int range_mode;
  int layout_mode;
  int cols_variant;
  int device;
  // Twiddle tables e^{-2 pi i m / P_k}, m in [0, P_k): one per axis, in the
  // plan's precision (float2 or double2), owned by the plan.
  void* tw_dev;
  size_t tw_offset[KDE_MAX_D];  // byte offset of axis k's table in tw_dev
};

namespace kde {

kde_status fail(kde_status s, const std::string& msg);
kde_status matrix_support(const kde_plan_s* plan, const double* A, double* Ainv, double* detA,
                          int64_t* L);
kde_status cuda_fail(cudaError_t e, const char* what);

// Launch bookkeeping: counts launches and, when profiling is on, records a
// pair of events around each launch on its stream.
struct LaunchScope {
  LaunchScope(const char* name, cudaStream_t stream);
  ~LaunchScope();
  int slot;
  cudaStream_t stream;
};

}  // namespace kde
