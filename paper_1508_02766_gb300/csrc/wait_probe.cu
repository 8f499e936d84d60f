// Check of the tensor-core kernels' bounded wait (tc_wait.cuh): one block
// initialises an mbarrier expecting one arrival, optionally arrives on it,
// and waits for its first phase with the same helper the GEMM and DFT
// kernels use.  Without the arrival nothing ever completes the phase, so the
// wait must give up after `limit` polls and the kernel must still finish and
// report it.  (A diagnostic of this library; the paper has no counterpart.)
#include <cuda_runtime.h>

#include <cstdint>

#include "kde_internal.h"
#include "tc_wait.cuh"

namespace kde {
namespace {

// out[0] = 0 if the phase completed, 1 if the wait gave up; out[1] = the
// clock64 cycles thread 0 spent waiting.
__global__ void __launch_bounds__(32) kde_wait_probe_kernel(int arrive, uint32_t limit,
                                                            long long* __restrict__ out) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) {
    asm volatile(
        "{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(b)
        : "memory");
  }
  __syncthreads();
  const long long t0 = clock64();
  const bool done = mbar_wait(b, 0u, limit);
  const long long t1 = clock64();
  const bool all = __syncthreads_and(done);
  if (threadIdx.x == 0) {
    out[0] = all ? 0 : 1;
    out[1] = t1 - t0;
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
  }
}

}  // namespace
}  // namespace kde

using namespace kde;

extern "C" kde_status kde_wait_probe(int arrive, uint32_t limit, long long* out,
                                     kde_stream_t stream) {
  if (!out) return fail(KDE_ERR_INVALID_ARG, "out is NULL");
  if (limit < 1) return fail(KDE_ERR_INVALID_ARG, "limit must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  kde_wait_probe_kernel<<<1, 32, 0, st>>>(arrive, limit, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_wait_probe_kernel");
}
