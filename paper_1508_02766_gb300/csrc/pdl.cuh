// Programmatic dependent launch: a kernel launched with
// programmaticStreamSerializationAllowed may start while the kernel before
// it on the stream is still running, once every block of that kernel has
// signalled (pdl_trigger) or exited.  It must call pdl_wait before it reads
// anything the earlier kernel writes and before any global write of its
// own; pdl_wait returns once the earlier kernels have completed and their
// memory operations are visible.  Launched without the attribute, both are
// no-ops.  What this buys is the next kernel's launch and block start-up
// (and any prologue that reads only inputs complete before the earlier
// kernel started) overlapping the earlier kernel's tail.
#pragma once

#include <cuda_runtime.h>

namespace kde {

__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// fn<<<grid, block, smem, st>>>(args...) with programmatic serialisation
// allowed against the previous kernel on st.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, static_cast<KArgs>(args)...);
}

}  // namespace kde
