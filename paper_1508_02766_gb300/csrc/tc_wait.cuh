// Bounded wait on an mbarrier phase, shared by the tensor-core kernels.
// A kernel that waits on the tensor cores (tcgen05.commit arrivals) never
// spins without limit: after `limit` polls it gives up, reports through its
// status word and frees what it holds, so a lost arrival leaves an error
// status instead of a hung GPU.
#pragma once

#include <cstdint>

namespace kde {

// Polls of mbarrier.try_wait before a wait gives up.  A poll that does not
// find the phase complete suspends the thread for a while (about 7 800
// cycles, 3.8 us, measured on GB300), so the limit is about one second; the
// waits it guards (tensor-core work of one tile) take microseconds.
constexpr uint32_t kWaitLimit = 1u << 18;

// True once the phase with the given parity has completed, false if it has
// not after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase,
                                          uint32_t limit = kWaitLimit) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
  }
  return done != 0;
}

}  // namespace kde
