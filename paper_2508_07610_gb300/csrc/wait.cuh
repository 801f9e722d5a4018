// Time-bounded waits on shared-memory mbarriers.  A wait that does not complete within its limit
// returns false instead of spinning forever; the caller records the timeout in a status word, waits
// (again bounded) for its own copies in flight, releases what it holds and returns, so the context
// stays usable and the host reads the error.
#pragma once
#include <stdint.h>

namespace mpdo {

// default limit of one wait inside a kernel: far above any legitimate wait (microseconds)
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// wait for phase `parity` of the mbarrier to complete; false when limit_ns passed first
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(mbar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(mbar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

}  // namespace mpdo
