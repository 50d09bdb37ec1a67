// Shared-memory mbarriers for the tensor-memory-accelerator copies (sm_90 and
// later), with waits that give up after a bounded time instead of spinning
// forever.
#pragma once

#include <cstdint>

namespace adafac {

constexpr long kWaitLimit = 1L << 22;                  // polls before a wait gives up
constexpr unsigned long long kWaitNs = 2000000000ull;  // or device time (2 s)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// an mbarrier expecting one arrival per phase
__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

// makes initialised mbarriers visible to the asynchronous copy unit
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// arrives and adds `bytes` to the transaction count of the current phase
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait on a phase of an mbarrier: gives up after kWaitNs of device
// time or `limit` polls (kWaitLimit by default), whichever comes first;
// limit 0 gives up before the first poll
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = kWaitLimit) {
  if (limit <= 0) return false;
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long i = 1; i < limit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 255 && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

}  // namespace adafac
