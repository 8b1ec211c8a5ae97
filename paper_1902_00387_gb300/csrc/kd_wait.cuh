// Bounded waits on mbarrier phases, shared by the kernels that use mbarriers (the coarse
// cluster kernel's point-to-point halo exchange, the tcgen05 GEMM) and by the self-test
// that makes such a wait run out (kd_selftest_wait).  A wait that runs out returns false;
// the caller records the failure in a status word and stops issuing work, so a missing
// producer never hangs the GPU.
#pragma once

#include <stdint.h>

namespace kd {

// true once the phase of the mbarrier at shared address `bar` with parity `parity` has
// completed; false after `max_cycles` SM clock cycles.  CLUSTER: acquire at cluster scope
// (data written by other CTAs of the cluster), else at CTA scope.
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long max_cycles) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    if (CLUSTER)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}"
          : "=r"(ok)
          : "r"(bar), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(ok)
          : "r"(bar), "r"(parity)
          : "memory");
    if (ok) return true;
    if (clock64() - t0 > max_cycles) return false;
  }
}

}  // namespace kd
