// Shared-memory mbarriers and bulk (TMA) copies completed on them, with
// bounded waits (sm_103a, inline PTX).  Used by the world-step kernel's
// input staging and by the surrogate's tensor-core GEMM.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vmas {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Global -> shared bulk copy of `bytes` (a multiple of 16; both addresses
// 16-byte aligned), counted against the mbarrier's transaction bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Wait for phase `parity` of the mbarrier to complete: at most `tries` polls,
// each suspending the thread for at most about 1 us, so at most about
// tries us in all; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int tries) {
  for (int i = 0; i < tries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(1000u)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace vmas
