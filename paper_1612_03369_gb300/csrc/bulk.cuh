// bulk.cuh -- one-dimensional bulk copies from global to shared memory
// (the TMA unit's non-tensor mode, cp.async.bulk) completed on an mbarrier,
// with time-bounded waits.
//
// Use: one thread initialises each barrier (count 1) and fences the init;
// per transfer it arms the barrier with the byte count it expects
// (arrive.expect_tx) and issues copies whose sizes sum to that count; every
// consumer waits for the barrier's phase (parity 0, 1, 0, ... on successive
// uses) before reading the destination.  Before reusing a destination that
// threads have read, the block synchronises and the issuing thread orders
// those reads before the copy with a proxy fence.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pic_internal.cuh"

namespace pic {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes initialised barriers visible to the copy engine.
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Arrive once and expect `bytes` of copies to complete the current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// its later bulk copies.
__device__ __forceinline__ void fence_proxy_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// `src` to shared `dst`, counted on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(static_cast<unsigned long long>(__cvta_generic_to_global(src))), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Wait for phase `parity` of bar, for at most timeout_ns of the global
// timer; false if the time ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > timeout_ns) return false;
  }
}

}  // namespace pic
