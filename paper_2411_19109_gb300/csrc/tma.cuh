// Bulk asynchronous global -> shared copies (the TMA engine's untiled
// cp.async.bulk) completed on shared-memory mbarriers, with bounded waits.
//
// Every copy must start and end on 16-byte boundaries (the callers copy
// whole rows of arrays whose row length is a multiple of 4 elements).  A wait
// that does not complete within its bound records kErrTimeout in the error
// word the host reads after the launch sequence, waits once more (bounded)
// for the copies still in flight, and lets the kernel finish.
#pragma once

#include <stdint.h>

namespace llg {

constexpr int kErrTimeout = 1;
constexpr long long kWaitBound = 1LL << 22;   // try_wait rounds before giving up

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of asynchronous transactions.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; on time-out flags `err`.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, unsigned parity, int* err) {
  for (long long i = 0; i < kWaitBound; ++i)
    if (mbar_test(bar, parity)) return;
  if (err) atomicOr(err, kErrTimeout);
  for (long long i = 0; i < kWaitBound; ++i)
    if (mbar_test(bar, parity)) return;
}

}  // namespace llg
