// Shared-memory mbarrier helpers (sm_90 and later) for the warp-specialised
// kernels of libfeasm. Every wait is bounded: after `limit` clock cycles it
// gives up and returns false, so that a kernel can record FE_ERR_TIMEOUT and
// leave instead of hanging.
#pragma once

#include <cstdint>

namespace feasm {

constexpr long long kWaitCycles = 1ll << 31;  // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of the given parity to complete; false after `limit` cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = kWaitCycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// Bulk copy (TMA engine) of `bytes` from shared to global memory, tracked by
// this thread's bulk-async groups; both addresses 16-byte aligned, bytes a
// multiple of 16. The shared source must have been written before a
// fence.proxy.async.shared::cta (fence_proxy_async) by the writing threads.
__device__ __forceinline__ void bulk_store(void* gdst, uint32_t ssrc, uint32_t bytes) {
  asm volatile(
      "{\n.reg .u64 g;\ncvta.to.global.u64 g, %0;\n"
      "cp.async.bulk.global.shared::cta.bulk_group [g], [%1], %2;\n"
      "cp.async.bulk.commit_group;\n}\n" ::"l"(gdst),
      "r"(ssrc), "r"(bytes)
      : "memory");
}
// Waits until the shared-memory source of every committed bulk copy has been read.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Waits until the shared-memory source of every committed bulk copy but the most recent one has been read.
__device__ __forceinline__ void bulk_wait_read_all_but_one() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// Waits until every committed bulk copy has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Orders this thread's shared-memory writes before later reads by the async proxy (bulk copies).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace feasm
