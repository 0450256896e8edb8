// Bulk asynchronous copies between global and shared memory through the
// Tensor Memory Accelerator (cp.async.bulk, PTX), completed on a shared-memory
// mbarrier (loads) or a bulk group (stores).  Used to stage whole contiguous
// pencil blocks of the FFT workspace.
//
// Rules the callers keep: both addresses 16-byte aligned, sizes multiples of
// 16 bytes; every wait on an mbarrier is bounded and, when it gives up, records
// a fault flag that the host reads after the work (the kernel then finishes
// with undefined data rather than hanging).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dda {
namespace bulk {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  // make the initialised barrier visible to the asynchronous proxy
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of transaction to come
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Wait for phase `phase` of the barrier at most `max_tries` polls (each poll may
// suspend the thread for a short hardware-defined time).  Returns false and
// sets *fault when it gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint32_t max_tries, unsigned int* fault) {
  for (uint32_t i = 0; i < max_tries; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  if (fault) atomicOr(fault, 1u);
  return false;
}

// global -> shared, completion counted on `bar` (transaction bytes)
__device__ __forceinline__ void load_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst_smem)),
               "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// shared -> global in the thread's bulk group
__device__ __forceinline__ void store_s2g(void* dst_gmem, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem), "r"(smem_addr(src_smem)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// block until every committed bulk store of this thread has finished reading shared memory
__device__ __forceinline__ void store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// order this thread's ordinary shared-memory writes before later asynchronous-proxy reads
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr uint32_t kMaxPolls = 1u << 20;

}  // namespace bulk
}  // namespace dda
