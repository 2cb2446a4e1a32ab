// doe_async.cuh -- asynchronous bulk copies global -> shared memory (cp.async.bulk, the
// non-tensor form of the Tensor Memory Accelerator) completed on an mbarrier, and the bounded
// waits on them.  Copies only move data of this GPU's own memory into the issuing CTA's own
// shared memory (no multicast).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace doe {

// Upper bound on the polls of one mbarrier wait.  A copy of this library's size lands within
// microseconds; the bound only keeps a kernel from spinning forever if one never does.
constexpr unsigned kMbarMaxPolls = 1u << 26;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
  // make the initialisation visible to the asynchronous proxy (and the cluster)
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of transactions the following copies will complete.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes) : "memory");
}
// A plain arrival (a phase with nothing to copy).
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global memory
// into this CTA's shared memory, completing `bytes` transactions on mbar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(mbar))
      : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later asynchronous
// (bulk-copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Waits for the phase of parity `parity` of mbar to complete.  Returns false if it did not
// within max_polls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, unsigned parity, unsigned max_polls = kMbarMaxPolls) {
  const unsigned a = smem_addr(mbar);
  for (unsigned i = 0; i < max_polls; ++i) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace doe
