// bulk_copy.cuh -- bulk global -> shared copies through the tensor memory
// accelerator (cp.async.bulk, sm_90+ including sm_103a) completed on shared
// memory barriers (mbarrier), with waits that give up after a bounded number
// of polls instead of spinning forever.
//
// One thread issues a copy of a contiguous run of bytes (16-byte aligned at
// both ends, a multiple of 16 bytes long) and tells the barrier how many bytes
// to expect; the barrier's phase completes when they have landed, and every
// thread that waits on that phase may then read them.
#pragma once

#include <cstdint>

namespace rsort {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Initialises a barrier whose phase completes after `count` arrivals (and,
// for a copy barrier, the transaction bytes announced with them).  Call from
// one thread, then publish with mbar_fence_init() and a block barrier before
// first use.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// One arrival on the barrier (release: this thread's earlier shared-memory
// reads are ordered before whoever waits for the phase).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses of shared memory before
// its later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrives on the barrier announcing `bytes` of transactions, then starts the
// bulk copy of `bytes` from global `src` to shared `dst` that completes them.
// The read carries the L2 cache policy `pol`.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar, uint64_t pol) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

// Polls the barrier for completion of the phase with the given parity; gives
// up (returns false) after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Asks the L2 to fetch the 16-byte granules that lie wholly inside the bytes
// [lo, hi) of global memory (an asynchronous hint: nothing waits for it, and
// no byte outside the range is touched).
__device__ __forceinline__ void prefetch_l2_range(const void* lo, const void* hi) {
  const uintptr_t a = ((uintptr_t)lo + 15) & ~(uintptr_t)15;
  const uintptr_t b = (uintptr_t)hi & ~(uintptr_t)15;
  if (b > a)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a))
                 : "memory");
}

// Polls before a bulk copy's bytes are given up on (each try_wait may suspend
// the thread for a system-dependent time before it reports "not yet"); a
// copy of 16 KB lands within microseconds, so only a fault reaches the limit.
constexpr uint32_t kBulkWaitPolls = 1u << 16;

}  // namespace rsort
