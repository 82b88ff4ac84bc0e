// async_copy.cuh -- asynchronous global -> shared copies (cp.async, sm_80+
// including sm_103a) used to stage input tiles of the partition kernels.
//
// Completion is awaited with cp.async.wait_group, a hardware wait on the
// thread's own copy groups (no spin loop).  The streamed input is read with an
// L2 evict-first policy so that it does not displace the partially written
// bucket frontiers of the scatter.
#pragma once

#include <cstdint>

namespace rsort {

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void cp_async_8(void* smem_dst, const void* gmem_src, uint64_t pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(s),
               "l"(gmem_src), "l"(pol)
               : "memory");
}

__device__ __forceinline__ void cp_async_4(void* smem_dst, const void* gmem_src, uint64_t pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;\n" ::"r"(s),
               "l"(gmem_src), "l"(pol)
               : "memory");
}

__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// Global stores that ask the L2 to keep the line (scatter frontiers: a sector
// written in pieces by consecutive sub-tiles should be complete before it is
// written back).
__device__ __forceinline__ void st_keep_u64(uint64_t* p, uint64_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep_u32(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace rsort
