// cta_quicksort.cuh -- one CTA sorts up to a few thousand (key, position)
// pairs in shared memory by quicksort, choosing every pivot with the
// binary-tree median approximation (tree_median.cuh; Section 3 of Axtmann &
// Sanders, "Approximate Median Selection with a Single Reduction").  This is
// the in-SM counterpart of the paper's robust hypercube quicksort (Section
// 5): the pivot of a segment is the approximate median of a stratified
// sample of it, elements lexicographically below the pivot go left, the rest
// right.  Since the pivot is a (key, position) pair, a run of copies of the
// pivot's key is split at the pivot's position -- the paper's balanced
// split of equal keys (choose x copies for the left side so that the sides
// are as even as possible) done implicitly by the median of the pairs.
//
// Segments are kept on a shared-memory stack; the smaller side is handled
// first, so the stack depth stays below log2 of the size.  A segment of at
// most kQsBase elements is finished by the bins sort of cta_sort.cuh, as the
// paper's quicksort hands small inputs to a local sort.
#pragma once

#include "cta_sort.cuh"
#include "rsort_internal.cuh"
#include "tree_median.cuh"

namespace rsort {

constexpr int kQsBase = 1024;      // segments up to this size: the bins sort
constexpr int kQsSample = 256;     // pivot sample (tree leaves) per segment
constexpr int kQsWindow = 16;      // window size k of the median tree
constexpr int kQsStack = 64;       // segment stack entries

struct QsSmem {
  uint64_t* ak;   // [cap] the elements (result ends here)
  uint32_t* ai;
  uint64_t* bk;   // [cap] partition target
  uint32_t* bi;
  uint64_t* tk0;  // [kQsSample] median-tree level buffers
  uint32_t* tp0;
  uint64_t* tk1;
  uint32_t* tp1;
  uint8_t* tn0;   // [kQsSample / 2]
  uint8_t* tr0;
  uint8_t* tn1;
  uint8_t* tr1;
  uint32_t* stack;  // [2 * kQsStack]
  CtaSortSmem base; // the bins sort of segments of at most kQsBase elements
};

// Shared memory of a QsSmem for `cap` elements, followed by the CtaSortSmem
// of the base case (kQsBase elements).
__host__ __device__ constexpr size_t qs_smem_bytes(size_t cap) {
  return cap * 24 + (size_t)kQsSample * 24 + (size_t)kQsSample * 2 + (size_t)kQsStack * 8 +
         (size_t)kQsBase * kCtaSortBytesPerElem;
}

__device__ inline QsSmem qs_carve(unsigned char* base, uint32_t cap) {
  QsSmem q;
  unsigned char* p = base;
  q.ak = (uint64_t*)p; p += (size_t)cap * 8;
  q.bk = (uint64_t*)p; p += (size_t)cap * 8;
  q.tk0 = (uint64_t*)p; p += (size_t)kQsSample * 8;
  q.tk1 = (uint64_t*)p; p += (size_t)kQsSample * 8;
  q.ai = (uint32_t*)p; p += (size_t)cap * 4;
  q.bi = (uint32_t*)p; p += (size_t)cap * 4;
  q.tp0 = (uint32_t*)p; p += (size_t)kQsSample * 4;
  q.tp1 = (uint32_t*)p; p += (size_t)kQsSample * 4;
  q.stack = (uint32_t*)p; p += (size_t)kQsStack * 8;
  q.tn0 = p; p += kQsSample / 2;
  q.tr0 = p; p += kQsSample / 2;
  q.tn1 = p; p += kQsSample / 2;
  q.tr1 = p; p += kQsSample / 2;
  q.base.k = (uint64_t*)p; p += (size_t)kQsBase * 8;
  q.base.i = (uint32_t*)p; p += (size_t)kQsBase * 4;
  q.base.hist = (uint32_t*)p;
  return q;
}

// Sorts q.ak/q.ai[0..m) in place.  seed drives the sample positions and the
// tree's coins (it changes the pivots, never the result).
template <int NT>
__device__ void cta_quicksort_pairs(const QsSmem& q, uint32_t m, uint64_t seed,
                                    uint64_t* scan_sm, uint64_t* red) {
  static_assert(kQsBase % NT == 0, "the base case holds kQsBase / NT elements per thread");
  constexpr int kBaseItems = kQsBase / NT;
  __shared__ uint32_t s_top;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    q.stack[0] = 0;
    q.stack[1] = m;
    s_top = m > 0 ? 1u : 0u;
  }
  __syncthreads();
  uint32_t round = 0;
  while (s_top > 0) {
    const uint32_t top = s_top - 1;
    const uint32_t lo = q.stack[2 * top], hi = q.stack[2 * top + 1];
    const uint32_t len = hi - lo;
    __syncthreads();
    if (tid == 0) s_top = top;
    if (len <= (uint32_t)kQsBase) {
      // base case: the bins sort (rank-by-counting when tiny); the segment's
      // elements are in no particular order
      uint64_t key[kBaseItems];
      uint32_t idx[kBaseItems];
#pragma unroll
      for (int r = 0; r < kBaseItems; ++r) {
        const uint32_t e = r * NT + tid;
        if (e < len) {
          key[r] = q.ak[lo + e];
          idx[r] = q.ai[lo + e];
        }
      }
      cta_sort_pairs<NT, kBaseItems>(key, idx, len, [] { return false; }, q.base, red, scan_sm,
                                     nullptr);
      for (uint32_t t = tid; t < len; t += NT) {
        q.ak[lo + t] = q.base.k[t];
        q.ai[lo + t] = q.base.i[t];
      }
      __syncthreads();
      continue;
    }
    // pivot: approximate median of a stratified sample of the segment,
    // ordered like the sort, by (key, original position)
    const uint64_t sseed = splitmix64_at(seed, ((uint64_t)lo << 32) | round++);
    const uint32_t S = len < (uint32_t)kQsSample ? len : (uint32_t)kQsSample;
    uint64_t pk;
    const uint32_t pi = cta_tree_median<kQsWindow, NT>(
        [&](uint32_t j, uint64_t& key, uint32_t& pos) {
          const uint32_t a = (uint32_t)(((uint64_t)j * len) / S);
          const uint32_t b = (uint32_t)(((uint64_t)(j + 1) * len) / S);
          const uint32_t slot = lo + a + (uint32_t)(splitmix64_at(sseed, j) % (b - a));
          key = q.ak[slot];
          pos = q.ai[slot];
        },
        S, next_pow2_u32(S), sseed, q.tk0, q.tp0, q.tn0, q.tr0, q.tk1, q.tp1, q.tn1, q.tr1, &pk);
    // partition into q.b: below the pivot left, the pivot, the rest right
    // (both counts in one scan: below in the high word, above in the low)
    uint64_t cnt = 0;
    for (uint32_t t = lo + tid; t < hi; t += NT) {
      const uint64_t k = q.ak[t];
      const uint32_t i = q.ai[t];
      if (pair_less(k, i, pk, pi)) cnt += 1ull << 32;
      else if (!(k == pk && i == pi)) cnt += 1ull;
    }
    uint64_t total;
    const uint64_t base = block_excl_scan_u64<NT>(cnt, &total, scan_sm);
    const uint32_t nleft = (uint32_t)(total >> 32);
    uint32_t cl = (uint32_t)(base >> 32), cr = (uint32_t)base;
    for (uint32_t t = lo + tid; t < hi; t += NT) {
      const uint64_t k = q.ak[t];
      const uint32_t i = q.ai[t];
      uint32_t d;
      if (pair_less(k, i, pk, pi)) d = lo + cl++;
      else if (k == pk && i == pi) d = lo + nleft;
      else d = lo + nleft + 1 + cr++;
      q.bk[d] = k;
      q.bi[d] = i;
    }
    __syncthreads();
    for (uint32_t t = lo + tid; t < hi; t += NT) {
      q.ak[t] = q.bk[t];
      q.ai[t] = q.bi[t];
    }
    if (tid == 0) {
      // push the larger side first so the smaller one is handled next
      const uint32_t l0 = lo, l1 = lo + nleft, r0 = lo + nleft + 1, r1 = hi;
      uint32_t t = s_top;
      const bool left_small = (l1 - l0) <= (r1 - r0);
      const uint32_t a0 = left_small ? r0 : l0, a1 = left_small ? r1 : l1;
      const uint32_t b0 = left_small ? l0 : r0, b1 = left_small ? l1 : r1;
      if (a1 > a0 && t < (uint32_t)kQsStack) { q.stack[2 * t] = a0; q.stack[2 * t + 1] = a1; ++t; }
      if (b1 > b0 && t < (uint32_t)kQsStack) { q.stack[2 * t] = b0; q.stack[2 * t + 1] = b1; ++t; }
      s_top = t;
    }
    __syncthreads();
  }
}

}  // namespace rsort
