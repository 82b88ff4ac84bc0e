// cta_sort.cuh -- one CTA sorts up to NT*ITEMS (key, position) pairs that its
// threads hold in registers (element e = r*NT + threadIdx.x sits in slot r).
//
// The result is the lexicographic (key, position) order, left in shared
// memory.  Size-dependent choice (the paper's per-input-size algorithm choice,
// Section 6, applied to one bucket):
//
//   m <= kRankMax       rank-by-counting: slot = #{pairs smaller than me}
//                       (the ranking of Appendix "Fast Work-Inefficient
//                       Ranking", all in one CTA)
//   otherwise           split the bucket's key range [min, max] into
//                       2 * next_pow2(m) equal-width bins (a counting sort in
//                       shared memory), then order each bin that holds
//                       several elements by insertion (an element alone in
//                       its bin is already in place); the bins of a bucket
//                       are tiny unless its keys cluster
//   a crowded bin       bitonic sort of the whole bucket (Appendix "Bitonic
//   (> kBinLimit)       Sort"), which needs no assumption on the keys
//
// A bucket whose keys are all equal and whose elements arrive in position
// order (every bucket produced by the stable scatter) is already sorted; if
// they arrive in another order, the bins are taken over the positions.
#pragma once

#include "rsort_internal.cuh"

namespace rsort {

constexpr int kBinLimit = 16;
static_assert(kRankMax <= kLocalThreads, "rank-by-counting holds one element per thread");

struct CtaSortSmem {
  uint64_t* k;     // [cap]      cap = NT * ITEMS
  uint32_t* i;     // [cap]
  uint32_t* hist;  // [cap + cap/4 + cap/2]  up to 2*cap 16-bit bin counters
                   //   packed in pairs (one pad word after every thread's run
                   //   of counter words), then the list of bins holding
                   //   several elements
};

// Shared memory per element of capacity that a CtaSortSmem needs.
constexpr int kCtaSortBytesPerElem = 8 + 4 + 4 + 1 + 2;

// Counter word w of a scan in which every thread owns 2^lp consecutive words
// sits at w + (w >> lp): each thread's run starts one bank further on, so the
// lanes of a warp walking their runs in step hit distinct banks.
__device__ __forceinline__ uint32_t padded_word(uint32_t w, int lp) { return w + (w >> lp); }

template <int NT>
__device__ __forceinline__ void block_minmax_u64(uint64_t& mn, uint64_t& mx, uint64_t* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t a = __shfl_xor_sync(0xffffffffu, mn, o);
    const uint64_t b = __shfl_xor_sync(0xffffffffu, mx, o);
    mn = a < mn ? a : mn;
    mx = b > mx ? b : mx;
  }
  if (lane == 0) {
    red[2 * w] = mn;
    red[2 * w + 1] = mx;
  }
  __syncthreads();
  mn = red[0];
  mx = red[1];
#pragma unroll
  for (int q = 1; q < NT / 32; ++q) {
    mn = red[2 * q] < mn ? red[2 * q] : mn;
    mx = red[2 * q + 1] > mx ? red[2 * q + 1] : mx;
  }
  __syncthreads();
}

__device__ __forceinline__ uint32_t bin_start(const uint32_t* hist, uint32_t b, int lp) {
  return (hist[padded_word(b >> 1, lp)] >> ((b & 1) << 4)) & 0xffffu;
}

// After a sort in which the positions stood in for keys that were all equal
// to key_all: writes that key back into the sorted slots.
template <int NT>
__device__ __forceinline__ void restore_common_key(const CtaSortSmem& s, uint32_t m, int by_pos,
                                                   uint64_t key_all) {
  if (!by_pos) return;
  for (uint32_t t = threadIdx.x; t < m; t += NT) s.k[t] = key_all;
  __syncthreads();
}

// Adds the m elements of a bucket to the counter of the algorithm that sorted
// it (algo: kNumAlgos counters, or nullptr when nobody counts).
__device__ __forceinline__ void count_algo(uint64_t* algo, int which, uint32_t m) {
  if (algo && threadIdx.x == 0) atomicAdd((unsigned long long*)&algo[which], (unsigned long long)m);
}

// Bitonic sort of the whole bucket (Appendix "Bitonic Sort"): pairs padded to
// a power of two with (UINT64_MAX, UINT32_MAX), ordered by (key, position).
template <int NT, int ITEMS>
__device__ __forceinline__ void cta_bitonic_pairs(const uint64_t (&key)[ITEMS],
                                                  const uint32_t (&idx)[ITEMS], uint32_t m,
                                                  const CtaSortSmem& s) {
  const uint32_t P = next_pow2_u32(m);
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const uint32_t e = r * NT + threadIdx.x;
    if (e < m) { s.k[e] = key[r]; s.i[e] = idx[r]; }
  }
  for (uint32_t e = m + threadIdx.x; e < P; e += NT) { s.k[e] = ~0ULL; s.i[e] = ~0u; }
  block_bitonic_sort<NT>(s.k, s.i, (int)P);
}

// No-op for cta_sort_pairs' released callback.
struct NoRelease {
  __device__ void operator()() const {}
};

// Sorts the m pairs; on return s.k[0..m) / s.i[0..m) hold them in order.
// in_position_order() says whether the elements arrive with increasing
// positions; it is asked only when all keys are equal.  algo (nullable) gets
// m added to the counter of the branch taken (kAlgoRank, kAlgoInOrder,
// kAlgoBitonic or kAlgoBins).  rank_max bounds rank-by-counting (at most NT
// elements: one per thread); force_bitonic sorts every larger bucket by
// bitonic sort instead of the bins.  released() is called once by every
// thread of the CTA, together, as soon as key[] and idx[] are no longer read
// (the pairs are in shared memory): the caller may then load the next
// bucket into them while this one is finished.
template <int NT, int ITEMS, typename InOrderFn, typename ReleaseFn = NoRelease>
__device__ void cta_sort_pairs(uint64_t (&key)[ITEMS], uint32_t (&idx)[ITEMS], uint32_t m,
                               InOrderFn in_position_order, const CtaSortSmem& s, uint64_t* red,
                               uint64_t* scan_sm, uint64_t* algo, uint32_t rank_max = kRankMax,
                               bool force_bitonic = false, ReleaseFn released = ReleaseFn()) {
  constexpr uint32_t kCap = NT * ITEMS;
  static_assert(ITEMS >= 4, "the padded counters need cap/4 >= NT words of slack");
  const uint32_t tid = threadIdx.x;
  if (m <= rank_max && m <= (uint32_t)NT) {
    count_algo(algo, kAlgoRank, m);
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const uint32_t e = r * NT + tid;
      if (e < m) { s.k[e] = key[r]; s.i[e] = idx[r]; }
    }
    __syncthreads();
    uint32_t rank = 0;
    if (tid < m) {
      for (uint32_t q = 0; q < m; ++q) rank += pair_less(s.k[q], s.i[q], key[0], idx[0]) ? 1u : 0u;
    }
    __syncthreads();
    if (tid < m) { s.k[rank] = key[0]; s.i[rank] = idx[0]; }
    __syncthreads();
    released();
    return;
  }
  if (force_bitonic) {
    count_algo(algo, kAlgoBitonic, m);
    cta_bitonic_pairs<NT, ITEMS>(key, idx, m, s);
    released();
    return;
  }
  uint64_t mn = ~0ULL, mx = 0;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    if (r * NT + tid < m) {
      mn = key[r] < mn ? key[r] : mn;
      mx = key[r] > mx ? key[r] : mx;
    }
  }
  block_minmax_u64<NT>(mn, mx, red);
  if (mn == mx && in_position_order()) {
    count_algo(algo, kAlgoInOrder, m);
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const uint32_t e = r * NT + tid;
      if (e < m) { s.k[e] = key[r]; s.i[e] = idx[r]; }
    }
    __syncthreads();
    released();
    return;
  }
  // all keys equal, in no particular order: (key, position) order is the
  // order of the positions, so the positions (distinct) stand in for the
  // keys below and the common key is put back at the end
  __shared__ uint64_t s_key_all;
  __shared__ int s_by_pos;
  if (tid == 0) {
    s_by_pos = mn == mx;
    s_key_all = mn;
  }
  if (mn == mx) {
    mn = ~0ULL;
    mx = 0;
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      if (r * NT + tid < m) {
        key[r] = idx[r];
        mn = key[r] < mn ? key[r] : mn;
        mx = key[r] > mx ? key[r] : mx;
      }
    }
    block_minmax_u64<NT>(mn, mx, red);
  }
  // equal-width bins over [mn, mx]
  const uint32_t nb = 2 * next_pow2_u32(m);  // <= 2 * kCap
  const int lognb = log2_u32(nb);
  const uint64_t range = mx - mn;
  const int bits = range ? 64 - __clzll((long long)range) : 0;
  const int shift = bits > lognb ? bits - lognb : 0;
  // counter words, each thread's run of them, and the padded layout
  const uint32_t words = nb / 2;
  const uint32_t per = (words + NT - 1) / NT;  // a power of two
  const int lp = log2_u32(per);
  for (uint32_t w = tid; w < words + (words >> lp); w += NT) s.hist[w] = 0;
  __shared__ uint32_t s_nmulti;
  if (tid == 0) s_nmulti = 0;
  __syncthreads();
  uint32_t bs[ITEMS];
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    if (r * NT + tid < m) {
      const uint32_t b = (uint32_t)((key[r] - mn) >> shift);
      const uint32_t sh = (b & 1) << 4;
      const uint32_t old = atomicAdd(&s.hist[padded_word(b >> 1, lp)], 1u << sh);
      bs[r] = (b << 16) | ((old >> sh) & 0xffffu);
    }
  }
  __syncthreads();
  // exclusive scan of the nb 16-bit counters (nb/2 words; each thread a run),
  // which also finds out whether any bin is crowded
  const uint32_t w0 = tid * per;
  bool crowd = false;
  {
    uint32_t loc = 0;
    for (uint32_t w = w0; w < w0 + per && w < words; ++w) {
      const uint32_t v = s.hist[padded_word(w, lp)];
      const uint32_t a = v & 0xffffu, b = v >> 16;
      loc += a + b;
      crowd |= a > (uint32_t)kBinLimit || b > (uint32_t)kBinLimit;
    }
    uint64_t tot;
    uint32_t run = (uint32_t)block_excl_scan_u64<NT>(loc, &tot, scan_sm);
    for (uint32_t w = w0; w < w0 + per && w < words; ++w) {
      const uint32_t pw = padded_word(w, lp);
      const uint32_t v = s.hist[pw];
      const uint32_t lo = run, hi = run + (v & 0xffffu);
      s.hist[pw] = lo | (hi << 16);
      run = hi + (v >> 16);
    }
  }
  if (__syncthreads_or(crowd)) {
    // clustered keys: bitonic sort of the whole bucket
    count_algo(algo, kAlgoBitonic, m);
    cta_bitonic_pairs<NT, ITEMS>(key, idx, m, s);
    restore_common_key<NT>(s, m, s_by_pos, s_key_all);
    released();
    return;
  }
  // counting-sort scatter into the bins; the second element to land in a bin
  // puts the bin on the list of bins that still need ordering
  count_algo(algo, kAlgoBins, m);
  uint32_t* multi = s.hist + kCap + kCap / 4;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    if (r * NT + tid < m) {
      const uint32_t b = bs[r] >> 16, o = bs[r] & 0xffffu;
      const uint32_t p = bin_start(s.hist, b, lp) + o;
      s.k[p] = key[r];
      s.i[p] = idx[r];
      if (o == 1) multi[atomicAdd(&s_nmulti, 1u)] = b;
    }
  }
  __syncthreads();
  released();
  // order every listed bin in place by insertion (at most kBinLimit elements;
  // an element alone in its bin is already in its final slot)
  const uint32_t nmulti = s_nmulti;
  for (uint32_t j = tid; j < nmulti; j += NT) {
    const uint32_t b = multi[j];
    const uint32_t lo = bin_start(s.hist, b, lp);
    const uint32_t hi = b + 1 < nb ? bin_start(s.hist, b + 1, lp) : m;
    uint64_t* bk = s.k + lo;
    uint32_t* bi = s.i + lo;
    for (uint32_t a = 1; a < hi - lo; ++a) {
      const uint64_t ka = bk[a];
      const uint32_t ia = bi[a];
      uint32_t q = a;
      while (q > 0 && pair_less(ka, ia, bk[q - 1], bi[q - 1])) {
        bk[q] = bk[q - 1];
        bi[q] = bi[q - 1];
        --q;
      }
      bk[q] = ka;
      bi[q] = ia;
    }
  }
  __syncthreads();
  restore_common_key<NT>(s, m, s_by_pos, s_key_all);
  (void)kCap;
}

}  // namespace rsort
