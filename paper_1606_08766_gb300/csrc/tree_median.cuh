// tree_median.cuh -- the binary-tree median approximation of Axtmann &
// Sanders (arXiv 1606.08766), Section 3 "Approximate Median Selection with a
// Single Reduction", as device building blocks.
//
// A node of the tree forwards a window of K entries: some entries below
// every element (undefined on the left), a sorted run of elements
// (key, position), and entries above every element.  The window is kept
// compactly as (neg, nre, reals[nre]); the count above is K - neg - nre.
//   leaf holding one element   coin 0: neg = K/2,     coin 1: neg = K/2 - 1
//   leaf holding nothing       neg = K/2, no element
//   internal node              the middle K of the 2K merged entries of its
//                              children (0-based merged positions K/2 .. 3K/2-1)
//   root                       entry K/2 - 1 (coin 0) or K/2 (coin 1), moved to
//                              the nearest element when that entry is undefined
// Leaf i flips bit 0 of splitmix64(seed, i); the root flips bit 0 of
// splitmix64(seed, number of leaves).
#pragma once

#include "rsort_internal.cuh"

namespace rsort {

// Combines two child windows into the parent's.  Children's elements are
// sorted pairs; the output gets the merged elements that fall inside the
// parent's window, in order.
template <int K>
__device__ __forceinline__ void tm_combine(int negA, int nA, const uint64_t* kA,
                                           const uint32_t* pA, int negB, int nB,
                                           const uint64_t* kB, const uint32_t* pB, int& neg,
                                           int& nre, uint64_t* ko, uint32_t* po) {
  const int N = negA + negB;   // merged entries below every element
  const int R = nA + nB;       // merged elements
  constexpr int s = K / 2;     // first merged position kept
  const int lo = s - N > 0 ? s - N : 0;             // first element index kept
  const int hi = s + K - N < R ? s + K - N : R;     // one past the last
  int nneg = N - s;
  nneg = nneg < 0 ? 0 : (nneg > K ? K : nneg);
  neg = nneg;
  nre = hi > lo ? hi - lo : 0;
  int ia = 0, ib = 0;
  for (int t = 0; t < hi; ++t) {
    const bool takeA = ib >= nB || (ia < nA && !pair_less(kB[ib], pB[ib], kA[ia], pA[ia]));
    uint64_t kk;
    uint32_t pp;
    if (takeA) {
      kk = kA[ia];
      pp = pA[ia];
      ++ia;
    } else {
      kk = kB[ib];
      pp = pB[ib];
      ++ib;
    }
    if (t >= lo) {
      ko[t - lo] = kk;
      po[t - lo] = pp;
    }
  }
}

// Window of leaf i: one element (present) or none, with its coin.
template <int K>
__device__ __forceinline__ int tm_leaf_neg(bool present, uint64_t seed, uint64_t i) {
  if (!present) return K / 2;
  return (splitmix64_at(seed, i) & 1ull) ? K / 2 - 1 : K / 2;
}

// Root choice: index into the root's elements of the returned entry.
template <int K>
__device__ __forceinline__ int tm_root_pick(int neg, int nre, uint64_t seed, uint64_t leaves) {
  const int pick = (splitmix64_at(seed, leaves) & 1ull) ? K / 2 : K / 2 - 1;
  if (nre == 0) return -1;
  if (pick < neg) return 0;
  if (pick >= neg + nre) return nre - 1;
  return pick - neg;
}

// One tree over `leaves` (a power of two) leaves, reduced by the NT threads
// of the calling CTA.  Leaf i < m holds the element leaf(i, key, pos); leaves
// i >= m are empty.  Two level buffers of `leaves` entries (key, position)
// plus leaves/2 counters each hold the windows of one tree level.  Returns,
// in every thread, the chosen element (m >= 1) as (*key_out, position).
template <int K, int NT, typename LeafFn>
__device__ uint32_t cta_tree_median(LeafFn leaf, uint32_t m, uint32_t leaves, uint64_t seed,
                                    uint64_t* bk0, uint32_t* bp0, uint8_t* bn0, uint8_t* br0,
                                    uint64_t* bk1, uint32_t* bp1, uint8_t* bn1, uint8_t* br1,
                                    uint64_t* key_out) {
  __shared__ uint32_t s_pos;
  __shared__ uint64_t s_key;
  const uint32_t tid = threadIdx.x;
  if (leaves == 1) {
    // a single leaf is the root: its window holds its element, the only one
    if (tid == 0) {
      uint64_t k0;
      uint32_t p0;
      leaf(0, k0, p0);
      s_pos = p0;
      s_key = k0;
    }
    __syncthreads();
    const uint32_t r = s_pos;
    *key_out = s_key;
    __syncthreads();
    return r;
  }
  // level 1: pairs of leaves
  uint32_t nodes = leaves / 2;
  int cap = 2 < K ? 2 : K;  // elements a level-1 window can hold
  for (uint32_t j = tid; j < nodes; j += NT) {
    const uint32_t a = 2 * j, b = 2 * j + 1;
    const bool pa = a < m, pb = b < m;
    uint64_t ka[1] = {0}, kb[1] = {0};
    uint32_t qa[1] = {0}, qb[1] = {0};
    if (pa) leaf(a, ka[0], qa[0]);
    if (pb) leaf(b, kb[0], qb[0]);
    int neg, nre;
    tm_combine<K>(tm_leaf_neg<K>(pa, seed, a), pa ? 1 : 0, ka, qa, tm_leaf_neg<K>(pb, seed, b),
                  pb ? 1 : 0, kb, qb, neg, nre, bk0 + (size_t)j * cap, bp0 + (size_t)j * cap);
    bn0[j] = (uint8_t)neg;
    br0[j] = (uint8_t)nre;
  }
  __syncthreads();
  uint64_t* ik = bk0;
  uint32_t* ip = bp0;
  uint8_t* in_n = bn0;
  uint8_t* in_r = br0;
  uint64_t* ok = bk1;
  uint32_t* op = bp1;
  uint8_t* on = bn1;
  uint8_t* orr = br1;
  while (nodes > 1) {
    const uint32_t half = nodes / 2;
    const int ncap = 2 * cap < K ? 2 * cap : K;
    for (uint32_t j = tid; j < half; j += NT) {
      const uint32_t a = 2 * j, b = 2 * j + 1;
      int neg, nre;
      tm_combine<K>(in_n[a], in_r[a], ik + (size_t)a * cap, ip + (size_t)a * cap, in_n[b],
                    in_r[b], ik + (size_t)b * cap, ip + (size_t)b * cap, neg, nre,
                    ok + (size_t)j * ncap, op + (size_t)j * ncap);
      on[j] = (uint8_t)neg;
      orr[j] = (uint8_t)nre;
    }
    __syncthreads();
    nodes = half;
    cap = ncap;
    uint64_t* tk = ik; ik = ok; ok = tk;
    uint32_t* tp = ip; ip = op; op = tp;
    uint8_t* tn = in_n; in_n = on; on = tn;
    uint8_t* tr = in_r; in_r = orr; orr = tr;
  }
  if (tid == 0) {
    const int pick = tm_root_pick<K>(in_n[0], in_r[0], seed, leaves);
    uint32_t r = 0;
    uint64_t kr = 0;
    if (pick >= 0) {
      r = ip[pick];
      kr = ik[pick];
    } else {
      leaf(0, kr, r);
    }
    s_pos = r;
    s_key = kr;
  }
  __syncthreads();
  const uint32_t r = s_pos;
  *key_out = s_key;
  __syncthreads();
  return r;
}

}  // namespace rsort
