// splitters.cuh -- the splitters of a partition step in shared memory and
// the two classifiers that search them (Appendix "Robust Multi-Level Sample
// Sort" of Axtmann & Sanders: the Super Scalar Sample Sort classifier, with
// the search repeated on a key tie using positions as tie-breakers).
//
// Shared by the classify / scatter kernels of every level.
#pragma once

#include "rsort_internal.cuh"

namespace rsort {

// Index of the last segment whose field is <= x (segments sorted by field).
template <typename F>
__device__ __forceinline__ uint32_t find_seg(const LevelSeg* segs, uint32_t G, uint64_t x,
                                             F field) {
  uint32_t lo = 0, hi = G;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (field(segs[mid]) <= x) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

__device__ __forceinline__ uint32_t ceil_log2_dev(uint32_t k) {
  uint32_t l = 0;
  while ((1u << l) < k) ++l;
  return l;
}

__device__ __forceinline__ uint64_t load_key(const Src& s, uint64_t pos) {
  const uint64_t k = __ldg(s.key + pos);
  return s.map_f64 ? f64_to_ordered(k) : k;
}

// ---------------------------------------------------------------------------
// Splitter structures in shared memory
//
// The k-1 splitters of a segment are the sorted sample's elements
// floor(j*S/k), j = 1..k-1 (Appendix "Generalizing Quicksort": every S/k-th
// sample), kept as sorted (key, position) pairs.  Two classifiers search them,
// both returning the same bucket:
//   tree   the branchless implicit search tree of Super Scalar Sample Sort that
//          the appendix names: the keys in Eytzinger order, padded with
//          UINT64_MAX to Kp - 1 = next_pow2(k) - 1 nodes;
//   table  a lookup table over the leading bits of (key - smallest splitter
//          key) giving, for every bin, the range of splitters whose key falls
//          in it; a key is located by one table read and a binary search over
//          its bin's splitters (a full binary search when keys cluster).
// A key equal to splitter keys is then placed among the run of those
// splitters by its position (tie_break).
// ---------------------------------------------------------------------------
constexpr int kTableBitsMax = 12;

struct Splitters {
  uint64_t* tree;   // [Kp]   node i at tree[i], i = 1..Kp-1          (tree mode)
  uint32_t* tbl;    // [2^tbits] packed (first, end) splitter of a bin (table mode)
  uint64_t* key;    // [k-1]  sorted splitter keys
  uint32_t* idx;    // [k-1]  their positions (tie-breakers)
  uint16_t* rend;   // [k-1]  end of the run of splitters whose key equals key[j]
  uint64_t lo, hi;  // smallest / largest splitter key
  int logK;         // log2(Kp)
  int tbits;        // table bits
  uint32_t tmax;    // last table entry (2^tbits - 1)
  int shift;        // key bits dropped before the table index
  int mode;         // 0 tree, 1 table
  int ntb;          // 1: no tie-breaking, classify by key only (ablation)
  uint32_t nspl;    // k - 1
};

__host__ __device__ inline int table_bits_for(uint32_t kp) {
  const int b = log2_u32(kp) + 1;
  return b < kTableBitsMax ? b : kTableBitsMax;
}

template <int NT>
__device__ void load_splitters(const LevelSeg& sg, const uint64_t* ssk, const uint32_t* ssi,
                               Splitters& sp) {
  const uint32_t k = sg.k;
  const uint32_t Kp = next_pow2_u32(k);
  sp.nspl = k - 1;
  sp.logK = log2_u32(Kp);
  for (uint32_t j = threadIdx.x; j < sp.nspl; j += NT) {
    const uint64_t r = ((uint64_t)(j + 1) * sg.S) / k;
    sp.key[j] = ssk[sg.samp_off + r];
    sp.idx[j] = ssi[sg.samp_off + r];
  }
  __syncthreads();
  // end of every run of equal splitter keys (keys are sorted, so the run of
  // key[j] is contiguous); tie-breaks search positions inside the run only
  for (uint32_t j = threadIdx.x; j < sp.nspl; j += NT) {
    const uint64_t kj = sp.key[j];
    uint32_t lo = j + 1, hi = sp.nspl;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (sp.key[mid] == kj) lo = mid + 1; else hi = mid;
    }
    sp.rend[j] = (uint16_t)lo;
  }
  if (sp.mode == 0) {
    for (uint32_t i = threadIdx.x + 1; i < Kp; i += NT) {
      const int d = 31 - __clz(i);
      const uint32_t r = i - (1u << d);
      const uint32_t in = ((2 * r + 1) << (sp.logK - 1 - d)) - 1;
      sp.tree[i] = in < sp.nspl ? sp.key[in] : ~0ULL;
    }
  } else if (sp.nspl > 0) {
    sp.lo = sp.key[0];
    sp.hi = sp.key[sp.nspl - 1];
    const uint64_t range = sp.hi - sp.lo;
    const int bits = range ? 64 - __clzll((long long)range) : 0;
    sp.tbits = table_bits_for(Kp);
    sp.shift = bits > sp.tbits ? bits - sp.tbits : 0;
    const uint32_t T = 1u << sp.tbits;
    sp.tmax = T - 1;
    // first splitter whose bin is >= t, by binary search over the sorted keys
    auto first_at_least = [&](uint32_t t) {
      uint32_t lo = 0, hi = sp.nspl;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (((sp.key[mid] - sp.lo) >> sp.shift) < t) lo = mid + 1; else hi = mid;
      }
      return lo;
    };
    for (uint32_t t = threadIdx.x; t < T; t += NT)
      sp.tbl[t] = first_at_least(t) | (first_at_least(t + 1) << 16);
  } else {
    // no splitters: one bin, empty, so every key lands in bucket 0
    sp.lo = 0;
    sp.hi = 0;
    sp.tbits = 0;
    sp.tmax = 0;
    sp.shift = 0;
    if (threadIdx.x == 0) sp.tbl[0] = 0;
  }
  __syncthreads();
}

// Bucket of element (x, i): the number of splitters lexicographically smaller
// than (x, i).  R elements descend the tree level by level together (R
// independent shared-memory loads in flight per level).  The descent counts
// the splitters whose key is smaller than x and remembers the key of the last
// node where it turned left, which is the bounding splitter's key; only if x
// equals it is the search repeated on the run of equal splitter keys with
// positions as tie-breakers (pos_of(r) is evaluated only then).
//
// The splitters whose key is x are [bb, rend[bb]), in increasing position;
// the bucket is bb plus the number of them placed before position i.  A long
// run (many copies of one key) holds positions of a stratified sample, close
// to evenly spaced: the search starts at an interpolated guess and gallops
// to a bracket around the answer, a few steps instead of log2 of the run.
__device__ __forceinline__ uint32_t tie_break(uint32_t bb, uint64_t x, uint32_t i,
                                              const Splitters& sp) {
  (void)x;
  uint32_t lo = bb, hi = sp.rend[bb];
  if (hi - lo > 8) {
    const uint32_t p0 = sp.idx[lo], p1 = sp.idx[hi - 1];
    if (i <= p0) return lo;
    if (i > p1) return hi;
    // now idx[lo] < i <= idx[hi - 1]: the answer is in (lo, hi - 1]
    const float f = __fdividef((float)(i - p0) * (float)(hi - 1 - lo), (float)(p1 - p0));
    uint32_t g = lo + (uint32_t)f;
    g = g < lo + 1 ? lo + 1 : (g > hi - 1 ? hi - 1 : g);
    uint32_t a, b;  // idx[a] < i <= idx[b]
    if (sp.idx[g] < i) {
      a = g;
      uint32_t d = 1;
      while (a + d < hi - 1 && sp.idx[a + d] < i) {
        a += d;
        d <<= 1;
      }
      b = a + d < hi - 1 ? a + d : hi - 1;
    } else {
      b = g;
      uint32_t d = 1;
      while (b - lo > d && sp.idx[b - d] >= i) {
        b -= d;
        d <<= 1;
      }
      a = b - lo > d ? b - d : lo;
    }
    lo = a + 1;
    hi = b;
  }
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (sp.idx[mid] < i) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <int R, typename PosFn>
__device__ __forceinline__ void classify_batch_tree(const uint64_t (&x)[R], uint32_t (&b)[R],
                                                    PosFn pos_of, const Splitters& sp) {
  uint32_t j[R];
  uint64_t ub[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    j[r] = 1;
    ub[r] = ~0ULL;
  }
  for (int l = 0; l < sp.logK; ++l) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint64_t t = sp.tree[j[r]];
      const bool right = x[r] > t;
      j[r] = 2 * j[r] + (right ? 1u : 0u);
      ub[r] = right ? ub[r] : t;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    uint32_t bb = j[r] - (1u << sp.logK);
    if (!sp.ntb && bb < sp.nspl && ub[r] == x[r]) bb = tie_break(bb, x[r], pos_of(r), sp);
    b[r] = bb;
  }
}

// Same result through the leading-bits table: one table read per element, then
// a lower-bound search over the splitters of its bin (usually 0-2 of them).
// PAIRS: elements 2j and 2j+1 sit at consecutive positions whenever
// valid(2j) and valid(2j+1); when both tie with the same run of splitter keys,
// the second element's bucket is the first's or the next (splitter positions
// are distinct, so at most one more of them lies below it): one comparison
// instead of a search.
template <int R, bool PAIRS = false, typename PosFn, typename ValidFn>
__device__ __forceinline__ void classify_batch_table(const uint64_t (&x)[R], uint32_t (&b)[R],
                                                     PosFn pos_of, ValidFn valid,
                                                     const Splitters& sp) {
  // A key below the smallest splitter reads bin 0 and one above the largest
  // the last bin: each then finds no splitter on its far side, so no case
  // needs its own branch.
  uint32_t pr[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint64_t t = (x[r] > sp.lo ? x[r] - sp.lo : 0ull) >> sp.shift;
    pr[r] = sp.tbl[t < sp.tmax ? (uint32_t)t : sp.tmax];
  }
  bool prev_tied = false;
  uint32_t prev_b = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    uint32_t bb;
    bool tied = false;
    {
      uint32_t lo = pr[r] & 0xffffu, hi = pr[r] >> 16;
      const uint32_t end = hi;
      uint64_t ub = ~0ULL;
      // the bin's first splitter may already bound x (always so when a run of
      // copies of x fills the bin): then no search is needed
      if (lo < hi) {
        const uint64_t k0 = sp.key[lo];
        if (k0 >= x[r]) {
          hi = lo;
          ub = k0;
        } else {
          ++lo;
        }
      }
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint64_t km = sp.key[mid];
        if (km < x[r]) {
          lo = mid + 1;
        } else {
          hi = mid;
          ub = km;
        }
      }
      bb = lo;
      tied = !sp.ntb && bb < end && ub == x[r];
      if (tied) {
        if (PAIRS && (r & 1) && prev_tied && x[r] == x[r - 1] && valid(r - 1) && valid(r)) {
          const uint32_t re = sp.rend[bb];
          bb = prev_b + (prev_b < re && sp.idx[prev_b] < pos_of(r) ? 1u : 0u);
        } else {
          bb = tie_break(bb, x[r], pos_of(r), sp);
        }
      }
    }
    b[r] = bb;
    prev_tied = tied;
    prev_b = bb;
  }
}

template <int R, typename PosFn>
__device__ __forceinline__ void classify_batch(const uint64_t (&x)[R], uint32_t (&b)[R],
                                               PosFn pos_of, const Splitters& sp) {
  if (sp.mode == 0) classify_batch_tree<R>(x, b, pos_of, sp);
  else classify_batch_table<R>(x, b, pos_of, [](int) { return false; }, sp);
}

// The same for elements in consecutive-position pairs (see
// classify_batch_table); valid(e) says whether element e is a real element.
template <int R, typename PosFn, typename ValidFn>
__device__ __forceinline__ void classify_batch_pairs(const uint64_t (&x)[R], uint32_t (&b)[R],
                                                     PosFn pos_of, ValidFn valid,
                                                     const Splitters& sp) {
  if (sp.mode == 0) classify_batch_tree<R>(x, b, pos_of, sp);
  else classify_batch_table<R, true>(x, b, pos_of, valid, sp);
}


}  // namespace rsort
