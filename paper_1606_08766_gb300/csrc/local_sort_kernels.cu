// local_sort_kernels.cu -- the in-SM sort of every final bucket, chosen by
// bucket size as the paper chooses its algorithm by input size (Section 6,
// "four algorithms cover the entire range"; Appendix "Parameter Tuning"):
//
//   size 1 or equality bucket  copy through (the stable scatter already left
//                              the elements in position order)
//   size <= kBucketCap         cta_sort_pairs (cta_sort.cuh): rank-by-counting
//                              for tiny buckets, equal-width bins + rank-by-
//                              counting for the rest, bitonic when keys cluster
//   larger (only after the     merge sort through global memory by one CTA:
//   last partition level)      bitonic-sorted runs, then pairwise merges
//
// Buckets are taken from a device work list with an atomic cursor by a
// persistent grid.  The final store restores float64 bit patterns.
#include "cta_sort.cuh"
#include "rsort_internal.cuh"

namespace rsort {

namespace {

struct Scope {
  const LaunchEnv& e;
  Scope(const LaunchEnv& env, const char* name) : e(env) {
    if (e.timer) e.timer->begin(name, e.stream);
  }
  ~Scope() {
    if (e.timer) e.timer->end(e.stream);
    if (e.launches) ++*e.launches;
  }
};

struct Bufs {
  const uint64_t* in_key;
  Dst out;
  Dst tmp;
  int f64;
};

__device__ __forceinline__ void load_elem(const Bufs& B, const FinalItem& f, uint64_t j,
                                          uint64_t& k, uint32_t& i) {
  const uint64_t pos = f.start + j;
  if (f.where == kWhereInput) {
    const uint64_t raw = B.in_key[pos];
    k = B.f64 ? f64_to_ordered(raw) : raw;
    i = (uint32_t)(pos - f.idx_base);
  } else {
    const Dst& s = f.where == kWhereOut ? B.out : B.tmp;
    k = s.key[pos];
    i = s.idx[pos];
  }
}

__device__ __forceinline__ void store_out(const Bufs& B, uint64_t pos, uint64_t k, uint32_t i) {
  B.out.key[pos] = B.f64 ? ordered_to_f64(k) : k;
  B.out.idx[pos] = i;
}

// Merge-path split: number of elements of A among the first d outputs of
// merge(A, B); (key, idx) pairs are distinct.
__device__ __forceinline__ uint64_t merge_split(const uint64_t* ak, const uint32_t* ai, uint64_t na,
                                                const uint64_t* bk, const uint32_t* bi, uint64_t nb,
                                                uint64_t d) {
  uint64_t lo = d > nb ? d - nb : 0;
  uint64_t hi = d < na ? d : na;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (pair_less(ak[mid], ai[mid], bk[d - 1 - mid], bi[d - 1 - mid])) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Oversize bucket (more than kBucketCap elements after the last partition
// level; the sampling makes this vanishingly rare).  One CTA sorts runs of
// kBucketCap in shared memory, then merges runs pairwise through the two
// global buffers.  The bucket's range in the other buffer is free: other
// levels only write ranges of segments that are still being partitioned.
__device__ void sort_big(const Bufs& B, const FinalItem& f, uint64_t* sk, uint32_t* si) {
  constexpr int NT = kLocalThreads;
  const uint64_t m = f.size;
  Dst A = f.where == kWhereOut ? B.out : B.tmp;
  Dst C = f.where == kWhereOut ? B.tmp : B.out;
  // runs
  for (uint64_t r0 = 0; r0 < m; r0 += kBucketCap) {
    const int len = (int)umin64(kBucketCap, m - r0);
    for (int t = threadIdx.x; t < kBucketCap; t += NT) {
      if (t < len) {
        sk[t] = A.key[f.start + r0 + t];
        si[t] = A.idx[f.start + r0 + t];
      } else {
        sk[t] = ~0ULL;
        si[t] = ~0u;
      }
    }
    block_bitonic_sort<NT>(sk, si, kBucketCap);
    for (int t = threadIdx.x; t < len; t += NT) {
      C.key[f.start + r0 + t] = sk[t];
      C.idx[f.start + r0 + t] = si[t];
    }
    __syncthreads();
  }
  Dst cur = C, nxt = A;
  constexpr int E = 8;
  for (uint64_t w = kBucketCap; w < m; w *= 2) {
    for (uint64_t p0 = 0; p0 < m; p0 += 2 * w) {
      const uint64_t na = umin64(w, m - p0);
      const uint64_t nb = p0 + w < m ? umin64(w, m - p0 - w) : 0;
      const uint64_t* ak = cur.key + f.start + p0;
      const uint32_t* ai = cur.idx + f.start + p0;
      const uint64_t* bk = ak + na;
      const uint32_t* bi = ai + na;
      for (uint64_t d0 = (uint64_t)threadIdx.x * E; d0 < na + nb; d0 += (uint64_t)NT * E) {
        uint64_t i = merge_split(ak, ai, na, bk, bi, nb, d0);
        uint64_t j = d0 - i;
        for (int e = 0; e < E && d0 + e < na + nb; ++e) {
          bool take_a;
          if (i >= na) take_a = false;
          else if (j >= nb) take_a = true;
          else take_a = pair_less(ak[i], ai[i], bk[j], bi[j]);
          const uint64_t o = f.start + p0 + d0 + e;
          if (take_a) { nxt.key[o] = ak[i]; nxt.idx[o] = ai[i]; ++i; }
          else { nxt.key[o] = bk[j]; nxt.idx[o] = bi[j]; ++j; }
        }
      }
    }
    __syncthreads();
    Dst t = cur; cur = nxt; nxt = t;
  }
  // result lives in cur; move it to the output with the final key map
  for (uint64_t t = threadIdx.x; t < m; t += NT) {
    const uint64_t pos = f.start + t;
    store_out(B, pos, cur.key[pos], cur.idx[pos]);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kLocalThreads)
k_local_sort(DevState* st, const FinalItem* items, uint64_t item_cap, Bufs B) {
  constexpr int NT = kLocalThreads, IT = kLocalItems;
  static_assert(NT * IT == kBucketCap, "one CTA holds one whole bucket");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CtaSortSmem s;
  s.k = (uint64_t*)smem_raw;                // [kBucketCap]
  s.i = (uint32_t*)(s.k + kBucketCap);      // [kBucketCap]
  s.hist = s.i + kBucketCap;                // [kBucketCap]
  __shared__ uint64_t red[2 * NT / 32];
  __shared__ uint64_t scan_sm[NT / 32];
  __shared__ uint32_t s_item;
  const uint64_t nitems = umin64(st->nfinal, item_cap);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&st->final_cursor, 1u);
    __syncthreads();
    const uint32_t it = s_item;
    __syncthreads();
    if (it >= nitems) break;
    const FinalItem f = items[it];
    const uint32_t m = f.size;
    if (f.kind == kKindCopy) {
      if (f.where == kWhereOut && !B.f64) continue;  // already in place
      for (uint32_t t = threadIdx.x; t < m; t += NT) {
        uint64_t k; uint32_t i;
        load_elem(B, f, t, k, i);
        store_out(B, f.start + t, k, i);
      }
      continue;
    }
    if (f.kind == kKindBig) {
      sort_big(B, f, s.k, s.i);
      continue;
    }
    uint64_t key[IT];
    uint32_t idx[IT];
#pragma unroll
    for (int r = 0; r < IT; ++r) {
      const uint32_t e = r * NT + threadIdx.x;
      if (e < m) load_elem(B, f, e, key[r], idx[r]);
    }
    cta_sort_pairs<NT, IT>(key, idx, m, true, s, red, scan_sm);
    for (uint32_t t = threadIdx.x; t < m; t += NT) store_out(B, f.start + t, s.k[t], s.i[t]);
    __syncthreads();
  }
}

}  // namespace

void set_local_kernel_attributes() {
  cudaFuncSetAttribute(k_local_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kBucketCap * (8 + 4 + 4));
}

void launch_local_sort(const LaunchEnv& e, DevState* st, const FinalItem* items,
                       uint64_t item_cap, const uint64_t* in_key, Dst out, Dst tmp, int f64) {
  Bufs B;
  B.in_key = in_key;
  B.out = out;
  B.tmp = tmp;
  B.f64 = f64;
  const int smem = kBucketCap * (8 + 4 + 4);
  Scope sc(e, "local_sort");
  k_local_sort<<<e.num_sms * 3, kLocalThreads, smem, e.stream>>>(st, items, item_cap, B);
}

}  // namespace rsort
