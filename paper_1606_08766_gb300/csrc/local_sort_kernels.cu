// local_sort_kernels.cu -- the in-SM sort of every final bucket, chosen by
// bucket size as the paper chooses its algorithm by input size (Section 6,
// "four algorithms cover the entire range"; Appendix "Parameter Tuning"):
//
//   size 1 or equality bucket  copy through (a stable scatter already left
//   of a stable level          the elements in position order)
//   size <= kBucketCap         cta_sort_pairs (cta_sort.cuh): rank-by-counting
//                              for tiny buckets, equal-width bins + rank-by-
//                              counting for the rest, bitonic when keys cluster
//   larger (only after the     merge sort through global memory by one CTA:
//   last partition level)      bitonic-sorted runs, then pairwise merges
//
// The sorted buckets come in three size classes, each its own kernel with a
// CTA shape that fits it: <= 1024 keys (128 threads, 10 CTAs per SM),
// <= 2048 keys (128 threads, 5 per SM), <= 4096 keys (256 threads, 2 per SM).
// Buckets are taken from a device work list with an atomic cursor by a
// persistent grid.  The final store restores float64 bit patterns.
#include "cta_quicksort.cuh"
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

template <int NT, int IT>
__device__ __forceinline__ void load_bucket(const Bufs& B, const FinalItem& f,
                                            uint64_t (&key)[IT], uint32_t (&idx)[IT]) {
#pragma unroll
  for (int r = 0; r < IT; ++r) {
    const uint32_t e = r * NT + threadIdx.x;
    if (e < f.size) load_elem(B, f, e, key[r], idx[r]);
  }
}

// Next item of size class cls for this CTA (atomic work counter), or -1.
__device__ __forceinline__ int64_t next_item(DevState* st, int cls, uint64_t cap,
                                             uint32_t* s_item) {
  if (threadIdx.x == 0) *s_item = atomicAdd(&st->cursor_c[cls], 1u);
  __syncthreads();
  const uint32_t it = *s_item;
  __syncthreads();
  return it < umin64(st->nfinal_c[cls], cap) ? (int64_t)it : -1;
}

// The same in two steps: claim_item() sends the atomic (thread 0 keeps its
// result in a register, so nothing waits for it), take_item() publishes the
// claimed item to the CTA later, after the atomic's round trip has passed in
// other work.
__device__ __forceinline__ uint32_t claim_item(DevState* st, int cls) {
  return threadIdx.x == 0 ? atomicAdd(&st->cursor_c[cls], 1u) : 0u;
}
__device__ __forceinline__ int64_t take_item(const DevState* st, int cls, uint64_t cap,
                                             uint32_t claimed, uint32_t* s_item) {
  if (threadIdx.x == 0) *s_item = claimed;
  __syncthreads();
  const uint32_t it = *s_item;
  __syncthreads();
  return it < umin64(st->nfinal_c[cls], cap) ? (int64_t)it : -1;
}

// Resident CTAs per SM of the small class: the sort is latency-bound per
// bucket, so more buckets in flight per SM pay more than registers (10 CTAs
// of 128 threads measured 17% faster than 6 at 2^28 keys).
constexpr int kSmallPerSm = 10;

// Buckets of up to NT*IT keys, sorted by one CTA each (cta_sort_pairs),
// MINB CTAs resident per SM.
template <int NT, int IT, int CLS, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_local_sort(DevState* st, const FinalItem* items, uint64_t cap, Bufs B) {
  constexpr int kCap = NT * IT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CtaSortSmem s;
  s.k = (uint64_t*)smem_raw;          // [kCap]
  s.i = (uint32_t*)(s.k + kCap);      // [kCap]
  s.hist = s.i + kCap;                // [kCap]
  __shared__ uint64_t red[2 * NT / 32];
  __shared__ uint64_t scan_sm[NT / 32];
  __shared__ uint32_t s_item;
  const FinalItem* list = items + (uint64_t)CLS * cap;
  const uint32_t rank_max = st->local.rank_max;
  const bool bitonic = st->local.algo[CLS - kClassSmall] == kLocalBitonic;
  uint64_t key[IT];
  uint32_t idx[IT];
  int64_t it = next_item(st, CLS, cap, &s_item);
  FinalItem f{};
  if (it >= 0) {
    f = list[it];
    load_bucket<NT, IT>(B, f, key, idx);
  }
  while (it >= 0) {
    // the next bucket is claimed now (the atomic's round trip passes during
    // this sort) and loaded into the registers as soon as this one's pairs
    // sit in shared memory (the classes above the small one, whose buckets
    // take long enough to finish), else after sorting, so its loads are in
    // flight while this one is finished and stored (the small class has too
    // few registers to hold the claim across the sort)
    const uint32_t claimed = claim_item(st, CLS);
    int64_t it2 = -1;
    FinalItem f2{};
    auto claim_next = [&] {
      it2 = take_item(st, CLS, cap, claimed, &s_item);
      if (it2 >= 0) {
        f2 = list[it2];
        load_bucket<NT, IT>(B, f2, key, idx);
      }
    };
    if constexpr (CLS == kClassSmall) {
      cta_sort_pairs<NT, IT>(key, idx, f.size, [&] { return list[it].kind == kKindSort; }, s,
                             red, scan_sm, st->algo_elems, rank_max, bitonic);
      claim_next();
    } else {
      cta_sort_pairs<NT, IT>(key, idx, f.size, [&] { return list[it].kind == kKindSort; }, s,
                             red, scan_sm, st->algo_elems, rank_max, bitonic, claim_next);
    }
    for (uint32_t t = threadIdx.x; t < f.size; t += NT) store_out(B, f.start + t, s.k[t], s.i[t]);
    __syncthreads();
    it = it2;
    f = f2;
  }
}

// The medium class sorted by quicksort instead (tunable "medium_sort" = 1):
// pivots from the binary-tree median approximation of a sample of every
// segment (cta_quicksort.cuh).  The result is the same; the bins of
// cta_sort_pairs measured faster, so this is an alternative, not the default.
template <int NT, int CAP, int CLS>
__global__ void __launch_bounds__(NT, 1)
k_local_quicksort(DevState* st, const FinalItem* items, uint64_t cap, Bufs B, uint64_t seed) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const QsSmem q = qs_carve(smem_raw, CAP);
  __shared__ uint64_t scan_sm[NT / 32];
  __shared__ uint64_t red[2 * NT / 32];
  __shared__ uint32_t s_item;
  const FinalItem* list = items + (uint64_t)CLS * cap;
  for (;;) {
    const int64_t it = next_item(st, CLS, cap, &s_item);
    if (it < 0) break;
    const FinalItem f = list[it];
    count_algo(st->algo_elems, kAlgoQuick, f.size);
    for (uint32_t t = threadIdx.x; t < f.size; t += NT) {
      uint64_t k;
      uint32_t i;
      load_elem(B, f, t, k, i);
      q.ak[t] = k;
      q.ai[t] = i;
    }
    __syncthreads();
    cta_quicksort_pairs<NT>(q, f.size, splitmix64_at(seed, (uint64_t)it), scan_sm, red);
    for (uint32_t t = threadIdx.x; t < f.size; t += NT) store_out(B, f.start + t, q.ak[t], q.ai[t]);
    __syncthreads();
  }
}

// Copy-through buckets (size 1, or equality buckets already in position
// order): a coalesced copy that restores float64 bit patterns.
__global__ void __launch_bounds__(256)
k_local_copy(DevState* st, const FinalItem* items, uint64_t cap, Bufs B) {
  __shared__ uint32_t s_item;
  const FinalItem* list = items + (uint64_t)kClassCopy * cap;
  for (;;) {
    const int64_t it = next_item(st, kClassCopy, cap, &s_item);
    if (it < 0) break;
    const FinalItem f = list[it];
    if (f.where == kWhereOut && !B.f64) continue;  // already in place
    for (uint32_t t = threadIdx.x; t < f.size; t += blockDim.x) {
      uint64_t k;
      uint32_t i;
      load_elem(B, f, t, k, i);
      store_out(B, f.start + t, k, i);
    }
  }
}

// Oversize buckets (after the last partition level; vanishingly rare).
__global__ void __launch_bounds__(kLocalThreads)
k_local_big(DevState* st, const FinalItem* items, uint64_t cap, Bufs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* sk = (uint64_t*)smem_raw;
  uint32_t* si = (uint32_t*)(sk + kBucketCap);
  __shared__ uint32_t s_item;
  const FinalItem* list = items + (uint64_t)kClassBig * cap;
  for (;;) {
    const int64_t it = next_item(st, kClassBig, cap, &s_item);
    if (it < 0) break;
    count_algo(st->algo_elems, kAlgoMerge, list[it].size);
    sort_big(B, list[it], sk, si);
  }
}

constexpr int kSmallThreads = 128;
constexpr int kSmallItems = kSmallCap / kSmallThreads;  // 8
static_assert(kSmallThreads * kSmallItems == (int)kSmallCap, "small class fits one CTA");
// The mid class (1025..2048 keys): 128 threads of 16 slots, 5 CTAs per SM
// (256 threads of 8 slots measured 3 % slower: every bucket's fixed work --
// scans, reductions -- is spread over fewer keys per thread).
constexpr int kMidThreads = 128;
constexpr int kMidItems = (int)kMidCap / kMidThreads;  // 16
constexpr int kMidPerSm = 5;
static_assert(kMidThreads * kMidItems == (int)kMidCap, "mid class fits one CTA");
// The medium class (2049..4096 keys): 256 threads of 16 slots, two CTAs per
// SM (with the next bucket claimed and loaded early, this measured 2 %
// faster than 512 threads of 8 slots, which had spread every bucket's fixed
// work over half the keys per thread).
constexpr int kMediumThreads = 256;
constexpr int kMediumItems = kBucketCap / kMediumThreads;  // 16
static_assert(kMediumThreads * kMediumItems == kBucketCap, "medium class fits one CTA");

}  // namespace

void set_local_kernel_attributes() {
  cudaFuncSetAttribute(k_local_sort<kSmallThreads, kSmallItems, kClassSmall, kSmallPerSm>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallCap * kCtaSortBytesPerElem);
  cudaFuncSetAttribute(k_local_sort<kMidThreads, kMidItems, kClassMid, kMidPerSm>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMidCap * kCtaSortBytesPerElem);
  cudaFuncSetAttribute(k_local_quicksort<kLocalThreads, (int)kMidCap, kClassMid>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qs_smem_bytes(kMidCap));
  cudaFuncSetAttribute(k_local_sort<kMediumThreads, kMediumItems, kClassMedium, 2>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, kBucketCap * kCtaSortBytesPerElem);
  cudaFuncSetAttribute(k_local_quicksort<kLocalThreads, kBucketCap, kClassMedium>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qs_smem_bytes(kBucketCap));
  cudaFuncSetAttribute(k_local_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kBucketCap * 12);
}

void launch_local_sort(const LaunchEnv& e, DevState* st, const FinalItem* items,
                       uint64_t item_cap, const uint64_t* in_key, Dst out, Dst tmp, int f64) {
  Bufs B;
  B.in_key = in_key;
  B.out = out;
  B.tmp = tmp;
  B.f64 = f64;
  {
    Scope sc(e, "local_copy");
    k_local_copy<<<e.num_sms * 4, 256, 0, e.stream>>>(st, items, item_cap, B);
  }
  {
    Scope sc(e, "local_sort");
    k_local_sort<kSmallThreads, kSmallItems, kClassSmall, kSmallPerSm>
        <<<e.num_sms * kSmallPerSm, kSmallThreads, kSmallCap * kCtaSortBytesPerElem, e.stream>>>(st, items, item_cap, B);
  }
  {
    Scope sc(e, "local_sort_mid");
    if (e.local.algo[kClassMid - kClassSmall] == kLocalQuick)
      k_local_quicksort<kLocalThreads, (int)kMidCap, kClassMid>
          <<<e.num_sms * 2, kLocalThreads, qs_smem_bytes(kMidCap), e.stream>>>(
              st, items, item_cap, B, 0x243f6a8885a308d3ULL);
    else
      k_local_sort<kMidThreads, kMidItems, kClassMid, kMidPerSm>
          <<<e.num_sms * kMidPerSm, kMidThreads, kMidCap * kCtaSortBytesPerElem, e.stream>>>(
              st, items, item_cap, B);
  }
  {
    Scope sc(e, "local_sort_medium");
    if (e.local.algo[kClassMedium - kClassSmall] == kLocalQuick)
      k_local_quicksort<kLocalThreads, kBucketCap, kClassMedium>
          <<<e.num_sms * 2, kLocalThreads, qs_smem_bytes(kBucketCap), e.stream>>>(
              st, items, item_cap, B, 0x9e3779b97f4a7c15ULL);
    else
      k_local_sort<kMediumThreads, kMediumItems, kClassMedium, 2>
          <<<e.num_sms * 2, kMediumThreads, kBucketCap * kCtaSortBytesPerElem, e.stream>>>(
              st, items, item_cap, B);
  }
  {
    Scope sc(e, "local_big");
    k_local_big<<<e.num_sms, kLocalThreads, kBucketCap * 12, e.stream>>>(st, items, item_cap, B);
  }
}

}  // namespace rsort
