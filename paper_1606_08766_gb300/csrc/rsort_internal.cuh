// rsort_internal.cuh -- device-side data structures, constants and helpers of
// librsort (robust multi-level sample sort on one GB300).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rsort.h"

namespace rsort {

// ---------------------------------------------------------------------------
// Tunables (defaults; a tune table may override the host-side ones)
// ---------------------------------------------------------------------------
constexpr int kPartThreads = 256;                 // classify / scatter CTA
constexpr int kPartWarps = kPartThreads / 32;
constexpr int kItems = 16;                        // keys per lane per sub-tile
constexpr int kWarpSpan = 32 * kItems;            // 512 consecutive keys per warp
constexpr int kSubTile = kPartThreads * kItems;   // 4096 keys staged per sub-tile
constexpr int kMaxK = 2048;                       // buckets per partition step
constexpr int kMaxKDeep = 512;                    // buckets at levels >= 2
constexpr int kMaxFine = 10240;                   // fine partitions of an overpartitioned step
constexpr int kBucketCap = 4096;                  // T_s: largest bucket one CTA sorts
constexpr int kTargetBucket = 1536;               // aim for this final bucket size
                                                  // (mostly below the 1024-key class)
constexpr int kSampleChunk = 8192;                // sample sort: pairs per CTA chunk
constexpr int kSampleThreads = 512;               // sample sort CTA
constexpr int kDeepOversample = 16;               // samples per bucket at levels >= 2
constexpr int kMaxLevels = 3;                     // partition levels before fallback
constexpr int kLocalThreads = 256;                // in-SM bucket sort CTA
constexpr int kLocalItems = 16;                   // kLocalThreads * kLocalItems = kBucketCap
constexpr int kRankMax = 64;                      // rank-by-counting up to this size
constexpr int kScanTile = 4096;                   // device scan tile (1024 x 4)
constexpr int kUnitMaxK = 1024;                   // buckets of the whole-unit scatter

// Where the elements of a final bucket live.
enum : uint16_t { kWhereOut = 0, kWhereTmp = 1, kWhereInput = 2 };
// How a final bucket is finished.
//   kKindSort     sort in one CTA; its elements arrive in position order
//   kKindCopy     already ordered (size 1, or an equality bucket of a stable level)
//   kKindBig      larger than one CTA sorts (after the last level)
//   kKindSortAny  sort in one CTA; its elements arrive in no particular order
enum : uint16_t { kKindSort = 0, kKindCopy = 1, kKindBig = 2, kKindSortAny = 3 };
// Work lists of the in-SM sort, one per size class (each has its own kernel):
// copy-through, <= kSmallCap keys, <= kMidCap keys, <= kBucketCap keys, oversize.
enum : int {
  kClassCopy = 0,
  kClassSmall = 1,   // <= kSmallCap keys
  kClassMid = 2,     // <= kMidCap keys
  kClassMedium = 3,  // <= kBucketCap keys
  kClassBig = 4,
  kNumClasses = 5
};
// Which in-SM algorithm finished a bucket (rsort_stats.algo_elems counts the
// elements each one handled):
enum : int {
  kAlgoRank = 0,     // rank-by-counting (tiny buckets)
  kAlgoBins = 1,     // equal-width bins + ranking inside crowded-free bins
  kAlgoBitonic = 2,  // bitonic sort (a bin held more than kBinLimit keys)
  kAlgoQuick = 3,    // quicksort with tree-median pivots (opt-in medium path)
  kAlgoMerge = 4,    // oversize merge sort through global memory
  kAlgoInOrder = 5,  // all keys equal and already in position order
  kNumAlgos = 6
};
constexpr uint32_t kSmallCap = 1024;   // capacity of the small-class kernel
constexpr uint32_t kMidCap = 2048;     // capacity of the mid-class kernel
// In-SM algorithm of a size class (LocalPlan::algo):
enum : uint8_t { kLocalBins = 0, kLocalQuick = 1, kLocalBitonic = 2 };

// The size-dependent choice of the in-SM sort, fixed per call (defaults from
// hand sweeps; an autotuned table may replace them):
//   buckets of at most small_cap keys go to the small-class kernel, at most
//   mid_cap to the mid-class kernel, the rest (<= kBucketCap) to the medium
//   one; rank_max bounds rank-by-counting; algo[class - 1] picks bins (with
//   bitonic for clustered keys), quicksort (mid / medium only) or bitonic.
struct LocalPlan {
  uint32_t small_cap = 1024;  // <= kSmallCap
  uint32_t mid_cap = 2048;    // small_cap..kMidCap
  uint32_t rank_max = 64;     // <= 128 (the small kernel's threads)
  uint8_t algo[3] = {kLocalBins, kLocalBins, kLocalBins};  // small, mid, medium
};

// A segment waiting to be partitioned (input of a level).
struct SegIn {
  uint64_t start;   // absolute position (identical in every buffer)
  uint32_t m;       // elements
  uint32_t k_hint;  // buckets requested (>= 1), or 0 to choose from m
};

// A segment being partitioned at the current level (written by the plan).
struct LevelSeg {
  uint64_t start;
  uint64_t seed;
  uint64_t samp_off;    // first sample slot
  uint64_t chunk_off;   // first global chunk id
  uint64_t hist_off;    // first histogram counter
  uint64_t schunk_off;  // first sample-sort chunk id
  uint64_t bkt_off;     // first global bucket id
  uint64_t delta;       // start - (sum of sizes of earlier segments), mod 2^64
  uint32_t m;
  uint32_t k;
  uint32_t S;
  uint32_t nchunks;
  uint32_t nschunks;
  uint32_t nunits;      // histogram units: nchunks (CTA chunks) or 8 * nchunks (warp sub-chunks)
  uint32_t W;           // keys per chunk of this segment (all chunks equal but the last)
  uint32_t pad;
};

// A bucket handed to the in-SM sort.
struct FinalItem {
  uint64_t start;     // absolute position of its first element
  uint64_t idx_base;  // position - idx_base = original position (input only)
  uint32_t size;
  uint16_t where;
  uint16_t kind;
};

// Device-resident control block of one call.
struct DevState {
  uint32_t nseg[2];         // segment lists (ping-pong by level parity)
  uint32_t nfinal_c[kNumClasses];  // final items per size class
  uint32_t cursor_c[kNumClasses];  // work counters of the in-SM sort kernels
  uint64_t class_elems[kNumClasses];  // elements handed to each size class
  uint64_t algo_elems[kNumAlgos];     // elements finished by each in-SM algorithm
  LocalPlan local;                    // the call's in-SM size classes and algorithms
  uint32_t error;           // capacity / wait errors (bit flags)
  uint32_t max_bucket_l1;   // largest level-1 bucket
  uint32_t levels_used;
  uint32_t cur_nseg;        // segments of the level being processed
  uint64_t total_samples;
  uint64_t total_chunks;
  uint64_t total_hist;
  uint64_t total_schunks;
  uint64_t total_buckets;
  uint64_t big_items;       // buckets that needed the oversize fallback
  uint64_t level_elems[4];  // elements partitioned at levels 1..4
  // level 1's order (LevelParams::stable == kOrderAuto): equality buckets
  // among its buckets, its bucket count, and whether its buckets hold their
  // elements in position order (written by level 1's collect for the levels
  // after it)
  uint32_t l1_eq;
  uint32_t l1_nb;
  uint32_t l1_ordered;
};

// LevelParams::stable / in_order value: decided on the device.  Level 1
// keeps input order when at least 1/kAutoOrderShare of its buckets are
// equality buckets (copies of one key: kept in position order they are final
// and skip the levels below), and ranks by atomics otherwise; in_order ==
// kOrderAuto means "as level 1 left them".
constexpr int kOrderAuto = 2;
constexpr uint32_t kAutoOrderShare = 16;

__device__ __forceinline__ bool l1_auto_ordered(const DevState* st) {
  return st->l1_nb > 0 && (uint64_t)st->l1_eq * kAutoOrderShare >= st->l1_nb;
}

enum : uint32_t {
  kErrSampleCap = 1u << 0,
  kErrHistCap = 1u << 1,
  kErrChunkCap = 1u << 2,
  kErrSegCap = 1u << 3,
  kErrFinalCap = 1u << 4,
  kErrSchunkCap = 1u << 5,
  kErrBucketCap = 1u << 6,
  kErrBadOffsets = 1u << 7,
  kErrWait = 1u << 8,         // a bounded wait on a bulk copy gave up
};

// Parameters of one level, fixed on the host.
struct LevelParams {
  int level;            // 1-based
  uint32_t W;           // keys per classify/scatter chunk
  uint64_t seed;
  uint64_t samp_cap, hist_cap, chunk_cap, seg_cap, final_cap, schunk_cap, bucket_cap;
  int level1_oversample;  // 1: a = 16 ceil(log2 k) for hinted k (the paper's rule)
  int classifier;         // 0: splitter tree, 1: leading-bits table
  int warp_direct;        // 1: per-warp sub-chunks scattered straight to HBM
  int wide_scatter_k;     // levels with at least this many buckets scatter 4096-key sub-tiles
  uint32_t target_bucket; // automatic fan-out aims at buckets of this many keys
  // per segment-size class c = ceil(log2 m): the fan-out target for segments
  // of that class (0: target_bucket)
  uint32_t target_by_class[33] = {};
  int no_tie_break = 0;   // 1: classify by key only (the NTB ablation)
  int stable = 1;         // 1: buckets keep input order (the partition step's
                          // layout); 0: a full sort's level, ranked by
                          // shared-memory atomics (the in-SM sort orders
                          // (key, position) pairs, so the result is the same);
                          // kOrderAuto (level 1 only): decided on the device
  int in_order = 1;       // 1: the level's segments hold their elements in
                          // position order (level 1, or after a stable level);
                          // kOrderAuto: as level 1 left them
  int unit_scatter = 1;   // 1: a stable level with at most kUnitMaxK buckets
                          // stores bucket ids when classifying and scatters
                          // whole 8-element units (unit_scatter.cu)
  int atomic_scatter = 0; // 1: an unordered level scatters with the
                          // small-footprint atomic-ranked kernel
  int bulk_classify = 0;  // 1: the id-storing classify stages its keys by
                          // bulk copies (16-byte aligned key arrays)
};

// AMS-sort overpartitioning of a one-segment partition step: b*k fine
// partitions are counted, grouped greedily into k outputs, and the k-1 group
// boundaries become the splitters of the ordinary k-way step.
struct Overpart {
  uint32_t k;            // outputs (the segment's k)
  uint32_t over;         // b >= 2
  uint32_t* fine_cnt;    // [b*k] scratch counters (cleared by the launch)
  uint32_t* prefix;      // [b*k + 1] scratch: prefix sums of the fine sizes
  uint64_t* search;      // [3] scratch: bracket of the greedy's bound, best candidate
  uint64_t* fine_out;    // [b*k] fine partition sizes, or nullptr
  uint32_t* first_out;   // [k+1] first fine partition of every output, or nullptr
};

// Element source / destination of a level.
struct Src {
  const uint64_t* key;
  const uint32_t* idx;  // nullptr: the original position is implicit
  int map_f64;          // keys need the float64 order map on load
  // [n + 16] bucket of every element by position, written by the classify
  // pass and read by the scatter (nullptr: the scatter classifies again)
  uint16_t* bid = nullptr;
};
struct Dst {
  uint64_t* key;
  uint32_t* idx;
};

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------

// splitmix64 (Steele, Lea & Flood 2014): output c of the stream at state s.
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t s, uint64_t c) {
  uint64_t z = s + (c + 1) * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Order map of binary64 bit patterns: negative -> all bits flipped,
// non-negative -> sign bit flipped.  Its inverse restores the original bits.
__device__ __forceinline__ uint64_t f64_to_ordered(uint64_t u) {
  return u ^ ((uint64_t)((int64_t)u >> 63) | 0x8000000000000000ULL);
}
__device__ __forceinline__ uint64_t ordered_to_f64(uint64_t o) {
  return o ^ ((uint64_t)(~((int64_t)o >> 63)) | 0x8000000000000000ULL);
}

__device__ __forceinline__ bool pair_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka < kb || (ka == kb && ia < ib);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive block scan of one u64 per thread (NT threads, NT % 32 == 0).
// sm must hold NT/32 u64.  Returns the exclusive prefix; *total gets the sum.
template <int NT>
__device__ __forceinline__ uint64_t block_excl_scan_u64(uint64_t v, uint64_t* total,
                                                        uint64_t* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[w] = x;
  __syncthreads();
  if (w == 0) {
    uint64_t s = (lane < NT / 32) ? sm[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) sm[lane] = s;
  }
  __syncthreads();
  uint64_t prefix = (w > 0 ? sm[w - 1] : 0) + x - v;
  *total = sm[NT / 32 - 1];
  __syncthreads();
  return prefix;
}

// In-place bitonic sort of P (a power of two) (key, idx) pairs in shared
// memory by NT threads; callers pad with (UINT64_MAX, UINT32_MAX).
template <int NT>
__device__ __forceinline__ void block_bitonic_sort(uint64_t* sk, uint32_t* si, int P) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < (P >> 1); t += NT) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t a = sk[lo], b = sk[hi];
        const uint32_t ia = si[lo], ib = si[hi];
        const bool gt = a > b || (a == b && ia > ib);
        if (gt == up) {
          sk[lo] = b; sk[hi] = a;
          si[lo] = ib; si[hi] = ia;
        }
      }
    }
  }
  __syncthreads();
}

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// Appends a final bucket to the work list of its size class
// (items holds kNumClasses lists of cap entries each).
__device__ __forceinline__ void push_final(DevState* st, FinalItem* items, uint64_t cap,
                                           const FinalItem& f, uint32_t err_flag) {
  const int cls = f.kind == kKindCopy ? kClassCopy
                  : f.kind == kKindBig ? kClassBig
                  : (f.size <= st->local.small_cap
                         ? kClassSmall
                         : (f.size <= st->local.mid_cap ? kClassMid : kClassMedium));
  // one atomic per (warp, class): the lanes appending to the same list share it
  const uint32_t act = __activemask();
  const uint32_t peers = __match_any_sync(act, (uint32_t)cls);
  const int leader = __ffs(peers) - 1;
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  const uint32_t keys = __reduce_add_sync(peers, f.size);
  if (lane == leader) {
    base = atomicAdd(&st->nfinal_c[cls], (uint32_t)__popc(peers));
    atomicAdd((unsigned long long*)&st->class_elems[cls], (unsigned long long)keys);
  }
  base = __shfl_sync(peers, base, leader);
  uint32_t lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  const uint32_t slot = base + __popc(peers & lt);
  if (slot < cap) items[(uint64_t)cls * cap + slot] = f;
  else atomicOr(&st->error, err_flag);
}
__host__ __device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// Per-warp counter rows of the scatters are padded to an even length so a warp
// can clear its row with 32-bit stores without touching the next warp's row.
__host__ __device__ inline uint32_t cnt_stride(uint32_t kmax) { return (kmax + 1) & ~1u; }

__host__ __device__ __forceinline__ uint32_t next_pow2_u32(uint32_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}
__host__ __device__ __forceinline__ int log2_u32(uint32_t p) {  // p a power of two
  int l = 0;
  while ((1u << l) < p) ++l;
  return l;
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// Profiling hook owned by the context: CUDA events around every launch.
struct KernelTimer {
  void begin(const char* name, cudaStream_t s);
  void end(cudaStream_t s);
  void* impl = nullptr;
};

struct LaunchEnv {
  cudaStream_t stream;
  int num_sms;
  KernelTimer* timer;   // may be null
  uint64_t* launches;   // launch counter
  LocalPlan local;      // in-SM size classes and algorithms (written to DevState at init)
};

void launch_init_plain(const LaunchEnv& e, DevState* st, SegIn* list0, FinalItem* items,
                       uint64_t n, uint32_t k1, int direct, uint64_t final_cap);
void launch_level(const LaunchEnv& e, const LevelParams& P, DevState* st, const SegIn* list_in,
                  SegIn* list_out, LevelSeg* segs, Src src, Dst dst, uint16_t dst_where,
                  uint64_t* samp_key, uint32_t* samp_idx, uint64_t* ssamp_key,
                  uint32_t* ssamp_idx, uint32_t* hist, uint32_t* block_sums, FinalItem* items,
                  int kmax_level, int last_level, int emit_final, uint64_t* offsets_out,
                  uint64_t n_total, int unmap_out, const Overpart* op = nullptr);
void launch_init_segments(const LaunchEnv& e, DevState* st, const uint64_t* offsets,
                          uint32_t nseg, uint64_t n, SegIn* list_l1, FinalItem* items,
                          uint64_t seg_cap, uint64_t final_cap);
void set_partition_kernel_attributes();
// Binary-tree median approximation of n <= 2^24 keys (median_kernels.cu);
// k in {2, 4, 8, 16, 32}.  Returns false for an unsupported k.
size_t tree_median_scratch_bytes(uint64_t n);
bool launch_tree_median(const LaunchEnv& e, const uint64_t* keys, uint32_t n, int f64,
                        uint32_t k, uint64_t seed, void* scratch, uint64_t* out_pos);
void launch_plain_groups(const LaunchEnv& e, const uint64_t* offsets, uint32_t k,
                         uint64_t* fine_out, uint32_t* first_out);
void set_local_kernel_attributes();
// Classify with stored bucket ids and the whole-unit scatter (unit_scatter.cu).
void set_unit_scatter_attributes();
bool unit_scatter_fits(uint32_t kmax);
void launch_classify_ids(const LaunchEnv& e, const LevelParams& P, DevState* st,
                         const LevelSeg* segs, Src src, const uint64_t* ssk, const uint32_t* ssi,
                         uint32_t* hist, uint32_t kmax, int mode, const char* name);
bool atomic_scatter_fits(uint32_t kmax);
void launch_scatter_atomic(const LaunchEnv& e, const LevelParams& P, DevState* st,
                           const LevelSeg* segs, Src src, const uint32_t* hist_scan, Dst dst,
                           uint32_t kmax, int unmap_out, const char* name);
void launch_scatter_units(const LaunchEnv& e, const LevelParams& P, DevState* st,
                          const LevelSeg* segs, Src src, const uint32_t* hist_scan, Dst dst,
                          uint32_t kmax, int unmap_out, const char* name);
void launch_local_sort(const LaunchEnv& e, DevState* st, const FinalItem* items,
                       uint64_t item_cap, const uint64_t* in_key, Dst out, Dst tmp, int f64);

}  // namespace rsort
