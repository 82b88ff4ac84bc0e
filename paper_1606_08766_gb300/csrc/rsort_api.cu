// rsort_api.cu -- the C ABI of librsort (see include/rsort.h): context and
// scratch management, the host-side plan of a sort, and the launch sequence.
//
// Host code here only validates arguments, sizes scratch and enqueues kernels;
// every step of the method runs in the kernels of partition_kernels.cu and
// local_sort_kernels.cu.  Nothing here synchronises unless a caller asks for
// a read-back (stats, rsort_check, phase times).
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "rsort_internal.cuh"

namespace rsort {

// ---------------------------------------------------------------------------
// Kernel timer: a pair of CUDA events around every launch, resolved lazily.
// ---------------------------------------------------------------------------
cudaEvent_t TimerImpl::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void TimerImpl::resolve() {
  for (auto& r : open) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto it = acc.find(r.name);
    if (it == acc.end()) {
      order.push_back(r.name);
      acc[r.name] = {ms, 1};
    } else {
      it->second.first += ms;
      it->second.second += 1;
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  open.clear();
}

TimerImpl::~TimerImpl() {
  for (auto& r : open) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
}

void KernelTimer::begin(const char* name, cudaStream_t s) {
  TimerImpl* t = (TimerImpl*)impl;
  t->pending = name;
  t->pending_ev = t->get();
  cudaEventRecord(t->pending_ev, s);
}
void KernelTimer::end(cudaStream_t s) {
  TimerImpl* t = (TimerImpl*)impl;
  cudaEvent_t b = t->get();
  cudaEventRecord(b, s);
  t->open.push_back({t->pending, t->pending_ev, b});
}

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Scratch plan of one sort / partition call.
struct Plan {
  uint64_t n = 0;
  uint32_t k1 = 0;          // level-1 buckets (0: automatic)
  int levels = 0;           // partition levels to launch
  int direct = 0;           // n small enough for one in-SM sort
  uint32_t W1 = 0, Wd = 0;  // chunk sizes (level 1, deeper levels)
  uint64_t seg_cap = 0, samp_cap = 0, hist_cap = 0, chunk_cap = 0, schunk_cap = 0;
  uint64_t bucket_cap = 0, final_cap = 0;
  uint64_t samp_cap1 = 0, hist_cap1 = 0, chunk_cap1 = 0, schunk_cap1 = 0, bucket_cap1 = 0;
  bool need_tmp = false;
  int classifier = 0;       // 0: splitter tree, 1: leading-bits table
  int wd_max_k = 0;         // levels with at most this many buckets run warp-direct
  int wide_scatter_k = 1024;  // levels with at least this many buckets use wide sub-tiles
  uint32_t target_bucket = kTargetBucket;  // automatic fan-out target
  uint32_t target_by_class[33] = {};       // per segment-size class (0: target_bucket)
  int unit_scatter = 1;     // stored bucket ids + whole-unit scatter where it fits
  int atomic_scatter = 0;   // unordered levels: atomic-ranked small-footprint scatter
  int bulk_classify = 0;    // id-storing classify staged by bulk copies
  uint64_t samp_extra = 0;  // sorted-sample slots past the sample (overpartitioning)
  uint64_t fine_cap = 0;    // fine partition counters (overpartitioning)
  // arena offsets
  size_t off_tmp_key = 0, off_tmp_idx = 0, off_samp_key = 0, off_samp_idx = 0;
  size_t off_ssamp_key = 0, off_ssamp_idx = 0, off_hist = 0, off_sums = 0, off_segs = 0;
  size_t off_list0 = 0, off_list1 = 0, off_items = 0, off_state = 0, off_fine = 0, off_bid = 0;
  size_t total = 0;
};

uint32_t ceil_log2_host(uint32_t k) {
  uint32_t l = 0;
  while ((1ull << l) < k) ++l;
  return l;
}

void layout(Plan& p) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + (bytes ? bytes : 16), 256);
    return at;
  };
  p.off_state = take(sizeof(DevState));
  p.off_items = take((size_t)kNumClasses * p.final_cap * sizeof(FinalItem));
  if (p.need_tmp) {
    p.off_tmp_key = take(p.n * 8);
    p.off_tmp_idx = take(p.n * 4);
  }
  p.off_samp_key = take(p.samp_cap * 8);
  p.off_samp_idx = take(p.samp_cap * 4);
  p.off_ssamp_key = take((p.samp_cap + p.samp_extra) * 8);
  p.off_ssamp_idx = take((p.samp_cap + p.samp_extra) * 4);
  p.off_fine = take(p.fine_cap * 4);
  p.off_bid = take((p.n + 16) * 2);
  p.off_hist = take(p.hist_cap * 4);
  p.off_sums = take((p.hist_cap / kScanTile + 2) * 4);
  p.off_segs = take(p.seg_cap * sizeof(LevelSeg));
  p.off_list0 = take(p.seg_cap * sizeof(SegIn));
  p.off_list1 = take(p.seg_cap * sizeof(SegIn));
  p.total = o;
}

// Capacities of the sample-sort levels for n elements, level-1 fan-out k1
// (0: automatic) and g1 level-1 segments.
void plan_levels(Plan& p, uint64_t n, uint32_t k1, uint64_t g1, int num_sms, int levels) {
  p.n = n;
  p.k1 = k1;
  // Levels the sizes call for (at most the max_levels tunable): the sample
  // keeps a level's largest bucket within ~1.5x its mean, so a level-1
  // bucket holds up to 1.5 n / k1 keys (an automatic fan-out aims at the
  // target, at most kMaxKDeep buckets per segment), and a level-2 bucket up
  // to 1.5x the target while level 2's fan-out stays below kMaxKDeep.  Where
  // those bounds keep the buckets within kBucketCap a further level would
  // find nothing to do (its launches cost ~0.1 ms); a bucket that still
  // exceeds kBucketCap after the last level goes to the oversize merge, so
  // the choice changes speed only.
  {
    uint64_t tmin = p.target_bucket, tmax = p.target_bucket;
    for (int c = 0; c <= 32; ++c)
      if (p.target_by_class[c]) {
        tmin = std::min<uint64_t>(tmin, p.target_by_class[c]);
        tmax = std::max<uint64_t>(tmax, p.target_by_class[c]);
      }
    const uint64_t mean1 =
        k1 >= 2 ? n / k1 : std::max<uint64_t>(n / (uint64_t)kMaxKDeep, tmax);
    int needed = 3;
    if (3 * mean1 <= 2 * (uint64_t)kBucketCap)
      needed = 1;
    else if (3 * tmax <= 2 * (uint64_t)kBucketCap &&
             3 * mean1 <= 2 * (uint64_t)kMaxKDeep * tmin)
      needed = 2;
    levels = std::min(levels, needed);
  }
  p.levels = levels;
  // level 1 of one segment: 6 chunks per SM, so grids of 1, 2, 3 or 6 resident
  // CTAs per SM all get the same number of chunks
  const uint64_t per = (n + 6ull * num_sms - 1) / (6ull * num_sms);
  p.W1 = (uint32_t)std::max<uint64_t>(kSubTile, align_up(per, kSubTile));
  if (g1 > 1) p.W1 = 65536;
  p.Wd = 65536;
  const uint64_t segs_deep = n / (kBucketCap + 1) + 1;
  p.seg_cap = std::max<uint64_t>(g1, segs_deep);
  const uint32_t kmax1 = k1 >= 2 ? k1 : kMaxKDeep;
  // automatic fan-outs aim at the smallest target any segment class uses
  uint64_t tmin = p.target_bucket;
  for (int c = 0; c <= 32; ++c)
    if (p.target_by_class[c] && p.target_by_class[c] < tmin) tmin = p.target_by_class[c];
  // level 1
  p.bucket_cap1 = k1 >= 2 ? (uint64_t)k1 * g1 : n / tmin + g1 + 1;
  p.bucket_cap1 = std::min<uint64_t>(p.bucket_cap1, (uint64_t)kmax1 * g1);
  const uint64_t a1 = k1 >= 2 ? 16ull * ceil_log2_host(k1) : (uint64_t)kDeepOversample;
  p.samp_cap1 = std::min<uint64_t>(n, a1 * p.bucket_cap1);
  p.chunk_cap1 = n / p.W1 + g1 + 1;
  // (x kPartWarps: a warp-direct level has one histogram unit per warp sub-chunk)
  p.hist_cap1 = ((uint64_t)kmax1 * (n / p.W1) + p.bucket_cap1) * kPartWarps;
  p.schunk_cap1 = p.samp_cap1 / kSampleChunk + g1 + 1;
  // deeper levels
  const uint64_t bucket_capd = n / tmin + segs_deep + 1;
  const uint64_t samp_capd = std::min<uint64_t>(n, (uint64_t)kDeepOversample * bucket_capd);
  const uint64_t chunk_capd = n / p.Wd + segs_deep + 1;
  const uint64_t hist_capd = ((uint64_t)kMaxKDeep * (n / p.Wd) + bucket_capd) * kPartWarps;
  const uint64_t schunk_capd = samp_capd / kSampleChunk + segs_deep + 1;
  const bool deep = levels > 1;
  p.bucket_cap = std::max<uint64_t>(p.bucket_cap1, deep ? bucket_capd : 0);
  p.samp_cap = std::max<uint64_t>(p.samp_cap1, deep ? samp_capd : 0);
  p.chunk_cap = std::max<uint64_t>(p.chunk_cap1, deep ? chunk_capd : 0);
  p.hist_cap = std::max<uint64_t>(p.hist_cap1, deep ? hist_capd : 0);
  p.schunk_cap = std::max<uint64_t>(p.schunk_cap1, deep ? schunk_capd : 0);
  p.final_cap = p.bucket_cap1 + (uint64_t)(levels - 1) * bucket_capd + 4;
}

LevelParams level_params(const Plan& p, int level, uint64_t seed, int kmax_level) {
  LevelParams P;
  P.level = level;
  P.W = level == 1 ? p.W1 : p.Wd;
  P.seed = seed;
  P.seg_cap = p.seg_cap;
  P.final_cap = p.final_cap;
  if (level == 1) {
    P.samp_cap = p.samp_cap1;
    P.hist_cap = p.hist_cap1;
    P.chunk_cap = p.chunk_cap1;
    P.schunk_cap = p.schunk_cap1;
    P.bucket_cap = p.bucket_cap1;
  } else {
    P.samp_cap = p.samp_cap;
    P.hist_cap = p.hist_cap;
    P.chunk_cap = p.chunk_cap;
    P.schunk_cap = p.schunk_cap;
    P.bucket_cap = p.bucket_cap;
  }
  P.level1_oversample = 1;
  P.classifier = p.classifier;
  P.warp_direct = kmax_level <= p.wd_max_k ? 1 : 0;
  P.wide_scatter_k = p.wide_scatter_k;
  P.target_bucket = p.target_bucket;
  for (int i = 0; i <= 32; ++i) P.target_by_class[i] = p.target_by_class[i];
  P.unit_scatter = p.unit_scatter;
  P.atomic_scatter = p.atomic_scatter;
  P.bulk_classify = p.bulk_classify;
  return P;
}

rsort_status latch(rsort_ctx* c, rsort_status s) {
  if (s != RSORT_OK && c->latched == RSORT_OK) c->latched = s;
  return s;
}

rsort_status cuda_status(rsort_ctx* c) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return RSORT_OK;
  if (e == cudaErrorMemoryAllocation) return latch(c, RSORT_ENOMEM);
  return latch(c, RSORT_ECUDA);
}

template <typename T>
T* at(Workspace& ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<unsigned char*>(ws.arena) + off);
}

// Kernel attributes (dynamic shared memory limits) are set once per device,
// outside any stream capture.
void set_attributes_once(int device) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lk(mu);
  for (int d : done)
    if (d == device) return;
  set_partition_kernel_attributes();
  set_local_kernel_attributes();
  set_unit_scatter_attributes();
  done.push_back(device);
}

// Enqueues the partition levels and the in-SM sort after the level-1 list and
// the directly sortable items have been initialised.
void enqueue_levels_and_local(rsort_ctx* c, Workspace& ws, const Plan& p, const LaunchEnv& e, DevState* st,
                              FinalItem* items, SegIn* const lists[2], rsort_key_type type,
                              const void* d_keys_in, const Dst& out, const Dst& tmp,
                              uint64_t seed, uint32_t k1) {
  // Level 1 scatters into the output buffer unless the input is that buffer
  // (an in-place sort): its equality buckets, final when kept in position
  // order, then need no copy.  Later levels alternate with the scratch
  // buffer.
  const int l1_out = (const void*)out.key != d_keys_in ? 1 : 0;
  auto level_dst = [&](int L) -> const Dst& { return ((L + l1_out) & 1) ? tmp : out; };
  for (int L = 1; L <= p.levels; ++L) {
    const int kmax = L == 1 ? (k1 >= 2 ? (int)k1 : kMaxKDeep) : kMaxKDeep;
    LevelParams P = level_params(p, L, seed, kmax);
    // the levels keep input order inside buckets or not as the tunables say
    // (the in-SM sort orders (key, position) pairs either way; level 1's
    // default leaves it to the device); a level's input is in position order
    // only after stable levels, and level 1's order is read on the device
    P.stable = L == 1 ? c->level1_stable : c->deep_levels_stable;
    P.in_order = L == 1 ? 1 : (L == 2 || c->deep_levels_stable ? kOrderAuto : 0);
    Src src;
    if (L == 1) {
      src = Src{(const uint64_t*)d_keys_in, nullptr, type == RSORT_KEY_F64};
    } else {
      const Dst& prev = level_dst(L - 1);
      src = Src{prev.key, prev.idx, 0};
    }
    src.bid = at<uint16_t>(ws, p.off_bid);
    const Dst& dst = level_dst(L);
    const uint16_t where = &dst == &tmp ? kWhereTmp : kWhereOut;
    launch_level(e, P, st, lists[L & 1], lists[(L + 1) & 1], at<LevelSeg>(ws, p.off_segs), src,
                 dst, where, at<uint64_t>(ws, p.off_samp_key), at<uint32_t>(ws, p.off_samp_idx),
                 at<uint64_t>(ws, p.off_ssamp_key), at<uint32_t>(ws, p.off_ssamp_idx),
                 at<uint32_t>(ws, p.off_hist), at<uint32_t>(ws, p.off_sums), items, kmax,
                 L == p.levels, 1, nullptr, p.n, 0);
  }
  launch_local_sort(e, st, items, p.final_cap, (const uint64_t*)d_keys_in, out, tmp,
                    type == RSORT_KEY_F64);
}

rsort_status set_tunable(rsort_ctx* c, const char* name, long long v) {
  if (strcmp(name, "classifier") == 0) {
    if (v != 0 && v != 1) return RSORT_EINVAL;
    c->classifier = (int)v;
    return RSORT_OK;
  }
  if (strcmp(name, "warp_direct_max_k") == 0) {
    if (v < 0 || v > kMaxK) return RSORT_EINVAL;
    c->wd_max_k = (int)v;
    return RSORT_OK;
  }
  if (strcmp(name, "wide_scatter_k") == 0) {
    if (v < 1) return RSORT_EINVAL;
    c->wide_scatter_k = (int)v;
    return RSORT_OK;
  }
  if (strcmp(name, "target_bucket") == 0) {
    if (v < 64 || v > kBucketCap) return RSORT_EINVAL;
    c->target_bucket = (uint32_t)v;
    return RSORT_OK;
  }
  if (strcmp(name, "deep_levels_stable") == 0) {
    if (v != 0 && v != 1) return RSORT_EINVAL;
    c->deep_levels_stable = (int)v;
    return RSORT_OK;
  }
  if (strcmp(name, "level1_stable") == 0) {
    if (v != 0 && v != 1 && v != kOrderAuto) return RSORT_EINVAL;
    c->level1_stable = (int)v;
    return RSORT_OK;
  }
  if (strcmp(name, "max_levels") == 0) {
    if (v < 1 || v > kMaxLevels) return RSORT_EINVAL;
    c->max_levels = (int)v;
    return RSORT_OK;
  }
  if (strcmp(name, "medium_sort") == 0) {
    if (v != 0 && v != 1) return RSORT_EINVAL;
    c->local.algo[1] = c->local.algo[2] = v ? kLocalQuick : kLocalBins;
    return RSORT_OK;
  }
  if (strcmp(name, "sort_small") == 0) {
    if (v != kLocalBins && v != kLocalBitonic) return RSORT_EINVAL;
    c->local.algo[0] = (uint8_t)v;
    return RSORT_OK;
  }
  if (strcmp(name, "sort_mid") == 0 || strcmp(name, "sort_medium") == 0) {
    if (v != kLocalBins && v != kLocalQuick && v != kLocalBitonic) return RSORT_EINVAL;
    c->local.algo[strcmp(name, "sort_mid") == 0 ? 1 : 2] = (uint8_t)v;
    return RSORT_OK;
  }
  if (strcmp(name, "small_cap") == 0) {
    if (v < 64 || v > (long long)kSmallCap) return RSORT_EINVAL;
    c->local.small_cap = (uint32_t)v;
    return RSORT_OK;
  }
  if (strcmp(name, "mid_cap") == 0) {
    if (v < 64 || v > (long long)kMidCap) return RSORT_EINVAL;
    c->local.mid_cap = (uint32_t)v;
    return RSORT_OK;
  }
  if (strcmp(name, "rank_max") == 0) {
    if (v < 0 || v > 128) return RSORT_EINVAL;
    c->local.rank_max = (uint32_t)v;
    return RSORT_OK;
  }
  if (strncmp(name, "target_bucket@", 14) == 0) {
    char* end = nullptr;
    const long cls = strtol(name + 14, &end, 10);
    if (end == name + 14 || *end != '\0' || cls < 1 || cls > 32) return RSORT_EINVAL;
    if (v != 0 && (v < 64 || v > kBucketCap)) return RSORT_EINVAL;
    c->target_by_class[cls] = (uint32_t)v;
    return RSORT_OK;
  }
  if (strcmp(name, "unit_scatter") == 0) {
    if (v != 0 && v != 1) return RSORT_EINVAL;
    c->unit_scatter = (int)v;
    return RSORT_OK;
  }
  if (strcmp(name, "atomic_scatter") == 0) {
    if (v != 0 && v != 1) return RSORT_EINVAL;
    c->atomic_scatter = (int)v;
    return RSORT_OK;
  }
  if (strcmp(name, "bulk_classify") == 0) {
    if (v != 0 && v != 1) return RSORT_EINVAL;
    c->bulk_classify = (int)v;
    return RSORT_OK;
  }
  if (c->server) return RSORT_EINVAL;  // serving tunables are fixed once it runs
  if (strcmp(name, "serve_slots") == 0) {
    if (v < 1 || v > 8) return RSORT_EINVAL;
    c->serve_slots = (int)v;
    return RSORT_OK;
  }
  if (strcmp(name, "serve_batch_keys") == 0) {
    if (v < 1 || v > (1ll << 30)) return RSORT_EINVAL;
    c->serve_batch_keys = (uint64_t)v;
    return RSORT_OK;
  }
  if (strcmp(name, "serve_alone_min") == 0) {
    if (v < 0 || v > 0xFFFFFFFFll) return RSORT_EINVAL;
    c->serve_alone_min = (uint64_t)v;
    return RSORT_OK;
  }
  if (strcmp(name, "serve_history") == 0) {
    if (v < 1 || v > (1ll << 26)) return RSORT_EINVAL;
    c->serve_history = (uint64_t)v;
    return RSORT_OK;
  }
  return RSORT_EINVAL;
}

}  // namespace

// ---------------------------------------------------------------------------
// Engine (engine.h): workspaces and whole-sort enqueue functions
// ---------------------------------------------------------------------------
LaunchEnv env_of(rsort_ctx* c, cudaStream_t s) {
  LaunchEnv e;
  e.stream = s;
  e.num_sms = c->num_sms;
  e.timer = c->profiling ? &c->timer : nullptr;
  e.launches = &c->launches;
  e.local = c->local;
  // a mid class below the small one is empty
  if (e.local.mid_cap < e.local.small_cap) e.local.mid_cap = e.local.small_cap;
  return e;
}


rsort_status ensure_workspace(rsort_ctx* c, Workspace& ws, size_t bytes, cudaStream_t s) {
  if (bytes <= ws.bytes) return RSORT_OK;
  std::lock_guard<std::mutex> lk(c->alloc_mu);
  const uint64_t others = c->held.load() - ws.bytes;
  if (c->budget && others + bytes > c->budget) return RSORT_ENOMEM;
  if (ws.arena) {
    cudaFreeAsync(ws.arena, s);
    c->held -= ws.bytes;
    ws.arena = nullptr;
    ws.bytes = 0;
  }
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return RSORT_ENOMEM;
  }
  ws.arena = p;
  ws.bytes = bytes;
  c->held += bytes;
  return RSORT_OK;
}

void release_workspace(rsort_ctx* c, Workspace& ws, cudaStream_t s) {
  if (!ws.arena) return;
  std::lock_guard<std::mutex> lk(c->alloc_mu);
  if (s) cudaFreeAsync(ws.arena, s);
  else cudaFree(ws.arena);
  c->held -= ws.bytes;
  ws.arena = nullptr;
  ws.bytes = 0;
}

namespace {

Plan plan_sort(rsort_ctx* c, uint64_t n, uint32_t p_virtual) {
  Plan p;
  p.classifier = c->classifier;
  p.wd_max_k = c->wd_max_k;
  p.wide_scatter_k = c->wide_scatter_k;
  p.target_bucket = c->target_bucket;
  for (int i = 0; i <= 32; ++i) p.target_by_class[i] = c->target_by_class[i];
  p.unit_scatter = c->unit_scatter;
  p.atomic_scatter = c->atomic_scatter;
  p.bulk_classify = c->bulk_classify;
  const uint32_t k1 = p_virtual >= 2 ? p_virtual : 0;
  if (n <= (uint64_t)kBucketCap) {
    p.n = n;
    p.direct = 1;
    p.final_cap = 4;
    p.seg_cap = 1;
    p.need_tmp = false;
    p.levels = 0;
  } else {
    plan_levels(p, n, k1, 1, c->num_sms, c->max_levels);
    p.need_tmp = true;
  }
  layout(p);
  return p;
}

Plan plan_segmented(rsort_ctx* c, uint64_t n, uint32_t num_segments) {
  Plan p;
  p.classifier = c->classifier;
  p.wd_max_k = c->wd_max_k;
  p.wide_scatter_k = c->wide_scatter_k;
  p.target_bucket = c->target_bucket;
  for (int i = 0; i <= 32; ++i) p.target_by_class[i] = c->target_by_class[i];
  p.unit_scatter = c->unit_scatter;
  p.atomic_scatter = c->atomic_scatter;
  p.bulk_classify = c->bulk_classify;
  const uint64_t g1 = std::min<uint64_t>(num_segments, n / (kBucketCap + 1) + 1);
  plan_levels(p, n, 0, std::max<uint64_t>(g1, 2), c->num_sms, c->max_levels);
  p.final_cap += num_segments;
  p.need_tmp = true;
  layout(p);
  return p;
}

}  // namespace

size_t sort_scratch_bytes(rsort_ctx* c, uint64_t n, uint32_t p_virtual) {
  return n == 0 ? 0 : plan_sort(c, n, p_virtual).total;
}

size_t segmented_scratch_bytes(rsort_ctx* c, uint64_t n, uint32_t num_segments) {
  return (n == 0 || num_segments == 0) ? 0 : plan_segmented(c, n, num_segments).total;
}

rsort_status enqueue_sort(rsort_ctx* c, Workspace& ws, const LaunchEnv& e, rsort_key_type type,
                          const void* d_keys_in, void* d_keys_out, uint32_t* d_perm_out,
                          uint64_t n, uint32_t p_virtual, uint64_t seed, DevState** st_out) {
  Plan p = plan_sort(c, n, p_virtual);
  const uint32_t k1 = p_virtual >= 2 ? p_virtual : 0;
  rsort_status rs = ensure_workspace(c, ws, p.total, e.stream);
  if (rs != RSORT_OK) return rs;
  DevState* st = at<DevState>(ws, p.off_state);
  FinalItem* items = at<FinalItem>(ws, p.off_items);
  SegIn* lists[2] = {at<SegIn>(ws, p.off_list0), at<SegIn>(ws, p.off_list1)};
  launch_init_plain(e, st, lists[1], items, n, k1, p.direct, p.final_cap);
  Dst out{(uint64_t*)d_keys_out, d_perm_out};
  Dst tmp{at<uint64_t>(ws, p.off_tmp_key), at<uint32_t>(ws, p.off_tmp_idx)};
  enqueue_levels_and_local(c, ws, p, e, st, items, lists, type, d_keys_in, out, tmp, seed, k1);
  if (st_out) *st_out = st;
  return RSORT_OK;
}

rsort_status enqueue_segmented(rsort_ctx* c, Workspace& ws, const LaunchEnv& e,
                               rsort_key_type type, const void* d_keys_in, void* d_keys_out,
                               uint32_t* d_perm_out, uint64_t n, const uint64_t* d_offsets,
                               uint32_t num_segments, uint64_t seed, DevState** st_out) {
  Plan p = plan_segmented(c, n, num_segments);
  rsort_status rs = ensure_workspace(c, ws, p.total, e.stream);
  if (rs != RSORT_OK) return rs;
  DevState* st = at<DevState>(ws, p.off_state);
  FinalItem* items = at<FinalItem>(ws, p.off_items);
  SegIn* lists[2] = {at<SegIn>(ws, p.off_list0), at<SegIn>(ws, p.off_list1)};
  launch_init_plain(e, st, lists[1], items, 0, 0, 0, p.final_cap);  // reset the control block
  launch_init_segments(e, st, d_offsets, num_segments, n, lists[1], items, p.seg_cap,
                       p.final_cap);
  Dst out{(uint64_t*)d_keys_out, d_perm_out};
  Dst tmp{at<uint64_t>(ws, p.off_tmp_key), at<uint32_t>(ws, p.off_tmp_idx)};
  enqueue_levels_and_local(c, ws, p, e, st, items, lists, type, d_keys_in, out, tmp, seed, 0);
  if (st_out) *st_out = st;
  return RSORT_OK;
}

}  // namespace rsort

using namespace rsort;

extern "C" {

const char* rsort_strerror(rsort_status s) {
  switch (s) {
    case RSORT_OK: return "ok";
    case RSORT_PENDING: return "pending";
    case RSORT_EINVAL: return "invalid argument";
    case RSORT_ENOMEM: return "out of memory (scratch exceeds budget or device memory)";
    case RSORT_ECUDA: return "CUDA error";
    case RSORT_ETIMEOUT: return "timed out";
    case RSORT_ECANCELLED: return "cancelled";
    case RSORT_EUNSUPPORTED: return "unsupported";
    case RSORT_EDEVICE: return "device-side error (capacity check failed)";
    default: return "unknown status";
  }
}

rsort_status rsort_create(rsort_ctx** out, int device, uint64_t hbm_budget_bytes,
                          const char* tune_table_path) {
  if (!out) return RSORT_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return RSORT_EINVAL;
  }
  rsort_ctx* c = new (std::nothrow) rsort_ctx();
  if (!c) return RSORT_ENOMEM;
  if (tune_table_path) {
    // "name value" lines; '#' starts a comment
    FILE* f = fopen(tune_table_path, "r");
    if (!f) {
      delete c;
      return RSORT_EINVAL;
    }
    char line[256];
    while (fgets(line, sizeof line, f)) {
      char name[128];
      long long v;
      if (line[0] == '#') continue;
      if (sscanf(line, "%127s %lld", name, &v) == 2 && set_tunable(c, name, v) != RSORT_OK) {
        fclose(f);
        delete c;
        return RSORT_EINVAL;
      }
    }
    fclose(f);
  }
  c->device = device;
  c->budget = hbm_budget_bytes;
  DeviceGuard g(device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  set_attributes_once(device);
  if (cudaMallocHost(&c->h_state, sizeof(DevState)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return RSORT_ECUDA;
  }
  c->timer.impl = &c->timer_impl;
  *out = c;
  return RSORT_OK;
}

rsort_status rsort_destroy(rsort_ctx* c) {
  if (!c) return RSORT_OK;
  {
    DeviceGuard g(c->device);
    destroy_server(c);
    cudaDeviceSynchronize();
    release_workspace(c, c->ws, nullptr);
    if (c->h_state) cudaFreeHost(c->h_state);
    cudaGetLastError();
  }
  delete c;
  return RSORT_OK;
}

rsort_status rsort_check(rsort_ctx* c) {
  if (!c) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) latch(c, RSORT_ECUDA);
  cuda_status(c);
  if (c->ws.arena) {
    DevState st;
    if (cudaMemcpy(&st, c->ws.arena, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess) {
      latch(c, RSORT_ECUDA);
    } else if (st.error) {
      latch(c, RSORT_EDEVICE);
      // the error is reported once: clear the device word
      cudaMemset(static_cast<unsigned char*>(c->ws.arena) + offsetof(DevState, error), 0,
                 sizeof(uint32_t));
    }
  }
  rsort_status s = c->latched;
  c->latched = RSORT_OK;
  return s;
}

namespace {

rsort_status partition_impl(rsort_ctx* c, rsort_key_type type, const void* d_keys_in,
                            uint64_t n, uint32_t k, uint64_t seed, uint32_t tie_break,
                            uint32_t over, void* d_keys_out, uint32_t* d_pos_out,
                            uint64_t* d_offsets_out, uint64_t* d_fine_out,
                            uint32_t* d_first_out, void* stream) {
  if (!c || (type != RSORT_KEY_U64 && type != RSORT_KEY_F64)) return RSORT_EINVAL;
  if (k < 1 || k > (uint32_t)kMaxK || n > 0xFFFFFFFFull) return RSORT_EINVAL;
  if (tie_break > 1 || over < 1 || (over > 1 && (uint64_t)k * over > (uint64_t)kMaxFine))
    return RSORT_EINVAL;
  if (!d_offsets_out || (n > 0 && (!d_keys_in || !d_keys_out || !d_pos_out)))
    return RSORT_EINVAL;
  if (n > 0 && d_keys_in == d_keys_out) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->latched != RSORT_OK) {
    rsort_status s = c->latched;
    c->latched = RSORT_OK;
    return s;
  }
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  LaunchEnv e = env_of(c, s);
  const uint32_t K = k * over;
  if (n == 0) {
    // every partition is empty; fine partition g is output g, or all fine
    // partitions sit in output 0 when overpartitioned
    cudaMemsetAsync(d_offsets_out, 0, (size_t)(k + 1) * 8, s);
    if (d_fine_out) cudaMemsetAsync(d_fine_out, 0, (size_t)K * 8, s);
    if (d_first_out) {
      if (over == 1) {
        launch_plain_groups(e, d_offsets_out, k, nullptr, d_first_out);
      } else {
        std::vector<uint32_t> h(k + 1, K);
        h[0] = 0;
        cudaMemcpyAsync(d_first_out, h.data(), h.size() * 4, cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
      }
    }
    return cuda_status(c);
  }
  Plan p;
  p.classifier = c->classifier;
  p.wd_max_k = c->wd_max_k;
  p.wide_scatter_k = c->wide_scatter_k;
  p.target_bucket = c->target_bucket;
  for (int i = 0; i <= 32; ++i) p.target_by_class[i] = c->target_by_class[i];
  p.unit_scatter = c->unit_scatter;
  p.atomic_scatter = c->atomic_scatter;
  p.bulk_classify = c->bulk_classify;
  const uint32_t kk = k < 2 ? 2 : k;  // capacities as for two buckets when k = 1
  plan_levels(p, n, kk, 1, c->num_sms, 1);
  p.final_cap = 4;
  p.need_tmp = false;
  if (over > 1) {
    p.samp_extra = (uint64_t)kk + 2;
    p.fine_cap = 2 * (uint64_t)K + 8;  // counters, prefix sums, search state
  }
  layout(p);
  Workspace& ws = c->ws;
  rsort_status rs = ensure_workspace(c, ws, p.total, s);
  if (rs != RSORT_OK) return latch(c, rs);
  DevState* st = at<DevState>(ws, p.off_state);
  SegIn* list1 = at<SegIn>(ws, p.off_list1);
  launch_init_plain(e, st, list1, at<FinalItem>(ws, p.off_items), n, k, 0, p.final_cap);
  LevelParams P = level_params(p, 1, seed, (int)kk);
  P.no_tie_break = tie_break ? 0 : 1;
  Src src{(const uint64_t*)d_keys_in, nullptr, type == RSORT_KEY_F64};
  src.bid = at<uint16_t>(ws, p.off_bid);
  Dst dst{(uint64_t*)d_keys_out, d_pos_out};
  uint32_t* fine = at<uint32_t>(ws, p.off_fine);
  Overpart op{k,
              over,
              fine,
              fine + K,
              reinterpret_cast<uint64_t*>(fine + 2 * (uint64_t)K + 2),
              d_fine_out,
              d_first_out};
  launch_level(e, P, st, list1, at<SegIn>(ws, p.off_list0), at<LevelSeg>(ws, p.off_segs), src,
               dst, kWhereOut, at<uint64_t>(ws, p.off_samp_key), at<uint32_t>(ws, p.off_samp_idx),
               at<uint64_t>(ws, p.off_ssamp_key), at<uint32_t>(ws, p.off_ssamp_idx),
               at<uint32_t>(ws, p.off_hist), at<uint32_t>(ws, p.off_sums),
               at<FinalItem>(ws, p.off_items), (int)kk, 1, 0, d_offsets_out, n,
               type == RSORT_KEY_F64, over > 1 ? &op : nullptr);
  if (over == 1 && (d_fine_out || d_first_out))
    launch_plain_groups(e, d_offsets_out, k, d_fine_out, d_first_out);
  return cuda_status(c);
}

}  // namespace

rsort_status rsort_partition(rsort_ctx* c, rsort_key_type type, const void* d_keys_in,
                             uint64_t n, uint32_t k, uint64_t seed, void* d_keys_out,
                             uint32_t* d_pos_out, uint64_t* d_offsets_out, void* stream) {
  return partition_impl(c, type, d_keys_in, n, k, seed, 1, 1, d_keys_out, d_pos_out,
                        d_offsets_out, nullptr, nullptr, stream);
}

rsort_status rsort_partition_ex(rsort_ctx* c, rsort_key_type type, const void* d_keys_in,
                                uint64_t n, uint32_t k, uint64_t seed,
                                const rsort_partition_opts* opts, void* d_keys_out,
                                uint32_t* d_pos_out, uint64_t* d_offsets_out,
                                uint64_t* d_fine_sizes_out, uint32_t* d_group_first_out,
                                void* stream) {
  const uint32_t tb = opts ? opts->tie_break : 1u;
  const uint32_t over = opts ? opts->overpartition : 1u;
  return partition_impl(c, type, d_keys_in, n, k, seed, tb, over, d_keys_out, d_pos_out,
                        d_offsets_out, d_fine_sizes_out, d_group_first_out, stream);
}

rsort_status rsort_approx_median(rsort_ctx* c, rsort_key_type type, const void* d_keys,
                                 uint64_t n, uint32_t k, uint64_t seed, uint64_t* d_pos_out,
                                 void* stream) {
  if (!c || (type != RSORT_KEY_U64 && type != RSORT_KEY_F64)) return RSORT_EINVAL;
  if (n < 1 || n > (1ull << 24) || !d_keys || !d_pos_out) return RSORT_EINVAL;
  if (k != 2 && k != 4 && k != 8 && k != 16 && k != 32) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->latched != RSORT_OK) {
    rsort_status s = c->latched;
    c->latched = RSORT_OK;
    return s;
  }
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  LaunchEnv e = env_of(c, s);
  rsort_status rs = ensure_workspace(c, c->ws, tree_median_scratch_bytes(n), s);
  if (rs != RSORT_OK) return latch(c, rs);
  if (!launch_tree_median(e, (const uint64_t*)d_keys, (uint32_t)n, type == RSORT_KEY_F64, k,
                          seed, c->ws.arena, d_pos_out))
    return RSORT_EINVAL;
  return cuda_status(c);
}

rsort_status rsort_sort(rsort_ctx* c, rsort_key_type type, const void* d_keys_in,
                        void* d_keys_out, uint32_t* d_perm_out, uint64_t n, uint32_t p_virtual,
                        uint64_t seed, void* stream, rsort_stats* opt_stats) {
  if (!c || (type != RSORT_KEY_U64 && type != RSORT_KEY_F64)) return RSORT_EINVAL;
  if (n > 0xFFFFFFFFull || p_virtual < 1 || p_virtual > (uint32_t)kMaxK) return RSORT_EINVAL;
  if (n > 0 && (!d_keys_in || !d_keys_out || !d_perm_out)) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->latched != RSORT_OK) {
    rsort_status s = c->latched;
    c->latched = RSORT_OK;
    return s;
  }
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  if (opt_stats) memset(opt_stats, 0, sizeof(*opt_stats));
  if (n == 0) return RSORT_OK;
  LaunchEnv e = env_of(c, s);
  const int direct = n <= (uint64_t)kBucketCap;
  const uint32_t k1 = p_virtual >= 2 ? p_virtual : 0;
  DevState* st = nullptr;
  rsort_status rs = enqueue_sort(c, c->ws, e, type, d_keys_in, d_keys_out, d_perm_out, n,
                                 p_virtual, seed, &st);
  if (rs != RSORT_OK) return latch(c, rs);
  rs = cuda_status(c);
  if (rs != RSORT_OK) return rs;
  if (opt_stats) {
    if (cudaMemcpyAsync(c->h_state, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return latch(c, RSORT_ECUDA);
    const DevState& h = *c->h_state;
    opt_stats->n = n;
    opt_stats->p = direct ? 1 : (k1 >= 2 ? k1 : 0);
    opt_stats->levels = h.levels_used;
    opt_stats->path = direct ? 0 : 1;
    opt_stats->max_bucket = direct ? (uint32_t)n : h.max_bucket_l1;
    const double mean = opt_stats->p ? (double)n / opt_stats->p : (double)n;
    opt_stats->max_over_mean = mean > 0 ? opt_stats->max_bucket / mean : 0.0;
    opt_stats->final_buckets = 0;
    for (int i = 0; i < kNumClasses; ++i) opt_stats->final_buckets += h.nfinal_c[i];
    // per key: level 1's classify reads 8 B and writes a 2-byte bucket id,
    // its scatter reads 8 + 2 and writes 12; a deeper level reads 8 and
    // writes 2, then reads 12 + 2 and writes 12; the in-SM sort reads and
    // writes 12 B/key.
    uint64_t bytes = 24ull * n;
    for (int i = 0; i < 4; ++i) {
      opt_stats->level_elems[i] = h.level_elems[i];
      bytes += (i == 0 ? 32ull : 36ull) * h.level_elems[i];
    }
    opt_stats->bytes_moved = bytes;
    static_assert(kNumClasses == 5, "rsort_stats.class_elems has one entry per size class");
    for (int i = 0; i < kNumClasses; ++i) opt_stats->class_elems[i] = h.class_elems[i];
    static_assert(kNumAlgos == 6, "rsort_stats.algo_elems has one entry per in-SM algorithm");
    for (int i = 0; i < kNumAlgos; ++i) opt_stats->algo_elems[i] = h.algo_elems[i];
    if (h.error) return latch(c, RSORT_EDEVICE);
  }
  return RSORT_OK;
}

rsort_status rsort_segmented(rsort_ctx* c, rsort_key_type type, const void* d_keys_in,
                             void* d_keys_out, uint32_t* d_perm_out, uint64_t n,
                             const uint64_t* d_offsets, uint32_t num_segments, uint64_t seed,
                             void* stream) {
  if (!c || (type != RSORT_KEY_U64 && type != RSORT_KEY_F64)) return RSORT_EINVAL;
  if (n > 0xFFFFFFFFull) return RSORT_EINVAL;
  if (num_segments > 0 && !d_offsets) return RSORT_EINVAL;
  if (n > 0 && (!d_keys_in || !d_keys_out || !d_perm_out)) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->latched != RSORT_OK) {
    rsort_status s = c->latched;
    c->latched = RSORT_OK;
    return s;
  }
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  if (n == 0 || num_segments == 0) return RSORT_OK;
  LaunchEnv e = env_of(c, s);
  rsort_status rs = enqueue_segmented(c, c->ws, e, type, d_keys_in, d_keys_out, d_perm_out, n,
                                      d_offsets, num_segments, seed, nullptr);
  if (rs != RSORT_OK) return latch(c, rs);
  return cuda_status(c);
}

rsort_status rsort_set_profiling(rsort_ctx* c, int enable) {
  if (!c) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  c->profiling = enable != 0;
  return RSORT_OK;
}

rsort_status rsort_phase_times(rsort_ctx* c, const char** names, double* ms, uint64_t* launches,
                               int max, int* count) {
  if (!c || !count) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  c->timer_impl.resolve();
  int i = 0;
  for (const std::string& nm : c->timer_impl.order) {
    if (i < max) {
      auto& a = c->timer_impl.acc[nm];
      // names point at the static literals used at launch time
      static std::mutex name_mu;
      static std::unordered_map<std::string, std::string> interned;
      std::lock_guard<std::mutex> lk2(name_mu);
      auto it = interned.emplace(nm, nm).first;
      if (names) names[i] = it->second.c_str();
      if (ms) ms[i] = a.first;
      if (launches) launches[i] = a.second;
    }
    ++i;
  }
  *count = i;
  c->timer_impl.acc.clear();
  c->timer_impl.order.clear();
  return cuda_status(c);
}

rsort_status rsort_set_tunable(rsort_ctx* c, const char* name, int64_t value) {
  if (!c || !name) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  return set_tunable(c, name, value);
}

rsort_status rsort_get_tunable(rsort_ctx* c, const char* name, int64_t* value) {
  if (!c || !name || !value) return RSORT_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  if (strcmp(name, "classifier") == 0) {
    *value = c->classifier;
    return RSORT_OK;
  }
  if (strcmp(name, "warp_direct_max_k") == 0) {
    *value = c->wd_max_k;
    return RSORT_OK;
  }
  if (strcmp(name, "serve_slots") == 0) {
    *value = c->serve_slots;
    return RSORT_OK;
  }
  if (strcmp(name, "wide_scatter_k") == 0) {
    *value = c->wide_scatter_k;
    return RSORT_OK;
  }
  if (strcmp(name, "target_bucket") == 0) {
    *value = c->target_bucket;
    return RSORT_OK;
  }
  if (strcmp(name, "deep_levels_stable") == 0) {
    *value = c->deep_levels_stable;
    return RSORT_OK;
  }
  if (strcmp(name, "level1_stable") == 0) {
    *value = c->level1_stable;
    return RSORT_OK;
  }
  if (strcmp(name, "max_levels") == 0) {
    *value = c->max_levels;
    return RSORT_OK;
  }
  if (strcmp(name, "medium_sort") == 0) {
    *value = (c->local.algo[1] == kLocalQuick && c->local.algo[2] == kLocalQuick) ? 1 : 0;
    return RSORT_OK;
  }
  if (strcmp(name, "sort_small") == 0) {
    *value = c->local.algo[0];
    return RSORT_OK;
  }
  if (strcmp(name, "sort_mid") == 0) {
    *value = c->local.algo[1];
    return RSORT_OK;
  }
  if (strcmp(name, "sort_medium") == 0) {
    *value = c->local.algo[2];
    return RSORT_OK;
  }
  if (strcmp(name, "small_cap") == 0) {
    *value = c->local.small_cap;
    return RSORT_OK;
  }
  if (strcmp(name, "mid_cap") == 0) {
    *value = c->local.mid_cap;
    return RSORT_OK;
  }
  if (strcmp(name, "rank_max") == 0) {
    *value = c->local.rank_max;
    return RSORT_OK;
  }
  if (strncmp(name, "target_bucket@", 14) == 0) {
    char* end = nullptr;
    const long cls = strtol(name + 14, &end, 10);
    if (end == name + 14 || *end != '\0' || cls < 1 || cls > 32) return RSORT_EINVAL;
    *value = c->target_by_class[cls];
    return RSORT_OK;
  }
  if (strcmp(name, "unit_scatter") == 0) {
    *value = c->unit_scatter;
    return RSORT_OK;
  }
  if (strcmp(name, "atomic_scatter") == 0) {
    *value = c->atomic_scatter;
    return RSORT_OK;
  }
  if (strcmp(name, "bulk_classify") == 0) {
    *value = c->bulk_classify;
    return RSORT_OK;
  }
  if (strcmp(name, "serve_batch_keys") == 0) {
    *value = (int64_t)c->serve_batch_keys;
    return RSORT_OK;
  }
  if (strcmp(name, "serve_alone_min") == 0) {
    *value = (int64_t)c->serve_alone_min;
    return RSORT_OK;
  }
  if (strcmp(name, "serve_history") == 0) {
    *value = (int64_t)c->serve_history;
    return RSORT_OK;
  }
  return RSORT_EINVAL;
}

rsort_status rsort_launch_count(rsort_ctx* c, uint64_t* out) {
  if (!c || !out) return RSORT_EINVAL;
  *out = c->launches;
  return RSORT_OK;
}

}  // extern "C"
