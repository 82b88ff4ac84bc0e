// engine.h -- host-side internals shared by the C ABI (rsort_api.cu) and the
// serving runtime (serve.cu): the context, scratch workspaces, and functions
// that enqueue a whole sort on a given workspace and stream.
#pragma once

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "rsort_internal.cuh"

namespace rsort {

// CUDA events around every launch, resolved lazily (tracing).
struct TimerImpl {
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> open;
  std::vector<cudaEvent_t> pool;
  std::unordered_map<std::string, std::pair<double, uint64_t>> acc;
  std::vector<std::string> order;
  const char* pending = nullptr;
  cudaEvent_t pending_ev = nullptr;

  cudaEvent_t get();
  void resolve();
  ~TimerImpl();
};

// One scratch arena (device memory owned by the context).
struct Workspace {
  void* arena = nullptr;
  size_t bytes = 0;
};

struct Server;  // serve.cu

}  // namespace rsort

struct rsort_ctx {
  int device = 0;
  int num_sms = 0;
  uint64_t budget = 0;                  // 0: no cap
  std::atomic<uint64_t> held{0};        // bytes held by all workspaces
  rsort::Workspace ws;                  // workspace of the synchronous entry points
  cudaStream_t last_stream = nullptr;
  rsort_status latched = RSORT_OK;
  rsort::DevState* h_state = nullptr;   // pinned read-back buffer
  uint64_t launches = 0;
  bool profiling = false;
  // tunable "classifier": 0 splitter tree, 1 leading-bits table (default: the
  // table; both give the same buckets and the table measured faster on GB300)
  int classifier = 1;
  // tunable "warp_direct_max_k": warp-direct kernels up to this k (default off:
  // direct scattered stores measured ~3x slower than shared-memory combining)
  int wd_max_k = 0;
  // tunable "wide_scatter_k": levels with at least this many buckets stage
  // 4096-key sub-tiles with 512 threads (longer runs per bucket)
  int wide_scatter_k = 1024;
  // tunable "target_bucket": automatic fan-outs aim at final buckets of this
  // many keys (mostly inside the 1025..2048-key in-SM size class)
  uint32_t target_bucket = rsort::kTargetBucket;
  // in-SM size classes and algorithms (tunables "small_cap", "mid_cap",
  // "rank_max", "sort_small", "sort_mid", "sort_medium"; "medium_sort" sets
  // the mid and medium classes to quicksort (1) or bins (0) at once)
  rsort::LocalPlan local;
  // tunable "target_bucket@c": fan-out target for segments of ceil(log2 m) = c
  // (0: target_bucket)
  uint32_t target_by_class[33] = {};
  // tunable "max_levels": partition levels before every bucket is final
  // (1..3, default 3); buckets still above one SM's capacity after the last
  // level are merge-sorted through global memory by one CTA each
  int max_levels = rsort::kMaxLevels;
  // tunable "deep_levels_stable": the sort's levels after the first keep
  // input order inside buckets (1) or rank by shared-memory atomics (0,
  // default); level 1, the partition step, always keeps it
  int deep_levels_stable = 0;
  // tunable "level1_stable": level 1 of rsort_sort / rsort_segmented keeps
  // input order inside buckets (1), ranks by shared-memory atomics (0), or
  // keeps it only when at least 1/16 of its buckets are equality buckets,
  // decided on the device (2, default); rsort_partition always keeps it
  int level1_stable = 2;
  // tunable "unit_scatter": stable levels with at most rsort::kUnitMaxK
  // buckets store every element's bucket id in the classify pass and scatter
  // in whole 8-element units (1, default), or classify again in the staged
  // scatter (0)
  int unit_scatter = 1;
  // tunable "atomic_scatter": unordered levels (a full sort's levels after the
  // first) scatter with the small-footprint kernel ranked by shared-memory
  // atomics (1) or the staged scatter (0, default)
  int atomic_scatter = 0;
  // tunable "bulk_classify": the id-storing classify stages its keys through
  // bulk copies into a shared-memory ring (1) or loads them into registers
  // (0, default: measured faster, 0.97 vs 1.12 ms at 2^28 keys)
  int bulk_classify = 0;
  rsort::KernelTimer timer;
  rsort::TimerImpl timer_impl;
  std::mutex mu;
  rsort::Server* server = nullptr;
  std::mutex server_mu;
  std::mutex alloc_mu;                    // serialises workspace growth (budget check)
  // serving tunables (read when the runtime starts, at the first submit)
  int serve_slots = 4;                    // batches in flight (streams)
  uint64_t serve_batch_keys = 1ull << 24; // keys per batch
  uint64_t serve_alone_min = 1ull << 20;  // larger requests run as a batch of their own
  uint64_t serve_history = 1ull << 20;    // finished requests whose status (and latency) is kept
};

namespace rsort {

// Grows ws to at least `bytes` (stream-ordered), within the context budget.
rsort_status ensure_workspace(rsort_ctx* c, Workspace& ws, size_t bytes, cudaStream_t s);
void release_workspace(rsort_ctx* c, Workspace& ws, cudaStream_t s);

// Scratch bytes a plain sort / a segmented sort of n keys needs.
size_t sort_scratch_bytes(rsort_ctx* c, uint64_t n, uint32_t p_virtual);
size_t segmented_scratch_bytes(rsort_ctx* c, uint64_t n, uint32_t num_segments);

// Enqueue a whole sort on `ws` and stream e.stream (arguments already
// validated).  *st_out receives the device control block of the call.
rsort_status enqueue_sort(rsort_ctx* c, Workspace& ws, const LaunchEnv& e, rsort_key_type type,
                          const void* d_keys_in, void* d_keys_out, uint32_t* d_perm_out,
                          uint64_t n, uint32_t p_virtual, uint64_t seed, DevState** st_out);
rsort_status enqueue_segmented(rsort_ctx* c, Workspace& ws, const LaunchEnv& e,
                               rsort_key_type type, const void* d_keys_in, void* d_keys_out,
                               uint32_t* d_perm_out, uint64_t n, const uint64_t* d_offsets,
                               uint32_t num_segments, uint64_t seed, DevState** st_out);

LaunchEnv env_of(rsort_ctx* c, cudaStream_t s);
void destroy_server(rsort_ctx* c);

}  // namespace rsort
