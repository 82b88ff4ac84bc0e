// noalloc.cu -- rsort_partition_noalloc: the robust partition step with its
// scratch in a fixed, statically allocated device array instead of memory the
// library allocates.
//
// Why it exists: some callers cannot allocate device memory at the time they
// need to partition -- callers whose device memory is owned by another
// allocator that must see every allocation, and real-time loops that forbid
// any allocation after start-up because an allocation can block.  They still
// pass their own inputs and outputs; only the scratch (samples, histograms,
// the control block) comes from here.
//
// The host plan below sizes every region for the largest plan k_level_plan
// computes from (n, k): the same sample count, chunk count, histogram and
// bucket count, so the device-side capacity checks never fire.  Nothing is
// read back from the device, so a device flag would go unreported.
//
// The scratch is one file-scope __device__ array of kNoAllocBytes (8 MiB).
// Every GPU that loads librsort holds it until the process exits.  In host
// code its name is only a host-side stand-in, not a device address, so the
// address is obtained once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels.
#include <mutex>
#include <vector>

#include "rsort_internal.cuh"

namespace rsort {
namespace {

constexpr size_t kNoAllocBytes = 8u << 20;      // 8 MiB
constexpr uint32_t kNoAllocMaxK = 1024;          // buckets per call
constexpr uint64_t kNoAllocMaxChunks = 512;      // chunks of the classify/scatter grid

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct DevScratch {
  int device;
  unsigned char* ptr;
};

// Device address of g_noalloc_scratch on the current device (set up on the
// first call on that device; the same call sets the kernels' shared-memory
// limits).  Returns nullptr if CUDA refuses.
unsigned char* scratch_for_current_device(int device) {
  static std::mutex mu;
  static std::vector<DevScratch> table;
  std::lock_guard<std::mutex> lk(mu);
  for (const DevScratch& d : table)
    if (d.device == device) return d.ptr;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return nullptr;
  }
  set_partition_kernel_attributes();
  table.push_back({device, static_cast<unsigned char*>(p)});
  return static_cast<unsigned char*>(p);
}

inline uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

uint32_t ceil_log2(uint32_t k) {
  uint32_t l = 0;
  while ((1ull << l) < k) ++l;
  return l;
}

}  // namespace
}  // namespace rsort

using namespace rsort;

extern "C" rsort_status rsort_partition_noalloc(rsort_key_type type, const void* d_keys_in,
                                                uint64_t n, uint32_t k, uint64_t seed,
                                                void* d_keys_out, uint32_t* d_pos_out,
                                                uint64_t* d_offsets_out, void* stream) {
  if (type != RSORT_KEY_U64 && type != RSORT_KEY_F64) return RSORT_EINVAL;
  if (k < 1 || k > kNoAllocMaxK || n > 0xFFFFFFFFull) return RSORT_EINVAL;
  if (!d_offsets_out || (n > 0 && (!d_keys_in || !d_keys_out || !d_pos_out)))
    return RSORT_EINVAL;
  if (n > 0 && d_keys_in == d_keys_out) return RSORT_EINVAL;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return RSORT_ECUDA;
  }
  unsigned char* base = scratch_for_current_device(device);
  if (!base) return RSORT_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (cudaMemsetAsync(d_offsets_out, 0, (size_t)(k + 1) * 8, s) != cudaSuccess) {
      cudaGetLastError();
      return RSORT_ECUDA;
    }
    return RSORT_OK;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (sms <= 0) sms = 1;

  // Plan of one level with a bounded chunk count (so the histogram is bounded).
  const uint32_t kk = k < 2 ? 2 : k;
  uint64_t W = (n + kNoAllocMaxChunks - 1) / kNoAllocMaxChunks;
  const uint64_t per_sm = (n + 2ull * sms - 1) / (2ull * sms);
  if (W < per_sm) W = per_sm;
  W = (W + kSubTile - 1) / kSubTile * kSubTile;
  if (W > 0xFFFFFFFFull) return RSORT_EINVAL;
  const uint64_t chunks = (n + W - 1) / W;
  const uint64_t samp = std::min<uint64_t>(n, 16ull * ceil_log2(kk) * kk);
  const uint64_t hist = (uint64_t)kk * chunks;
  LevelParams P;
  P.level = 1;
  P.W = (uint32_t)W;
  P.seed = seed;
  P.samp_cap = samp;
  P.hist_cap = hist;
  P.chunk_cap = chunks;
  P.seg_cap = 1;
  P.final_cap = 1;
  P.schunk_cap = samp / kSampleChunk + 2;
  P.bucket_cap = kk;
  P.level1_oversample = 1;
  P.classifier = 0;
  P.warp_direct = 0;
  P.wide_scatter_k = 1 << 30;  // always the 2048-key sub-tile scatter
  P.target_bucket = kTargetBucket;

  uint64_t o = 0;
  auto take = [&](uint64_t bytes) {
    const uint64_t at = o;
    o = align256(o + (bytes ? bytes : 16));
    return base + at;
  };
  DevState* st = (DevState*)take(sizeof(DevState));
  FinalItem* items = (FinalItem*)take(sizeof(FinalItem));
  SegIn* list0 = (SegIn*)take(sizeof(SegIn));
  SegIn* list1 = (SegIn*)take(sizeof(SegIn));
  LevelSeg* segs = (LevelSeg*)take(sizeof(LevelSeg));
  uint64_t* samp_key = (uint64_t*)take(samp * 8);
  uint32_t* samp_idx = (uint32_t*)take(samp * 4);
  uint64_t* ssamp_key = (uint64_t*)take(samp * 8);
  uint32_t* ssamp_idx = (uint32_t*)take(samp * 4);
  uint32_t* hist_arr = (uint32_t*)take(hist * 4);
  uint32_t* sums = (uint32_t*)take((hist / kScanTile + 2) * 4);
  if (o > kNoAllocBytes) return RSORT_EINVAL;  // cannot happen for k <= kNoAllocMaxK

  LaunchEnv e;
  e.stream = s;
  e.num_sms = sms;
  e.timer = nullptr;
  e.launches = nullptr;
  // The control block is reset by the first kernel; every other scratch word
  // read later is written earlier in the same call.
  launch_init_plain(e, st, list1, items, n, k, 0, 1);
  Src src{(const uint64_t*)d_keys_in, nullptr, type == RSORT_KEY_F64};
  Dst dst{(uint64_t*)d_keys_out, d_pos_out};
  launch_level(e, P, st, list1, list0, segs, src, dst, kWhereOut, samp_key, samp_idx, ssamp_key,
               ssamp_idx, hist_arr, sums, items, (int)kk, 1, 0, d_offsets_out, n,
               type == RSORT_KEY_F64);
  if (cudaGetLastError() != cudaSuccess) return RSORT_ECUDA;
  return RSORT_OK;
}
