// partition_kernels.cu -- one level of the robust multi-level sample sort
// (Appendix "Robust Multi-Level Sample Sort" of Axtmann & Sanders,
// arXiv 1606.08766) over a device-resident list of segments:
//
//   plan -> sample -> sort the sample -> classify + per-chunk histograms ->
//   exclusive scan -> scatter -> collect the buckets
//
// The scatter keeps input order inside every bucket (the partition step's
// layout) unless the level is a full sort's deeper level, which may rank by
// shared-memory atomics instead (the in-SM sort orders (key, position) pairs).
//
// Every segment of the level is partitioned independently; all segments share
// the launches, so one level of a plain sort (one segment) and of a batched
// segmented sort (thousands of segments) run the same kernels.  The paper's
// processing elements are virtual partitions of HBM: the k buckets of a
// segment are its k virtual partitions, and the MPI_Alltoallv data exchange of
// the paper's sample sort becomes the scan + scatter through HBM.
#include <cstdio>

#include "async_copy.cuh"
#include "cta_sort.cuh"
#include "rsort_internal.cuh"
#include "splitters.cuh"

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

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

__global__ void k_init_plain(DevState* st, SegIn* list_l1, FinalItem* items, uint64_t n,
                             uint32_t k1, int direct, uint64_t final_cap, LocalPlan local) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->local = local;
  st->nseg[0] = st->nseg[1] = 0;
  for (int c = 0; c < kNumClasses; ++c) {
    st->nfinal_c[c] = 0;
    st->cursor_c[c] = 0;
    st->class_elems[c] = 0;
  }
  for (int a = 0; a < kNumAlgos; ++a) st->algo_elems[a] = 0;
  st->error = 0;
  st->max_bucket_l1 = 0;
  st->levels_used = 0;
  st->cur_nseg = 0;
  st->total_samples = st->total_chunks = st->total_hist = 0;
  st->total_schunks = st->total_buckets = 0;
  st->big_items = 0;
  for (int i = 0; i < 4; ++i) st->level_elems[i] = 0;
  if (n == 0) return;
  if (direct) {
    FinalItem f;
    f.start = 0;
    f.idx_base = 0;
    f.size = (uint32_t)n;
    f.where = kWhereInput;
    f.kind = n == 1 ? kKindCopy : kKindSort;
    push_final(st, items, final_cap, f, kErrFinalCap);
  } else {
    SegIn s;
    s.start = 0;
    s.m = (uint32_t)n;
    s.k_hint = k1;
    list_l1[0] = s;
    st->nseg[1] = 1;  // level 1 reads list parity 1
  }
}

// Per-segment parameters and prefix sums of one level (one CTA).
constexpr int kPlanThreads = 1024;
__global__ void __launch_bounds__(kPlanThreads)
k_level_plan(DevState* st, const SegIn* list_in, LevelSeg* segs, LevelParams P, int par_in,
             uint32_t kmax_level) {
  __shared__ uint64_t sm[kPlanThreads / 32];
  __shared__ uint64_t carry[6];
  __shared__ uint32_t sG;
  if (threadIdx.x == 0) {
    uint32_t G = st->nseg[par_in];
    st->nseg[par_in ^ 1] = 0;
    if (G > P.seg_cap) {
      atomicOr(&st->error, kErrSegCap);
      G = 0;
    }
    if (G) st->levels_used = P.level;
    if (P.level == 1) {
      st->l1_eq = 0;
      st->l1_nb = 0;
      st->l1_ordered = 0;
    }
    sG = G;
    for (int i = 0; i < 6; ++i) carry[i] = 0;
  }
  __syncthreads();
  const uint32_t G = sG;
  for (uint32_t base = 0; base < G; base += kPlanThreads) {
    const uint32_t g = base + threadIdx.x;
    uint64_t v[6] = {0, 0, 0, 0, 0, 0};
    SegIn in{};
    uint32_t k = 0, S = 0, nch = 0, nsch = 0;
    if (g < G) {
      in = list_in[g];
      if (in.k_hint >= 1) {
        k = min(in.k_hint, kmax_level);
      } else {
        const uint32_t cls = ceil_log2_dev(in.m);
        const uint32_t tb = (cls <= 32 && P.target_by_class[cls]) ? P.target_by_class[cls]
                                                                  : P.target_bucket;
        const uint64_t want = ((uint64_t)in.m + tb - 1) / tb;
        k = (uint32_t)umax64(2, umin64(want, kmax_level));
      }
      const uint64_t a = (in.k_hint >= 1 && P.level1_oversample)
                             ? 16ull * ceil_log2_dev(k) : (uint64_t)kDeepOversample;
      S = (uint32_t)umin64(in.m, a * k);
      nch = (uint32_t)((in.m + (uint64_t)P.W - 1) / P.W);
      nsch = (S + kSampleChunk - 1) / kSampleChunk;
      v[0] = S;
      v[1] = nch;
      v[2] = (uint64_t)k * nch * (P.warp_direct ? kPartWarps : 1);
      v[3] = nsch;
      v[4] = k;
      v[5] = in.m;
    }
    uint64_t ex[6], tot[6];
    for (int i = 0; i < 6; ++i) ex[i] = block_excl_scan_u64<kPlanThreads>(v[i], &tot[i], sm);
    if (g < G) {
      LevelSeg s;
      s.start = in.start;
      s.seed = P.level == 1 ? P.seed
                            : splitmix64_at(P.seed, ((uint64_t)P.level << 40) ^ in.start);
      s.samp_off = carry[0] + ex[0];
      s.chunk_off = carry[1] + ex[1];
      s.hist_off = carry[2] + ex[2];
      s.schunk_off = carry[3] + ex[3];
      s.bkt_off = carry[4] + ex[4];
      s.delta = in.start - (carry[5] + ex[5]);
      s.m = in.m;
      s.k = k;
      s.S = S;
      s.nchunks = nch;
      s.nschunks = nsch;
      s.nunits = nch * (P.warp_direct ? kPartWarps : 1);
      // equal chunks inside the segment (the level's W bounds their size)
      s.W = nch ? (uint32_t)(((uint64_t)in.m + nch - 1) / nch) : P.W;
      s.pad = 0;
      segs[g] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 0; i < 6; ++i) carry[i] += tot[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    uint32_t err = 0;
    if (carry[0] > P.samp_cap) err |= kErrSampleCap;
    if (carry[1] > P.chunk_cap) err |= kErrChunkCap;
    if (carry[2] > P.hist_cap) err |= kErrHistCap;
    if (carry[3] > P.schunk_cap) err |= kErrSchunkCap;
    if (carry[4] > P.bucket_cap) err |= kErrBucketCap;
    if (err) {
      atomicOr(&st->error, err);
      st->cur_nseg = 0;
      st->total_samples = st->total_chunks = st->total_hist = 0;
      st->total_schunks = st->total_buckets = 0;
    } else {
      st->cur_nseg = G;
      st->total_samples = carry[0];
      st->total_chunks = carry[1];
      st->total_hist = carry[2];
      st->total_schunks = carry[3];
      st->total_buckets = carry[4];
      if (P.level >= 1 && P.level <= 4) st->level_elems[P.level - 1] = carry[5];
    }
  }
}

// Step 1: stratified random samples, each carrying its position.  Sample j of
// a segment of m elements with S samples comes from positions
// [floor(j*m/S), floor((j+1)*m/S)) at offset splitmix64(seed, j) mod size.
__global__ void __launch_bounds__(256)
k_sample(const DevState* st, const LevelSeg* segs, Src src, uint64_t* samp_key,
         uint32_t* samp_idx) {
  const uint64_t total = st->total_samples;
  const uint32_t G = st->cur_nseg;
  // every CTA draws a contiguous range of samples, so a thread's segment
  // changes rarely and the segment search runs once per segment, not per sample
  const uint64_t span = (total + gridDim.x - 1) / gridDim.x;
  const uint64_t s0 = (uint64_t)blockIdx.x * span;
  const uint64_t s1 = umin64(total, s0 + span);
  uint32_t g = 0;
  uint64_t g_lo = 1, g_hi = 0;  // sample range of the cached segment (empty)
  for (uint64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    if (s < g_lo || s >= g_hi) {
      g = find_seg(segs, G, s, [](const LevelSeg& x) { return x.samp_off; });
      g_lo = segs[g].samp_off;
      g_hi = g_lo + segs[g].S;
    }
    const LevelSeg& sg = segs[g];
    const uint64_t j = s - sg.samp_off;
    const uint64_t lo = (j * sg.m) / sg.S, hi = ((j + 1) * sg.m) / sg.S;
    const uint64_t pos = lo + splitmix64_at(sg.seed, j) % (hi - lo);
    const uint64_t at = sg.start + pos;
    samp_key[s] = load_key(src, at);
    samp_idx[s] = src.idx ? src.idx[at] : (uint32_t)pos;
  }
}

// Step 2a: sort chunks of up to kSampleChunk sample pairs in one CTA each
// (cta_sort_pairs).  Single-chunk samples go straight to the sorted-sample
// array.  Samples are drawn in segment order, which is position order when
// the segment's level input is (in_order).
__global__ void __launch_bounds__(kSampleThreads, 1)
k_sample_sort_chunks(const DevState* st, const LevelSeg* segs, uint64_t* samp_key,
                     uint32_t* samp_idx, uint64_t* ssamp_key, uint32_t* ssamp_idx,
                     int in_order) {
  constexpr int NT = kSampleThreads, IT = kSampleChunk / kSampleThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CtaSortSmem s;
  s.k = (uint64_t*)smem_raw;
  s.i = (uint32_t*)(s.k + kSampleChunk);
  s.hist = s.i + kSampleChunk;
  __shared__ uint64_t red[2 * NT / 32];
  __shared__ uint64_t scan_sm[NT / 32];
  const uint64_t total = st->total_schunks;
  const uint32_t G = st->cur_nseg;
  for (uint64_t c = blockIdx.x; c < total; c += gridDim.x) {
    const uint32_t g = find_seg(segs, G, c, [](const LevelSeg& x) { return x.schunk_off; });
    const LevelSeg sg = segs[g];
    const uint64_t cl = c - sg.schunk_off;
    const uint64_t base = sg.samp_off + cl * kSampleChunk;
    const uint32_t len = (uint32_t)umin64(kSampleChunk, sg.S - cl * kSampleChunk);
    uint64_t key[IT];
    uint32_t idx[IT];
#pragma unroll
    for (int r = 0; r < IT; ++r) {
      const uint32_t e = r * NT + threadIdx.x;
      if (e < len) {
        key[r] = samp_key[base + e];
        idx[r] = samp_idx[base + e];
      }
    }
    cta_sort_pairs<NT, IT>(key, idx, len,
                           [&] { return in_order == kOrderAuto ? st->l1_ordered != 0
                                                               : in_order != 0; },
                           s, red, scan_sm, nullptr);
    uint64_t* ok = sg.nschunks == 1 ? ssamp_key : samp_key;
    uint32_t* oi = sg.nschunks == 1 ? ssamp_idx : samp_idx;
    for (uint32_t t = threadIdx.x; t < len; t += NT) {
      ok[base + t] = s.k[t];
      oi[base + t] = s.i[t];
    }
    __syncthreads();
  }
}

// Step 2b: merge sorted chunks by ranking (the fast work-inefficient ranking
// idea of Appendix "Fast Work-Inefficient Ranking": the rank of an element is
// its rank in its own sorted sequence plus its ranks in the other sorted
// sequences).
__global__ void __launch_bounds__(256)
k_sample_merge_rank(const DevState* st, const LevelSeg* segs, const uint64_t* samp_key,
                    const uint32_t* samp_idx, uint64_t* ssamp_key, uint32_t* ssamp_idx) {
  const uint64_t total = st->total_samples;
  const uint32_t G = st->cur_nseg;
  // contiguous sample range per CTA, segment searched once per segment
  const uint64_t span = (total + gridDim.x - 1) / gridDim.x;
  const uint64_t s0 = (uint64_t)blockIdx.x * span;
  const uint64_t s1 = umin64(total, s0 + span);
  uint32_t g = 0;
  uint64_t g_lo = 1, g_hi = 0;
  for (uint64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    if (s < g_lo || s >= g_hi) {
      g = find_seg(segs, G, s, [](const LevelSeg& x) { return x.samp_off; });
      g_lo = segs[g].samp_off;
      g_hi = g_lo + segs[g].S;
    }
    const LevelSeg& sg = segs[g];
    if (sg.nschunks <= 1) continue;
    const uint64_t j = s - sg.samp_off;
    const uint32_t c = (uint32_t)(j / kSampleChunk);
    const uint64_t myk = samp_key[s];
    const uint32_t myi = samp_idx[s];
    uint64_t rank = j - (uint64_t)c * kSampleChunk;
    for (uint32_t c2 = 0; c2 < sg.nschunks; ++c2) {
      if (c2 == c) continue;
      const uint64_t b0 = sg.samp_off + (uint64_t)c2 * kSampleChunk;
      const uint64_t len = umin64(kSampleChunk, sg.S - (uint64_t)c2 * kSampleChunk);
      uint64_t lo = 0, hi = len;
      while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (pair_less(samp_key[b0 + mid], samp_idx[b0 + mid], myk, myi)) lo = mid + 1;
        else hi = mid;
      }
      rank += lo;
    }
    ssamp_key[sg.samp_off + rank] = myk;
    ssamp_idx[sg.samp_off + rank] = myi;
  }
}

// Shared-memory carve-up of the classify / scatter kernels.
constexpr int kCT = 2048;                       // keys per classify pipeline stage
constexpr int kCStages = 3;                     // classify stages at level 1 (2 in flight)
constexpr int kCStagesDeep = 2;                 // deeper levels: fewer stages, more CTAs per SM
constexpr int kCItems = kCT / kPartThreads;     // 8 keys per lane per stage
constexpr int kST = 2048;                       // keys per scatter sub-tile
constexpr int kSItems = kST / kPartThreads;     // 8 keys per lane per sub-tile
static_assert(kSItems * 32 * kPartWarps == kST, "warp w owns kSItems*32 consecutive keys");

struct PartSmem {
  Splitters sp;
  uint32_t* hist;      // [K]   classify: counts;  scatter: running offsets
  uint32_t* sbase;     // [K+1] scatter: sub-tile bucket starts
  uint16_t* wcnt;      // [kPartWarps][cnt_stride(K)] scatter: per-warp counts / bases
  uint32_t* dlt;       // scatter: [K] output position minus sub-tile run start, per bucket
  uint8_t* wwin;       // [kPartWarps][K] scatter: per-warp winner lane of each bucket
  unsigned char* buf;  // classify: kCStages key stages; scatter: two sub-tile buffers
};


// one scatter sub-tile buffer: keys, positions, bucket ids
constexpr size_t kSBufBytes = (size_t)kST * (8 + 4 + 2);

// mode: bit 0 the classifier (0 tree, 1 table), bit 1 no tie-breaking.
__host__ __device__ inline size_t part_common_bytes(uint32_t kmax, int mode) {
  const size_t Kp = next_pow2_u32(kmax);
  size_t b = (mode & 1) == 0 ? Kp * 8 : ((size_t)4 << table_bits_for((uint32_t)Kp));
  b += (size_t)kmax * 8 + (size_t)kmax * 4 + (size_t)kmax * 2 + (size_t)kmax * 4;
  return (b + 15) & ~(size_t)15;
}

__host__ __device__ inline size_t classify_smem_bytes(uint32_t kmax, int mode, int stages) {
  return part_common_bytes(kmax, mode) + (size_t)stages * kCT * 8;
}

__host__ __device__ inline size_t part_smem_bytes(uint32_t kmax, bool scatter, int mode) {
  size_t b = part_common_bytes(kmax, mode);
  if (scatter) {
    b += (size_t)(kmax + 1) * 4 + 4;
    b += (size_t)kPartWarps * cnt_stride(kmax) * 2;
    b = (b + 15) & ~(size_t)15;
    b += 2 * kSBufBytes;
  } else {
    b += (size_t)kCStages * kCT * 8;
  }
  return b;
}

__device__ inline PartSmem carve(unsigned char* base, uint32_t kmax, bool scatter, int mode) {
  PartSmem s;
  const size_t Kp = next_pow2_u32(kmax);
  unsigned char* p = base;
  s.sp.mode = mode & 1;
  s.sp.ntb = (mode >> 1) & 1;
  s.sp.tree = nullptr;
  s.sp.tbl = nullptr;
  if (s.sp.mode == 0) {
    s.sp.tree = (uint64_t*)p;
    p += Kp * 8;
  } else {
    s.sp.tbl = (uint32_t*)p;
    p += (size_t)4 << table_bits_for((uint32_t)Kp);
  }
  s.sp.key = (uint64_t*)p; p += (size_t)kmax * 8;
  s.sp.idx = (uint32_t*)p; p += (size_t)kmax * 4;
  s.hist = (uint32_t*)p; p += (size_t)kmax * 4;
  s.sp.rend = (uint16_t*)p; p += (size_t)kmax * 2;
  p = base + part_common_bytes(kmax, mode);
  s.sbase = nullptr;
  s.wcnt = nullptr;
  s.dlt = nullptr;
  s.wwin = nullptr;
  if (scatter) {
    s.sbase = (uint32_t*)p; p += (size_t)(kmax + 1) * 4 + 4;
    s.wcnt = (uint16_t*)p; p += (size_t)kPartWarps * cnt_stride(kmax) * 2;
    p = (unsigned char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  }
  s.buf = p;
  return s;
}

// Dynamic shared memory the wide (512-thread, 4096-key) scatter may use: the
// device's opt-in limit minus the kernel's static shared memory, found when
// the kernel attributes are set (0 until then, or if CUDA refused).  The wide
// scatter runs only when its carve-up fits.
static size_t g_wide_scatter_smem_max = 0;

// Shared memory of the staged scatter with NW warps and ST-key sub-tiles.
// The stable scatter keeps per-warp counters and winner slots per bucket; the
// unstable one a single 32-bit counter per bucket (in place of the former).
__host__ __device__ inline size_t scatter_smem_bytes(uint32_t kmax, int mode, int nw, int st,
                                                     bool stable = true) {
  size_t b = part_common_bytes(kmax, mode);
  b += (size_t)(kmax + 1) * 4 + 4;
  b += stable ? (size_t)nw * cnt_stride(kmax) * 2 : (size_t)kmax * 4;
  b += (size_t)kmax * 4;
  b += stable ? (size_t)nw * kmax : 0;
  b = (b + 15) & ~(size_t)15;
  return b + 2 * ((size_t)st * (8 + 4 + 2) + 16);
}

__device__ inline PartSmem carve_scatter(unsigned char* base, uint32_t kmax, int mode, int nw,
                                         bool stable = true) {
  PartSmem s = carve(base, kmax, false, mode);
  unsigned char* p = base + part_common_bytes(kmax, mode);
  s.sbase = (uint32_t*)p;
  p += (size_t)(kmax + 1) * 4 + 4;
  s.wcnt = (uint16_t*)p;
  p += stable ? (size_t)nw * cnt_stride(kmax) * 2 : (size_t)kmax * 4;
  s.dlt = (uint32_t*)p;
  p += (size_t)kmax * 4;
  s.wwin = (uint8_t*)p;
  p += stable ? (size_t)nw * kmax : 0;
  s.buf = (unsigned char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  return s;
}

// Steps 4 + 5a: classify every element and count, per chunk of W elements,
// how many fall into each bucket.  hist is laid out per segment bucket-major:
// hist[hist_off + b * nchunks + chunk].  The chunk's keys stream through a
// STAGES-deep cp.async pipeline of kCT-key stages in shared memory.  Level 1
// (few long chunks) runs 3 stages at 3 CTAs per SM; deeper levels (many
// short chunks, each loading its segment's splitters) measured faster with 2
// stages at 4 CTAs per SM.
template <int STAGES>
__global__ void __launch_bounds__(kPartThreads, STAGES == 2 ? 4 : 3)
k_classify_count(const DevState* st, const LevelSeg* segs, Src src, const uint64_t* ssk,
                 const uint32_t* ssi, uint32_t* hist, uint32_t W, uint32_t kmax, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PartSmem sm = carve(smem_raw, kmax, false, mode);
  uint64_t* stage = (uint64_t*)sm.buf;
  const uint64_t pol = l2_evict_first_policy();
  const uint64_t total = st->total_chunks;
  const uint32_t G = st->cur_nseg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t cur_g = 0xffffffffu;
  for (uint64_t c = blockIdx.x; c < total; c += gridDim.x) {
    const uint32_t g = find_seg(segs, G, c, [](const LevelSeg& x) { return x.chunk_off; });
    const LevelSeg sg = segs[g];
    __syncthreads();
    if (g != cur_g) {
      load_splitters<kPartThreads>(sg, ssk, ssi, sm.sp);
      cur_g = g;
    }
    for (uint32_t b = threadIdx.x; b < sg.k; b += kPartThreads) sm.hist[b] = 0;
    const uint64_t cl = c - sg.chunk_off;
    const uint64_t cs = sg.start + cl * sg.W;
    const uint64_t ce = umin64(cs + sg.W, sg.start + sg.m);
    const uint64_t nst = (ce - cs + kCT - 1) / kCT;
    auto issue = [&](uint64_t s) {
      if (s < nst) {
        const uint64_t b0 = cs + s * kCT;
        const uint32_t len = (uint32_t)umin64(kCT, ce - b0);
        uint64_t* dst = stage + (s % STAGES) * kCT;
        for (uint32_t t = threadIdx.x; t < len; t += kPartThreads)
          cp_async_8(dst + t, src.key + b0 + t, pol);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) issue(s);
    for (uint64_t s = 0; s < nst; ++s) {
      cp_async_wait<STAGES - 2>();
      __syncthreads();
      issue(s + STAGES - 1);
      const uint64_t b0 = cs + s * kCT;
      const uint32_t len = (uint32_t)umin64(kCT, ce - b0);
      const uint64_t* stg = stage + (s % STAGES) * kCT;
      const uint32_t q0 = (uint32_t)warp * (kCItems * 32) + lane;
      uint64_t key[kCItems];
#pragma unroll
      for (int r = 0; r < kCItems; ++r) {
        const uint32_t q = q0 + r * 32;
        const uint64_t k = q < len ? stg[q] : 0;
        key[r] = src.map_f64 ? f64_to_ordered(k) : k;
      }
      uint32_t bk[kCItems];
      // positions are read only when a key ties with a splitter key, and
      // never past the stage (a padding slot's key 0 may tie; its result is
      // discarded)
      classify_batch<kCItems>(key, bk, [&](int r) {
        const uint32_t q = q0 + r * 32;
        if (q >= len) return 0u;
        const uint64_t pos = b0 + q;
        return src.idx ? src.idx[pos] : (uint32_t)(pos - sg.start);
      }, sm.sp);
      if (src.bid) {
#pragma unroll
        for (int r = 0; r < kCItems; ++r)
          if (q0 + r * 32 < len) src.bid[b0 + q0 + r * 32] = (uint16_t)bk[r];
      }
      // runs of one bucket across the warp (duplicate-heavy inputs) take one
      // atomic per warp and slot; otherwise one atomic per key
      const uint32_t bw = __shfl_sync(0xffffffffu, bk[0], 0);
      if (__popc(__ballot_sync(0xffffffffu, bk[0] == bw)) > 8) {
#pragma unroll
        for (int r = 0; r < kCItems; ++r) {
          const bool v = q0 + r * 32 < len;
          const uint32_t b = bk[r];
          const uint32_t bl = __shfl_sync(0xffffffffu, b, 0);
          if (__all_sync(0xffffffffu, v && b == bl)) {
            if (lane == 0) atomicAdd(&sm.hist[bl], 32u);
          } else if (v) {
            atomicAdd(&sm.hist[b], 1u);
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < kCItems; ++r)
          if (q0 + r * 32 < len) atomicAdd(&sm.hist[bk[r]], 1u);
      }
    }
    cp_async_wait<0>();
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < sg.k; b += kPartThreads)
      hist[sg.hist_off + (uint64_t)b * sg.nunits + cl] = sm.hist[b];
  }
}

// Step 5b: exclusive scan of the histogram counters (three launches).
__global__ void __launch_bounds__(1024)
k_scan_reduce(const DevState* st, const uint32_t* a, uint32_t* sums) {
  __shared__ uint64_t sm[32];
  const uint64_t total = st->total_hist;
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  if (base >= total) return;
  uint64_t v = 0;
  for (int r = 0; r < 4; ++r) {
    const uint64_t i = base + threadIdx.x * 4 + r;
    if (i < total) v += a[i];
  }
  uint64_t tot;
  block_excl_scan_u64<1024>(v, &tot, sm);
  if (threadIdx.x == 0) sums[blockIdx.x] = (uint32_t)tot;
}

__global__ void __launch_bounds__(1024)
k_scan_sums(const DevState* st, uint32_t* sums) {
  __shared__ uint64_t sm[32];
  const uint64_t total = st->total_hist;
  const uint64_t ntiles = (total + kScanTile - 1) / kScanTile;
  uint64_t carry = 0;
  for (uint64_t b = 0; b < ntiles; b += 1024) {
    const uint64_t i = b + threadIdx.x;
    const uint64_t v = i < ntiles ? sums[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_excl_scan_u64<1024>(v, &tot, sm);
    if (i < ntiles) sums[i] = (uint32_t)(carry + ex);
    carry += tot;
  }
}

__global__ void __launch_bounds__(1024)
k_scan_down(const DevState* st, uint32_t* a, const uint32_t* sums) {
  __shared__ uint64_t sm[32];
  const uint64_t total = st->total_hist;
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  if (base >= total) return;
  uint32_t x[4];
  uint64_t v = 0;
  for (int r = 0; r < 4; ++r) {
    const uint64_t i = base + threadIdx.x * 4 + r;
    x[r] = i < total ? a[i] : 0;
    v += x[r];
  }
  uint64_t tot;
  uint64_t run = block_excl_scan_u64<1024>(v, &tot, sm) + sums[blockIdx.x];
  for (int r = 0; r < 4; ++r) {
    const uint64_t i = base + threadIdx.x * 4 + r;
    if (i < total) a[i] = (uint32_t)run;
    run += x[r];
  }
}

// Step 5c: scatter.  Every chunk streams through two ST-key sub-tile buffers
// (cp.async: sub-tile s+1 loads while s is processed).  Every element gets a
// rank among the elements of its bucket in the sub-tile; the sub-tile is then
// counting-sorted by bucket into its own buffer and every bucket's run is
// written out contiguously (write-combining through shared memory).
//   STABLE   warp w owns IT*32 consecutive elements; ranks come from
//            warp-synchronous peer counting (warp order, then lane order =
//            input order), so buckets keep input order -- the layout of the
//            partition step.
//   unstable one shared-memory atomic per element on its bucket's counter:
//            buckets come out in no particular order, which a full sort's
//            deeper levels may do (the in-SM sort orders (key, position)
//            pairs).
template <int NT, int ST, bool STABLE>
__global__ void __launch_bounds__(NT, (NT <= 256 ? 2 : 1))
k_scatter(const DevState* st, const LevelSeg* segs, Src src, const uint64_t* ssk,
          const uint32_t* ssi, const uint32_t* hist_scan, Dst dst, uint32_t W, uint32_t kmax,
          int unmap_out, int mode) {
  constexpr int NW = NT / 32;
  constexpr int IT = ST / NT;
  static_assert(IT * 32 * NW == ST, "warp w owns IT*32 consecutive keys of a sub-tile");
  // keys, positions, bucket ids (+16 bytes: the staged ids start at an even
  // position, one before the sub-tile when it starts at an odd one)
  constexpr size_t BUFB = (size_t)ST * (8 + 4 + 2) + 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PartSmem sm = carve_scatter(smem_raw, kmax, mode, NW, STABLE);
  uint32_t* cntu = reinterpret_cast<uint32_t*>(sm.wcnt);  // unstable: one counter per bucket
  if constexpr (!STABLE) {
    for (uint32_t b = threadIdx.x; b < kmax; b += NT) cntu[b] = 0;
  }
  __shared__ uint64_t scan_sm[NW];
  // sub-tile buffer i: keys, positions, bucket ids (addressed arithmetically so
  // that no descriptor array lives in local memory)
  struct Buf {
    uint64_t* key;
    uint32_t* idx;
    uint16_t* b;
  };
  auto buf_of = [&](uint64_t i) {
    unsigned char* p = sm.buf + (size_t)(i & 1) * BUFB;
    Buf r;
    r.key = (uint64_t*)p;
    r.idx = (uint32_t*)(p + (size_t)ST * 8);
    r.b = (uint16_t*)(p + (size_t)ST * 12);
    return r;
  };
  const uint64_t pol = l2_evict_first_policy();
  const uint64_t pol_keep = l2_evict_last_policy();
  const uint64_t total = st->total_chunks;
  const uint32_t G = st->cur_nseg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t ltmask = lanemask_lt();
  const uint32_t kst = cnt_stride(kmax);
  uint16_t* my_cnt = sm.wcnt + (size_t)warp * kst;
  uint8_t* my_win = sm.wwin + (size_t)warp * kmax;
  uint32_t cur_g = 0xffffffffu;
  for (uint64_t c = blockIdx.x; c < total; c += gridDim.x) {
    const uint32_t g = find_seg(segs, G, c, [](const LevelSeg& x) { return x.chunk_off; });
    const LevelSeg sg = segs[g];
    __syncthreads();
    if (g != cur_g) {
      load_splitters<NT>(sg, ssk, ssi, sm.sp);
      cur_g = g;
    }
    const uint32_t k = sg.k;
    const int nbits = k > 32 ? 5 : (int)ceil_log2_dev(k);
    const uint64_t cl = c - sg.chunk_off;
    for (uint32_t b = threadIdx.x; b < k; b += NT)
      sm.hist[b] = (uint32_t)(hist_scan[sg.hist_off + (uint64_t)b * sg.nunits + cl] + sg.delta);
    const uint64_t cs = sg.start + cl * sg.W;
    const uint64_t ce = umin64(cs + sg.W, sg.start + sg.m);
    const uint64_t nst = (ce - cs + ST - 1) / ST;
    auto issue = [&](uint64_t s) {
      if (s < nst) {
        const uint64_t b0 = cs + s * ST;
        const uint32_t len = (uint32_t)umin64(ST, ce - b0);
        const Buf B = buf_of(s);
        for (uint32_t t = threadIdx.x; t < len; t += NT) {
          cp_async_8(B.key + t, src.key + b0 + t, pol);
          if (src.idx) cp_async_4(B.idx + t, src.idx + b0 + t, pol);
        }
        if (src.bid) {  // bucket ids as 4-byte pairs from the even position at or below b0
          const uint64_t w0 = b0 >> 1;
          const uint32_t nw = (uint32_t)(((b0 + len + 1) >> 1) - w0);
          const uint32_t* gw = reinterpret_cast<const uint32_t*>(src.bid) + w0;
          for (uint32_t t = threadIdx.x; t < nw; t += NT)
            cp_async_4(reinterpret_cast<uint32_t*>(B.b) + t, gw + t, pol);
        }
      }
      cp_async_commit();
    };
    issue(0);
    for (uint64_t s = 0; s < nst; ++s) {
      cp_async_wait<0>();
      __syncthreads();
      issue(s + 1);
      const Buf B = buf_of(s);
      const uint64_t b0 = cs + s * ST;
      const uint32_t len = (uint32_t)umin64(ST, ce - b0);
      const uint32_t q0 = (uint32_t)warp * (IT * 32) + lane;
      uint64_t key[IT];
      uint32_t idx[IT];
      uint32_t bk[IT];
      uint32_t lrank[IT];
#pragma unroll
      for (int r = 0; r < IT; ++r) {
        const uint32_t q = q0 + r * 32;
        const bool v = q < len;
        const uint64_t kv = v ? B.key[q] : 0;
        key[r] = src.map_f64 ? f64_to_ordered(kv) : kv;
        idx[r] = v ? (src.idx ? B.idx[q] : (uint32_t)(b0 + q - sg.start)) : 0;
      }
      if (src.bid) {
        const uint16_t* bh = B.b + (b0 & 1);
#pragma unroll
        for (int r = 0; r < IT; ++r) {
          const uint32_t q = q0 + r * 32;
          bk[r] = q < len ? bh[q] : 0u;
        }
      } else {
        classify_batch<IT>(key, bk, [&](int r) { return idx[r]; }, sm.sp);
      }
      if constexpr (!STABLE) {
#pragma unroll
        for (int r = 0; r < IT; ++r) {
          const bool v = q0 + r * 32 < len;
          bk[r] = v ? bk[r] : 0xffffffffu;
          lrank[r] = v ? atomicAdd(&cntu[bk[r]], 1u) : 0u;
        }
      } else {
      for (uint32_t q = lane; q < (k + 1) / 2; q += 32) ((uint32_t*)my_cnt)[q] = 0;
      __syncwarp();
#pragma unroll
      for (int r = 0; r < IT; ++r) {
        const bool v = q0 + r * 32 < len;
        const uint32_t b = v ? bk[r] : 0xffffffffu;
        bk[r] = b;
        // peers = the lanes holding the same bucket.  Up to 32 buckets the
        // bucket bits are compared by ballots; beyond, every lane first writes
        // its lane id to the warp's slot of its bucket, and the lane id that
        // stayed there (one per distinct bucket) is compared instead: 5
        // ballots whatever k is.
        uint32_t w = b;
        if (k > 32) {
          if (v) my_win[b] = (uint8_t)lane;
          __syncwarp();
          w = v ? my_win[b] : 0u;
          __syncwarp();
        }
        uint32_t peers = __ballot_sync(0xffffffffu, v);
        // every lane kept its own slot: the warp's buckets are distinct, so
        // each lane is its bucket's only peer (the common case for k >> 32)
        const bool alone = k > 32 && __all_sync(0xffffffffu, !v || w == (uint32_t)lane);
        if (alone) {
          peers &= 1u << lane;
        } else {
#pragma unroll
          for (int bit = 0; bit < 5; ++bit) {
            if (bit < nbits) {
              const bool one = (w >> bit) & 1u;
              const uint32_t m = __ballot_sync(0xffffffffu, one);
              peers &= one ? m : ~m;
            }
          }
        }
        const uint32_t c0 = v ? my_cnt[b] : 0;
        __syncwarp();
        if (v && lane == __ffs(peers) - 1) my_cnt[b] = (uint16_t)(c0 + __popc(peers));
        __syncwarp();
        lrank[r] = c0 + __popc(peers & ltmask);
      }
      }  // STABLE
      __syncthreads();
      {  // per bucket (each thread a run of buckets): exclusive prefix over the
         // warps' counts, in place; an exclusive scan of the bucket totals then
         // places every bucket's run in the sub-tile, and the running output
         // offsets advance by the totals
        const uint32_t per = (k + NT - 1) / NT;
        const uint32_t bb0 = threadIdx.x * per;
        const uint32_t bb1 = bb0 + per < k ? bb0 + per : k;
        uint32_t loc = 0;
        uint32_t b0s = bb0;
        if constexpr (STABLE) {
          // two buckets at a time: their 16-bit counters share a 32-bit word
          // (rows have even length, bb0 is even when per is), and no count or
          // prefix exceeds the sub-tile, so halfword adds never carry
          for (; (per & 1) == 0 && b0s + 1 < bb1; b0s += 2) {
            uint32_t tot2 = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
              uint32_t* cw = reinterpret_cast<uint32_t*>(sm.wcnt + (size_t)w * kst + b0s);
              const uint32_t cnt2 = *cw;
              *cw = tot2;
              tot2 = __vadd2(tot2, cnt2);
            }
            sm.sbase[b0s] = tot2 & 0xffffu;
            sm.sbase[b0s + 1] = tot2 >> 16;
            loc += (tot2 & 0xffffu) + (tot2 >> 16);
          }
        }
        for (uint32_t b = b0s; b < bb1; ++b) {
          uint32_t tot = 0;
          if constexpr (STABLE) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
              const uint32_t cnt = sm.wcnt[(size_t)w * kst + b];
              sm.wcnt[(size_t)w * kst + b] = (uint16_t)tot;
              tot += cnt;
            }
          } else {
            tot = cntu[b];
            cntu[b] = 0;  // ready for the next sub-tile (its atomics follow barriers)
          }
          sm.sbase[b] = tot;
          loc += tot;
        }
        uint64_t tot;
        uint32_t run = (uint32_t)block_excl_scan_u64<NT>(loc, &tot, scan_sm);
        for (uint32_t b = bb0; b < bb1; ++b) {
          const uint32_t t = sm.sbase[b];
          sm.sbase[b] = run;
          sm.dlt[b] = sm.hist[b] - run;  // modulo 2^32: positions are below 2^32
          sm.hist[b] += t;
          run += t;
        }
      }
      __syncthreads();
      // counting-sort the sub-tile by bucket into its own buffer
#pragma unroll
      for (int r = 0; r < IT; ++r) {
        const uint32_t b = bk[r];
        if (b != 0xffffffffu) {
          const uint32_t q = sm.sbase[b] + (STABLE ? (uint32_t)my_cnt[b] : 0u) + lrank[r];
          B.key[q] = key[r];
          B.idx[q] = idx[r];
          B.b[q] = (uint16_t)b;
        }
      }
      __syncthreads();
      for (uint32_t q = threadIdx.x; q < len; q += NT) {
        const uint32_t b = B.b[q];
        const uint64_t d = (uint32_t)(sm.dlt[b] + q);
        const uint64_t kv = B.key[q];
        st_keep_u64(dst.key + d, unmap_out ? ordered_to_f64(kv) : kv, pol_keep);
        st_keep_u32(dst.idx + d, B.idx[q], pol_keep);
      }
    }
    cp_async_wait<0>();
  }
}

// ---------------------------------------------------------------------------
// Warp-direct variant of steps 4-5a / 5c.  Every chunk is split into
// kPartWarps contiguous warp sub-chunks; the histogram has one unit per
// (chunk, warp).  A warp streams its own sub-chunk through kWdStages
// cp.async stages of kWdKeys keys (warp-level waits only), ranks elements
// among equal buckets with match counting, and writes them straight to HBM
// from warp-private running offsets.  No block barrier inside a chunk; the
// order inside a bucket is still the input order.
// ---------------------------------------------------------------------------
constexpr int kWdItems = 4;                   // keys per lane per stage
constexpr int kWdKeys = 32 * kWdItems;        // keys per warp per stage
constexpr int kWdStages = 2;

__host__ __device__ inline size_t wd_smem_bytes(uint32_t kmax, int mode) {
  return part_common_bytes(kmax, mode) + (size_t)kPartWarps * kmax * 4 +
         (size_t)kPartWarps * kWdStages * kWdKeys * (8 + 4);
}

struct WdSmem {
  Splitters sp;
  uint32_t* rows;   // [kPartWarps][kmax]: counts (classify) / next position (scatter)
  uint64_t* skey;   // [kPartWarps][kWdStages][kWdKeys]
  uint32_t* sidx;   // [kPartWarps][kWdStages][kWdKeys]
};

__device__ inline WdSmem carve_wd(unsigned char* base, uint32_t kmax, int mode) {
  PartSmem ps = carve(base, kmax, false, mode);
  WdSmem w;
  w.sp = ps.sp;
  unsigned char* p = base + part_common_bytes(kmax, mode);
  w.rows = (uint32_t*)p;
  p += (size_t)kPartWarps * kmax * 4;
  w.skey = (uint64_t*)p;
  p += (size_t)kPartWarps * kWdStages * kWdKeys * 8;
  w.sidx = (uint32_t*)p;
  return w;
}

// This warp's sub-chunk [ws, we) of chunk [cs, ce).
__device__ __forceinline__ void warp_subchunk(uint64_t cs, uint64_t ce, int warp, uint64_t& ws,
                                              uint64_t& we) {
  const uint64_t cnt = ce - cs;
  const uint64_t wsz = (cnt + kPartWarps - 1) / kPartWarps;
  ws = cs + umin64((uint64_t)warp * wsz, cnt);
  we = cs + umin64((uint64_t)(warp + 1) * wsz, cnt);
}

__global__ void __launch_bounds__(kPartThreads, 3)
k_classify_count_wd(const DevState* st, const LevelSeg* segs, Src src, const uint64_t* ssk,
                    const uint32_t* ssi, uint32_t* hist, uint32_t W, uint32_t kmax, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WdSmem sm = carve_wd(smem_raw, kmax, mode);
  const uint64_t pol = l2_evict_first_policy();
  const uint64_t total = st->total_chunks;
  const uint32_t G = st->cur_nseg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* row = sm.rows + (size_t)warp * kmax;
  uint64_t* stk = sm.skey + (size_t)warp * kWdStages * kWdKeys;
  uint32_t cur_g = 0xffffffffu;
  for (uint64_t c = blockIdx.x; c < total; c += gridDim.x) {
    const uint32_t g = find_seg(segs, G, c, [](const LevelSeg& x) { return x.chunk_off; });
    const LevelSeg sg = segs[g];
    __syncthreads();
    if (g != cur_g) {
      load_splitters<kPartThreads>(sg, ssk, ssi, sm.sp);
      cur_g = g;
    }
    const uint32_t k = sg.k;
    for (uint32_t b = lane; b < k; b += 32) row[b] = 0;
    const uint64_t cl = c - sg.chunk_off;
    const uint64_t cs = sg.start + cl * sg.W;
    const uint64_t ce = umin64(cs + sg.W, sg.start + sg.m);
    uint64_t ws, we;
    warp_subchunk(cs, ce, warp, ws, we);
    const uint64_t nsteps = (we - ws + kWdKeys - 1) / kWdKeys;
    auto issue = [&](uint64_t t) {
      if (t < nsteps) {
        const uint64_t b0 = ws + t * kWdKeys;
        uint64_t* dstk = stk + (t % kWdStages) * kWdKeys;
#pragma unroll
        for (int r = 0; r < kWdItems; ++r) {
          const uint32_t q = r * 32 + lane;
          if (b0 + q < we) cp_async_8(dstk + q, src.key + b0 + q, pol);
        }
      }
      cp_async_commit();
    };
    issue(0);
    __syncwarp();
    for (uint64_t t = 0; t < nsteps; ++t) {
      issue(t + 1);
      cp_async_wait<1>();
      __syncwarp();
      const uint64_t b0 = ws + t * kWdKeys;
      const uint64_t* sk = stk + (t % kWdStages) * kWdKeys;
      uint64_t key[kWdItems];
#pragma unroll
      for (int r = 0; r < kWdItems; ++r) {
        const uint32_t q = r * 32 + lane;
        const uint64_t kv = b0 + q < we ? sk[q] : 0;
        key[r] = src.map_f64 ? f64_to_ordered(kv) : kv;
      }
      uint32_t bk[kWdItems];
      // (never past the sub-chunk: a padding slot's result is discarded)
      classify_batch<kWdItems>(key, bk, [&](int r) {
        const uint64_t pos = b0 + r * 32 + lane;
        if (pos >= we) return 0u;
        return src.idx ? src.idx[pos] : (uint32_t)(pos - sg.start);
      }, sm.sp);
#pragma unroll
      for (int r = 0; r < kWdItems; ++r) {
        const bool v = b0 + r * 32 + lane < we;
        const uint32_t b = v ? bk[r] : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        if (v && lane == __ffs(peers) - 1) row[b] += __popc(peers);
        __syncwarp();
      }
    }
    cp_async_wait<0>();
    __syncwarp();
    for (uint32_t b = lane; b < k; b += 32)
      hist[sg.hist_off + (uint64_t)b * sg.nunits + cl * kPartWarps + warp] = row[b];
  }
}

__global__ void __launch_bounds__(kPartThreads, 3)
k_scatter_wd(const DevState* st, const LevelSeg* segs, Src src, const uint64_t* ssk,
             const uint32_t* ssi, const uint32_t* hist_scan, Dst dst, uint32_t W, uint32_t kmax,
             int unmap_out, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WdSmem sm = carve_wd(smem_raw, kmax, mode);
  const uint64_t pol = l2_evict_first_policy();
  const uint64_t total = st->total_chunks;
  const uint32_t G = st->cur_nseg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t ltmask = lanemask_lt();
  uint32_t* row = sm.rows + (size_t)warp * kmax;
  uint64_t* stk = sm.skey + (size_t)warp * kWdStages * kWdKeys;
  uint32_t* sti = sm.sidx + (size_t)warp * kWdStages * kWdKeys;
  uint32_t cur_g = 0xffffffffu;
  for (uint64_t c = blockIdx.x; c < total; c += gridDim.x) {
    const uint32_t g = find_seg(segs, G, c, [](const LevelSeg& x) { return x.chunk_off; });
    const LevelSeg sg = segs[g];
    __syncthreads();
    if (g != cur_g) {
      load_splitters<kPartThreads>(sg, ssk, ssi, sm.sp);
      cur_g = g;
    }
    const uint32_t k = sg.k;
    const uint64_t cl = c - sg.chunk_off;
    for (uint32_t b = lane; b < k; b += 32)
      row[b] = (uint32_t)(hist_scan[sg.hist_off + (uint64_t)b * sg.nunits + cl * kPartWarps +
                                    warp] + sg.delta);
    const uint64_t cs = sg.start + cl * sg.W;
    const uint64_t ce = umin64(cs + sg.W, sg.start + sg.m);
    uint64_t ws, we;
    warp_subchunk(cs, ce, warp, ws, we);
    const uint64_t nsteps = (we - ws + kWdKeys - 1) / kWdKeys;
    auto issue = [&](uint64_t t) {
      if (t < nsteps) {
        const uint64_t b0 = ws + t * kWdKeys;
        const size_t so = (t % kWdStages) * kWdKeys;
#pragma unroll
        for (int r = 0; r < kWdItems; ++r) {
          const uint32_t q = r * 32 + lane;
          if (b0 + q < we) {
            cp_async_8(stk + so + q, src.key + b0 + q, pol);
            if (src.idx) cp_async_4(sti + so + q, src.idx + b0 + q, pol);
          }
        }
      }
      cp_async_commit();
    };
    issue(0);
    __syncwarp();
    for (uint64_t t = 0; t < nsteps; ++t) {
      issue(t + 1);
      cp_async_wait<1>();
      __syncwarp();
      const uint64_t b0 = ws + t * kWdKeys;
      const size_t so = (t % kWdStages) * kWdKeys;
      uint64_t key[kWdItems];
      uint32_t idx[kWdItems];
#pragma unroll
      for (int r = 0; r < kWdItems; ++r) {
        const uint32_t q = r * 32 + lane;
        const bool v = b0 + q < we;
        const uint64_t kv = v ? stk[so + q] : 0;
        key[r] = src.map_f64 ? f64_to_ordered(kv) : kv;
        idx[r] = v ? (src.idx ? sti[so + q] : (uint32_t)(b0 + q - sg.start)) : 0;
      }
      uint32_t bk[kWdItems];
      classify_batch<kWdItems>(key, bk, [&](int r) { return idx[r]; }, sm.sp);
#pragma unroll
      for (int r = 0; r < kWdItems; ++r) {
        const bool v = b0 + r * 32 + lane < we;
        const uint32_t b = v ? bk[r] : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        const uint32_t c0 = v ? row[b] : 0;
        __syncwarp();
        if (v && lane == __ffs(peers) - 1) row[b] = c0 + __popc(peers);
        __syncwarp();
        if (v) {
          const uint64_t d = (uint64_t)c0 + __popc(peers & ltmask);
          dst.key[d] = unmap_out ? ordered_to_f64(key[r]) : key[r];
          dst.idx[d] = idx[r];
        }
      }
    }
    cp_async_wait<0>();
    __syncwarp();
  }
}

// Level 1 with its order left to the device (LevelParams::stable ==
// kOrderAuto): counts the level's equality buckets, those whose two bounding
// splitters hold one key (every element of such a bucket has that key, so in
// position order it is final and skips the levels below).  The scatter and
// the collect keep input order when they are at least 1/kAutoOrderShare of
// the buckets (duplicate-heavy inputs) and rank by atomics otherwise.
__global__ void __launch_bounds__(256)
k_l1_order(DevState* st, const LevelSeg* segs, const uint64_t* ssk) {
  const uint64_t total = st->total_buckets;
  const uint32_t G = st->cur_nseg;
  uint32_t cnt = 0;
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = find_seg(segs, G, f, [](const LevelSeg& x) { return x.bkt_off; });
    const LevelSeg& sg = segs[g];
    const uint32_t b = (uint32_t)(f - sg.bkt_off);
    if (b >= 1 && b + 1 < sg.k)
      cnt += ssk[sg.samp_off + ((uint64_t)b * sg.S) / sg.k] ==
                     ssk[sg.samp_off + ((uint64_t)(b + 1) * sg.S) / sg.k]
                 ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&st->l1_eq, cnt);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->l1_nb = (uint32_t)umin64(total, 0xffffffffull);
}

// Collect the buckets of the level: bucket sizes follow from the scanned
// histogram.  Buckets that fit one SM, equality buckets of a stable level on
// input in position order (both bounding splitters share one key, so every
// element has that key and the stable scatter left them in position order)
// and empty ones are final; the rest become segments of the next level.
// Otherwise an equality bucket is a bucket like any other, and its elements
// arrive at the in-SM sort in no particular order.
__global__ void __launch_bounds__(256)
k_collect(DevState* st, const LevelSeg* segs, const uint64_t* ssk, const uint32_t* hist_scan,
          SegIn* list_out, int par_out, FinalItem* items, LevelParams P, uint16_t where,
          int last_level, int emit_final, uint64_t* offsets_out) {
  const uint64_t total = st->total_buckets;
  const uint32_t G = st->cur_nseg;
  // buckets keep position order only if the level is stable and its input
  // was in position order (level 1 records this for the levels below)
  const bool stable = P.stable == kOrderAuto ? l1_auto_ordered(st) : P.stable != 0;
  const bool in_order = P.in_order == kOrderAuto ? st->l1_ordered != 0 : P.in_order != 0;
  const bool ordered = stable && in_order;
  if (P.level == 1 && blockIdx.x == 0 && threadIdx.x == 0) st->l1_ordered = ordered ? 1u : 0u;
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = find_seg(segs, G, f, [](const LevelSeg& x) { return x.bkt_off; });
    const LevelSeg& sg = segs[g];
    const uint32_t b = (uint32_t)(f - sg.bkt_off);
    const uint64_t start = hist_scan[sg.hist_off + (uint64_t)b * sg.nunits] + sg.delta;
    const uint64_t end = (b + 1 < sg.k)
                             ? hist_scan[sg.hist_off + (uint64_t)(b + 1) * sg.nunits] + sg.delta
                             : sg.start + sg.m;
    const uint32_t size = (uint32_t)(end - start);
    if (offsets_out) {
      offsets_out[b] = start - sg.start;
      if (b == 0) offsets_out[sg.k] = sg.m;
    }
    if (P.level == 1) atomicMax(&st->max_bucket_l1, size);
    if (!emit_final || size == 0) continue;
    bool eq = false;
    if (ordered && b >= 1 && b + 1 < sg.k) {
      const uint64_t klo = ssk[sg.samp_off + ((uint64_t)b * sg.S) / sg.k];
      const uint64_t khi = ssk[sg.samp_off + ((uint64_t)(b + 1) * sg.S) / sg.k];
      eq = klo == khi;
    }
    if (eq || size <= kBucketCap || last_level) {
      FinalItem it;
      it.start = start;
      it.idx_base = 0;
      it.size = size;
      it.where = where;
      it.kind = (eq || size == 1)      ? kKindCopy
                : size > kBucketCap    ? kKindBig
                : ordered              ? kKindSort
                                       : kKindSortAny;
      if (it.kind == kKindBig) atomicAdd((unsigned long long*)&st->big_items, 1ull);
      push_final(st, items, P.final_cap, it, kErrFinalCap);
    } else {
      SegIn s;
      s.start = start;
      s.m = size;
      s.k_hint = 0;
      const uint32_t slot = atomicAdd(&st->nseg[par_out], 1u);
      if (slot < P.seg_cap) list_out[slot] = s;
      else atomicOr(&st->error, kErrSegCap);
    }
  }
}

// ---------------------------------------------------------------------------
// AMS-sort overpartitioning of a one-segment step (Section 3, AMS-sort;
// Appendix "Implementation Details": b = 2 / ((1 + eps)^(1/l) - 1)).
//
//   k_fine_count    exact sizes of the K = b*k fine partitions of the same
//                   sample (fine splitter j = sorted sample floor(j*S/K)),
//                   counted per CTA in shared memory
//   k_group_*       the smallest load bound L for which the in-order greedy
//                   scan needs at most k groups (candidate bounds checked by
//                   every thread of the GPU per round), then that scan; the
//                   k-1 group boundaries are written after the sample as the
//                   splitters of the ordinary k-way step, and the segment is
//                   pointed at them
// ---------------------------------------------------------------------------
constexpr int kFineThreads = 1024;
constexpr int kFineItems = 4;
constexpr int kGreedyThreads = 1024;

__host__ __device__ inline size_t fine_smem_bytes(uint32_t K) {
  const uint32_t Kp = next_pow2_u32(K);
  return ((size_t)4 << table_bits_for(Kp)) + (size_t)K * (8 + 4 + 4 + 2);
}

__host__ __device__ inline size_t greedy_smem_bytes(uint32_t K, uint32_t k) {
  return (size_t)(K + 1) * 4 + (size_t)(k + 1) * 4 + (size_t)K * 2;
}

__global__ void __launch_bounds__(kFineThreads, 1)
k_fine_count(const LevelSeg* segs, Src src, const uint64_t* ssk, const uint32_t* ssi,
             uint32_t over, int ntb, uint32_t* fine_cnt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LevelSeg sg = segs[0];
  const uint32_t K = sg.k * over;
  // no sample (S = 0, the sample-size rule for k = 1): no fine splitters, so
  // every element counts for fine partition 0
  sg.k = sg.S > 0 ? K : 1;
  Splitters sp;
  sp.mode = 1;
  sp.ntb = ntb;
  sp.tree = nullptr;
  unsigned char* p = smem_raw;
  sp.tbl = (uint32_t*)p;
  p += (size_t)4 << table_bits_for(next_pow2_u32(K));
  sp.key = (uint64_t*)p;
  p += (size_t)K * 8;
  sp.idx = (uint32_t*)p;
  p += (size_t)K * 4;
  uint32_t* cnt = (uint32_t*)p;
  p += (size_t)K * 4;
  sp.rend = (uint16_t*)p;
  load_splitters<kFineThreads>(sg, ssk, ssi, sp);
  for (uint32_t b = threadIdx.x; b < K; b += kFineThreads) cnt[b] = 0;
  __syncthreads();
  constexpr uint64_t kSpan = (uint64_t)kFineThreads * kFineItems;
  const uint64_t m = sg.m;
  for (uint64_t base = (uint64_t)blockIdx.x * kSpan; base < m;
       base += (uint64_t)gridDim.x * kSpan) {
    uint64_t x[kFineItems];
    uint32_t b[kFineItems];
#pragma unroll
    for (int r = 0; r < kFineItems; ++r) {
      const uint64_t q = base + (uint64_t)r * kFineThreads + threadIdx.x;
      x[r] = q < m ? load_key(src, sg.start + q) : 0;
    }
    // level 1 of a one-segment step: the position is the offset in the segment
    classify_batch<kFineItems>(x, b, [&](int r) {
      return (uint32_t)(base + (uint64_t)r * kFineThreads + threadIdx.x);
    }, sp);
#pragma unroll
    for (int r = 0; r < kFineItems; ++r)
      if (base + (uint64_t)r * kFineThreads + threadIdx.x < m) atomicAdd(&cnt[b[r]], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < K; b += kFineThreads)
    if (cnt[b]) atomicAdd(&fine_cnt[b], cnt[b]);
}

// End of the greedy group that starts at fine partition j0: the largest
// j in (j0, K] with P[j] - P[j0] <= L (P: prefix sums, every size <= L).
__device__ __forceinline__ uint32_t greedy_next(const uint32_t* P, uint32_t K, uint32_t j0,
                                                uint64_t L, uint32_t guess) {
  // the group starting at fine partition j0 ends after the last j with
  // P[j] - P[j0] <= L (it takes at least one partition); prefix sums are
  // below 2^32, so the target saturates there
  const uint64_t t64 = (uint64_t)P[j0] + L;
  const uint32_t target = t64 > 0xffffffffull ? 0xffffffffu : (uint32_t)t64;
  const uint32_t first = j0 + 1;
  if (first >= K || P[first] > target) return first;
  // answer in [first, K]: start at the guess and gallop to a bracket a < b
  // with P[a] <= target < P[b] (b = K + 1 stands for "past the end")
  uint32_t g = j0 + guess;
  g = g < first ? first : (g > K ? K : g);
  uint32_t a, b;
  if (P[g] <= target) {
    a = g;
    uint32_t d = 1;
    while (a + d <= K && P[a + d] <= target) {
      a += d;
      d <<= 1;
    }
    b = a + d <= K ? a + d : K + 1;
  } else {
    b = g;
    uint32_t d = 1;
    while (b - first > d && P[b - d] > target) {
      b -= d;
      d <<= 1;
    }
    a = b - first > d ? b - d : first;
  }
  while (b - a > 1) {
    const uint32_t mid = (a + b) >> 1;
    if (P[mid] <= target) a = mid; else b = mid;
  }
  return a;
}

// Groups the greedy scan opens under bound L (stops counting past kmax).
__device__ __forceinline__ uint32_t greedy_count(const uint32_t* P, uint32_t K, uint64_t L,
                                                 uint32_t kmax, uint32_t guess) {
  uint32_t g = 0, j = 0;
  while (j < K && g <= kmax) {
    j = greedy_next(P, K, j, L, guess);
    ++g;
  }
  return g == 0 ? 1 : g;
}

// The greedy's bound L is searched by the whole GPU.  k_group_prep (one CTA)
// writes the prefix sums P of the fine sizes and the first bracket
// [lo, hi] (hi always feasible); every k_group_search launch spreads
// gridDim candidate bounds over the bracket, one per CTA, each checked by a
// greedy scan over P in shared memory; k_group_narrow keeps the sub-bracket
// below the smallest feasible candidate.  Four rounds of 3 CTAs per SM narrow
// any bracket below 2^33 to one value, the smallest feasible bound;
// k_group_finish (one CTA) runs the greedy scan with it.
// search[0] = lo, search[1] = hi, search[2] = smallest feasible candidate index.
constexpr int kSearchThreads = 256;
constexpr int kSearchRounds = 4;

__global__ void __launch_bounds__(kGreedyThreads, 1)
k_group_prep(const LevelSeg* segs, Overpart op) {
  __shared__ uint64_t scan_sm[kGreedyThreads / 32];
  const LevelSeg sg = segs[0];
  const uint32_t k = sg.k, K = k * op.over;
  uint32_t* P = op.prefix;
  const uint32_t tid = threadIdx.x;
  // prefix sums of the fine sizes, one run of fine partitions per thread
  const uint32_t per = (K + kGreedyThreads - 1) / kGreedyThreads;
  const uint32_t j0 = tid * per, j1 = j0 + per < K ? j0 + per : K;
  uint64_t loc = 0, mx = 0;
  for (uint32_t j = j0; j < j1; ++j) {
    const uint64_t c = op.fine_cnt[j];
    loc += c;
    mx = c > mx ? c : mx;
    if (op.fine_out) op.fine_out[j] = c;
  }
  uint64_t n;
  uint64_t run = block_excl_scan_u64<kGreedyThreads>(loc, &n, scan_sm);
  if (tid == 0) P[0] = 0;
  for (uint32_t j = j0; j < j1; ++j) {
    run += op.fine_cnt[j];
    P[j + 1] = (uint32_t)run;  // sums below 2^32
  }
  // largest fine size (max-reduce through the scan scratch)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((tid & 31) == 0) scan_sm[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    uint64_t maxc = 0;
    for (int w = 0; w < kGreedyThreads / 32; ++w) maxc = scan_sm[w] > maxc ? scan_sm[w] : maxc;
    // every group holds at least ceil(n/k) in the worst case and at least the
    // largest fine partition; ceil(n/k) + maxc always needs at most k groups
    const uint64_t avg = (n + k - 1) / k;
    const uint64_t lo = avg > maxc ? avg : maxc;
    op.search[0] = lo;
    op.search[1] = avg + maxc > lo ? avg + maxc : lo;
    op.search[2] = ~0ull;
  }
}

__global__ void __launch_bounds__(kSearchThreads)
k_group_search(const LevelSeg* segs, Overpart op) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint64_t lo = op.search[0], hi = op.search[1];
  if (lo >= hi) return;  // settled (the same for every CTA of this launch)
  const uint32_t k = segs[0].k, K = k * op.over;
  uint32_t* P = (uint32_t*)smem_raw;   // [K + 1]
  uint16_t* nxt = (uint16_t*)(P + K + 1);  // [K]
  for (uint32_t j = threadIdx.x; j <= K; j += kSearchThreads) P[j] = op.prefix[j];
  __syncthreads();
  // this CTA's candidate bound (the last CTA's is hi): the end of the group
  // that would start at every fine partition, in parallel, then one thread
  // counts the groups of the scan from partition 0 by following the links
  const uint64_t t = blockIdx.x, T = gridDim.x;
  const uint64_t L = lo + ((hi - lo) * (t + 1)) / T;
  for (uint32_t j = threadIdx.x; j < K; j += kSearchThreads)
    nxt[j] = (uint16_t)greedy_next(P, K, j, L, op.over);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t g = 0, j = 0;
    while (j < K && g <= k) {
      j = nxt[j];
      ++g;
    }
    if (g <= k) atomicMin((unsigned long long*)&op.search[2], (unsigned long long)t);
  }
}

__global__ void k_group_narrow(Overpart op, uint64_t T) {
  const uint64_t lo = op.search[0], hi = op.search[1];
  if (lo >= hi) return;
  const uint64_t t = op.search[2];  // < T: the candidate hi is feasible
  const uint64_t span = hi - lo;
  op.search[1] = lo + (span * (t + 1)) / T;
  op.search[0] = t == 0 ? lo : lo + (span * t) / T + 1;
  op.search[2] = ~0ull;
}

__global__ void __launch_bounds__(kGreedyThreads, 1)
k_group_finish(LevelSeg* segs, uint64_t* ssk, uint32_t* ssi, Overpart op) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const LevelSeg sg = segs[0];
  const uint32_t k = sg.k, K = k * op.over;
  uint32_t* P = (uint32_t*)smem_raw;                 // [K + 1]
  uint32_t* first = P + K + 1;                       // [k + 1]
  uint16_t* nxt = (uint16_t*)(first + k + 1);        // [K] (K <= kMaxFine < 2^16)
  const uint32_t tid = threadIdx.x;
  for (uint32_t j = tid; j <= K; j += kGreedyThreads) P[j] = op.prefix[j];
  __syncthreads();
  // the end of the group that would start at every fine partition, in
  // parallel; the scan from partition 0 then only follows these links
  const uint64_t L = op.search[1];  // == search[0] once settled; always feasible
  for (uint32_t j = tid; j < K; j += kGreedyThreads)
    nxt[j] = (uint16_t)greedy_next(P, K, j, L, op.over);
  __syncthreads();
  if (tid == 0) {
    uint32_t g = 0, j = 0;
    while (j < K && g < k) {
      first[g++] = j;
      j = nxt[j];
    }
    if (g == 0) first[g++] = 0;
    for (; g <= k; ++g) first[g] = K;
  }
  __syncthreads();
  // group boundaries become the splitters of the k-way step, stored after the
  // sample: entry g (g = 1..k-1) is fine splitter first[g] (an element-free
  // sentinel above every pair when the group is empty and past the end)
  const uint64_t extra = sg.samp_off + sg.S;
  for (uint32_t g = tid + 1; g < k; g += kGreedyThreads) {
    const uint32_t f = first[g];
    uint64_t key = ~0ULL;
    uint32_t idx = ~0u;
    if (f < K) {
      const uint64_t r = ((uint64_t)f * sg.S) / K;
      key = ssk[sg.samp_off + r];
      idx = ssi[sg.samp_off + r];
    }
    ssk[extra + g] = key;
    ssi[extra + g] = idx;
  }
  if (op.first_out)
    for (uint32_t g = tid; g <= k; g += kGreedyThreads) op.first_out[g] = first[g];
  __syncthreads();
  if (tid == 0) {
    segs[0].samp_off = extra;
    segs[0].S = k;
  }
}

// Without overpartitioning the fine partitions are the outputs themselves.
__global__ void k_plain_groups(const uint64_t* offsets, uint32_t k, uint64_t* fine_out,
                               uint32_t* first_out) {
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= k; g += gridDim.x * blockDim.x) {
    if (fine_out && g < k) fine_out[g] = offsets[g + 1] - offsets[g];
    if (first_out) first_out[g] = g;
  }
}

inline int grid_for(uint64_t work, int per_block, int max_blocks) {
  uint64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  return (int)umin64(b, (uint64_t)max_blocks);
}

}  // namespace

namespace {

void launch_overpartition(const LaunchEnv& e, const LevelParams& P, LevelSeg* segs, Src src,
                          uint64_t* ssk, uint32_t* ssi, const Overpart& op) {
  const uint32_t k = op.k, K = op.k * op.over;
  cudaMemsetAsync(op.fine_cnt, 0, (size_t)K * 4, e.stream);
  {
    Scope sc(e, "L1.fine_count");
    k_fine_count<<<e.num_sms, kFineThreads, fine_smem_bytes(K), e.stream>>>(
        segs, src, ssk, ssi, op.over, P.no_tie_break, op.fine_cnt);
  }
  {
    Scope sc(e, "L1.group");
    k_group_prep<<<1, kGreedyThreads, 0, e.stream>>>(segs, op);
    const int grid = e.num_sms * 3;
    for (int r = 0; r < kSearchRounds; ++r) {
      k_group_search<<<grid, kSearchThreads, (size_t)(K + 1) * 4 + (size_t)K * 2, e.stream>>>(
          segs, op);
      k_group_narrow<<<1, 1, 0, e.stream>>>(op, (uint64_t)grid);
    }
    k_group_finish<<<1, kGreedyThreads, greedy_smem_bytes(K, k), e.stream>>>(segs, ssk, ssi,
                                                                               op);
  }
}

}  // namespace

void launch_plain_groups(const LaunchEnv& e, const uint64_t* offsets, uint32_t k,
                         uint64_t* fine_out, uint32_t* first_out) {
  Scope sc(e, "L1.group");
  k_plain_groups<<<(k + 256) / 256, 256, 0, e.stream>>>(offsets, k, fine_out, first_out);
}

void launch_init_plain(const LaunchEnv& e, DevState* st, SegIn* list0, FinalItem* items,
                       uint64_t n, uint32_t k1, int direct, uint64_t final_cap) {
  Scope sc(e, "init");
  k_init_plain<<<1, 32, 0, e.stream>>>(st, list0, items, n, k1, direct, final_cap, e.local);
}

void set_partition_kernel_attributes() {
  cudaFuncSetAttribute(k_sample_sort_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kSampleChunk * kCtaSortBytesPerElem);
  const size_t c = umax64(part_smem_bytes(kMaxK, false, 0), part_smem_bytes(kMaxK, false, 1));
  const size_t s = umax64(part_smem_bytes(kMaxK, true, 0), part_smem_bytes(kMaxK, true, 1));
  cudaFuncSetAttribute(k_classify_count<kCStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)c);
  cudaFuncSetAttribute(k_classify_count<kCStagesDeep>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)umax64(classify_smem_bytes(kMaxKDeep, 0, kCStagesDeep),
                                   classify_smem_bytes(kMaxKDeep, 1, kCStagesDeep)));
  (void)s;
  cudaFuncSetAttribute(k_scatter<kPartThreads, 2048, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)umax64(scatter_smem_bytes(kMaxK, 0, kPartWarps, 2048),
                                   scatter_smem_bytes(kMaxK, 1, kPartWarps, 2048)));
  cudaFuncSetAttribute(k_scatter<kPartThreads, 2048, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)umax64(scatter_smem_bytes(kMaxK, 0, kPartWarps, 2048, false),
                                   scatter_smem_bytes(kMaxK, 1, kPartWarps, 2048, false)));
  {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    size_t limit = 0;
    if (cudaFuncGetAttributes(&fa, k_scatter<512, 4096, true>) == cudaSuccess &&
        (size_t)optin > fa.sharedSizeBytes) {
      limit = (size_t)optin - fa.sharedSizeBytes;
      if (cudaFuncSetAttribute(k_scatter<512, 4096, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)limit) != cudaSuccess ||
          cudaFuncSetAttribute(k_scatter<512, 4096, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)limit) != cudaSuccess)
        limit = 0;
    }
    g_wide_scatter_smem_max = limit;
  }
  cudaFuncSetAttribute(k_fine_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fine_smem_bytes(kMaxFine));
  cudaFuncSetAttribute(k_group_search, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)((kMaxFine + 1) * 4 + kMaxFine * 2));
  cudaFuncSetAttribute(k_group_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)greedy_smem_bytes(kMaxFine, kMaxK));
  cudaGetLastError();  // a refused attribute only disables the variant
  const size_t w = umax64(wd_smem_bytes(kMaxK, 0), wd_smem_bytes(kMaxK, 1));
  cudaFuncSetAttribute(k_classify_count_wd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w);
  cudaFuncSetAttribute(k_scatter_wd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w);
}

int wd_blocks_per_sm(uint32_t kmax, bool scatter, int mode) {
  int nb = 0;
  const size_t smem = wd_smem_bytes(kmax, mode);
  if (scatter)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scatter_wd, kPartThreads, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_classify_count_wd, kPartThreads, smem);
  return nb > 0 ? nb : 1;
}

// Resident CTAs per SM of the classify / scatter kernels for a bucket bound.
int part_blocks_per_sm(uint32_t kmax, bool scatter, int mode, bool stable = true) {
  int nb = 0;
  const size_t smem = part_smem_bytes(kmax, scatter, mode);
  if (scatter && stable)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scatter<kPartThreads, 2048, true>,
                                                  kPartThreads,
                                                  scatter_smem_bytes(kmax, mode, kPartWarps, 2048));
  else if (scatter)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, k_scatter<kPartThreads, 2048, false>, kPartThreads,
        scatter_smem_bytes(kmax, mode, kPartWarps, 2048, false));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_classify_count<kCStages>, kPartThreads,
                                                  smem);
  return nb > 0 ? nb : 1;
}

int classify_deep_blocks_per_sm(uint32_t kmax, int mode) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_classify_count<kCStagesDeep>, kPartThreads,
                                                classify_smem_bytes(kmax, mode, kCStagesDeep));
  return nb > 0 ? nb : 1;
}

int wide_scatter_blocks_per_sm(uint32_t kmax, int mode, bool stable) {
  int nb = 0;
  if (stable)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scatter<512, 4096, true>, 512,
                                                  scatter_smem_bytes(kmax, mode, 16, 4096));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scatter<512, 4096, false>, 512,
                                                  scatter_smem_bytes(kmax, mode, 16, 4096, false));
  return nb > 0 ? nb : 1;
}

// Segmented input: every segment [offsets[s], offsets[s+1]) is checked and
// routed by size: empty ones are skipped, those that fit one CTA go straight
// to the in-SM sort (original positions relative to the segment start), the
// rest become level-1 segments of the sample sort.  Bad offsets raise a
// device error flag instead of being followed.
__global__ void __launch_bounds__(256)
k_init_segments(DevState* st, const uint64_t* offsets, uint32_t nseg, uint64_t n,
                SegIn* list_l1, FinalItem* items, uint64_t seg_cap, uint64_t final_cap) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
       s += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = offsets[s], b = offsets[s + 1];
    if (b < a || b > n || (b - a) > 0xFFFFFFFFull) {
      atomicOr(&st->error, kErrBadOffsets);
      continue;
    }
    const uint64_t m = b - a;
    if (m == 0) continue;
    if (m <= (uint64_t)kBucketCap) {
      FinalItem f;
      f.start = a;
      f.idx_base = a;
      f.size = (uint32_t)m;
      f.where = kWhereInput;
      f.kind = m == 1 ? kKindCopy : kKindSort;
      push_final(st, items, final_cap, f, kErrFinalCap);
    } else {
      SegIn in;
      in.start = a;
      in.m = (uint32_t)m;
      in.k_hint = 0;
      const uint32_t slot = atomicAdd(&st->nseg[1], 1u);
      if (slot < seg_cap) list_l1[slot] = in;
      else atomicOr(&st->error, kErrSegCap);
    }
  }
}

void launch_init_segments(const LaunchEnv& e, DevState* st, const uint64_t* offsets,
                          uint32_t nseg, uint64_t n, SegIn* list_l1, FinalItem* items,
                          uint64_t seg_cap, uint64_t final_cap) {
  Scope sc(e, "init_segments");
  const int grid = (int)umin64((nseg + 255) / 256 + 1, (uint64_t)e.num_sms * 8);
  k_init_segments<<<grid, 256, 0, e.stream>>>(st, offsets, nseg, n, list_l1, items, seg_cap,
                                              final_cap);
}

void launch_level(const LaunchEnv& e, const LevelParams& P, DevState* st, const SegIn* list_in,
                  SegIn* list_out, LevelSeg* segs, Src src, Dst dst, uint16_t dst_where,
                  uint64_t* samp_key, uint32_t* samp_idx, uint64_t* ssamp_key,
                  uint32_t* ssamp_idx, uint32_t* hist, uint32_t* block_sums, FinalItem* items,
                  int kmax_level, int last_level, int emit_final, uint64_t* offsets_out,
                  uint64_t /*n_total*/, int unmap_out, const Overpart* op) {
  const int par_in = P.level & 1;
  const int sms = e.num_sms;
  static const char* kNames[kMaxLevels + 1][11] = {
      {"L?.plan", "L?.sample", "L?.sample_sort", "L?.sample_merge", "L?.classify",
       "L?.scan_reduce", "L?.scan_sums", "L?.scan_down", "L?.scatter", "L?.collect", "L?.order"},
      {"L1.plan", "L1.sample", "L1.sample_sort", "L1.sample_merge", "L1.classify",
       "L1.scan_reduce", "L1.scan_sums", "L1.scan_down", "L1.scatter", "L1.collect", "L1.order"},
      {"L2.plan", "L2.sample", "L2.sample_sort", "L2.sample_merge", "L2.classify",
       "L2.scan_reduce", "L2.scan_sums", "L2.scan_down", "L2.scatter", "L2.collect", "L2.order"},
      {"L3.plan", "L3.sample", "L3.sample_sort", "L3.sample_merge", "L3.classify",
       "L3.scan_reduce", "L3.scan_sums", "L3.scan_down", "L3.scatter", "L3.collect", "L3.order"}};
  const char* const* nm = kNames[(P.level >= 1 && P.level <= kMaxLevels) ? P.level : 0];
  {
    Scope sc(e, nm[0]);
    k_level_plan<<<1, kPlanThreads, 0, e.stream>>>(st, list_in, segs, P, par_in,
                                                  (uint32_t)kmax_level);
  }
  {
    Scope sc(e, nm[1]);
    k_sample<<<grid_for(P.samp_cap, 256, sms * 8), 256, 0, e.stream>>>(st, segs, src, samp_key,
                                                                       samp_idx);
  }
  {
    Scope sc(e, nm[2]);
    const int smem = kSampleChunk * kCtaSortBytesPerElem;
    k_sample_sort_chunks<<<grid_for(P.schunk_cap, 1, sms), kSampleThreads, smem, e.stream>>>(
        st, segs, samp_key, samp_idx, ssamp_key, ssamp_idx, P.in_order);
  }
  {
    Scope sc(e, nm[3]);
    k_sample_merge_rank<<<grid_for(P.samp_cap, 256, sms * 8), 256, 0, e.stream>>>(
        st, segs, samp_key, samp_idx, ssamp_key, ssamp_idx);
  }
  if (op) launch_overpartition(e, P, segs, src, ssamp_key, ssamp_idx, *op);
  const int mode = P.classifier | (P.no_tie_break ? 2 : 0);
  const size_t smem_c = part_smem_bytes((uint32_t)kmax_level, false, mode);
  const size_t smem_s = part_smem_bytes((uint32_t)kmax_level, true, mode);
  // deeper levels take the 2-stage classify when their buckets fit its shared memory
  const bool deep_c = P.level > 1 && (uint32_t)kmax_level <= (uint32_t)kMaxKDeep;
  const size_t smem_cd = classify_smem_bytes((uint32_t)kmax_level, mode, kCStagesDeep);
  const int grid_c = grid_for(
      P.chunk_cap, 1,
      sms * (deep_c ? classify_deep_blocks_per_sm((uint32_t)kmax_level, mode)
                    : part_blocks_per_sm((uint32_t)kmax_level, false, mode)));
  const bool stable = P.stable == 1;
  const int grid_s = grid_for(P.chunk_cap, 1,
                              sms * part_blocks_per_sm((uint32_t)kmax_level, true, mode, stable));
  const size_t smem_wd = wd_smem_bytes((uint32_t)kmax_level, mode);
  const int grid_wd_c =
      grid_for(P.chunk_cap, 1, sms * wd_blocks_per_sm((uint32_t)kmax_level, false, mode));
  const int grid_wd_s =
      grid_for(P.chunk_cap, 1, sms * wd_blocks_per_sm((uint32_t)kmax_level, true, mode));
  const bool wide = !P.warp_direct && kmax_level >= P.wide_scatter_k &&
                    scatter_smem_bytes((uint32_t)kmax_level, mode, 16, 4096, stable) <=
                        g_wide_scatter_smem_max;
  // A stable level with at most kUnitMaxK buckets classifies once, storing
  // every element's bucket id, and scatters whole 8-element units
  // (unit_scatter.cu).  Otherwise stored bucket ids spare the staged scatter
  // its second classification, except in the warp-direct scatter and at
  // 1024+ buckets, where the staged scatter's L2-resident write frontiers
  // were the bottleneck and the extra id stream measured slower.
  // With atomic_scatter, an unordered level (a full sort's levels after the
  // first) keeps the ids of its classify pass and ranks by shared-memory
  // atomics in the small-footprint scatter (measured slower than the staged
  // scatter at 2^28 keys with ~171 buckets per segment; a tuner candidate).
  // (a level that need not keep input order -- a full sort's levels -- has
  // the unit scatter rank by shared-memory atomics)
  const bool units = P.unit_scatter && !P.warp_direct && src.bid != nullptr &&
                     kmax_level > 32 && unit_scatter_fits((uint32_t)kmax_level);
  const bool atomics = !units && P.atomic_scatter && !stable && !P.warp_direct &&
                       src.bid != nullptr && atomic_scatter_fits((uint32_t)kmax_level);
  if (!units && !atomics && (P.warp_direct || kmax_level >= 1024)) src.bid = nullptr;
  // level 1 with its order left to the device: count its equality buckets
  // (without the unit scatter the level stays unordered)
  if (units && P.stable == kOrderAuto) {
    Scope sc(e, nm[10]);
    k_l1_order<<<grid_for(P.bucket_cap, 256, sms * 4), 256, 0, e.stream>>>(st, segs, ssamp_key);
  }
  // Deeper levels keep the staged classify below, which stores the ids as
  // well: with many short chunks it measured faster (1.00 vs 1.09 ms at 2^28
  // keys) than the register-streaming one.
  if (units && P.level == 1) {
    launch_classify_ids(e, P, st, segs, src, ssamp_key, ssamp_idx, hist, (uint32_t)kmax_level,
                        mode, nm[4]);
  } else {
    Scope sc(e, nm[4]);
    if (P.warp_direct)
      k_classify_count_wd<<<grid_wd_c, kPartThreads, smem_wd, e.stream>>>(
          st, segs, src, ssamp_key, ssamp_idx, hist, P.W, (uint32_t)kmax_level, mode);
    else if (deep_c)
      k_classify_count<kCStagesDeep><<<grid_c, kPartThreads, smem_cd, e.stream>>>(
          st, segs, src, ssamp_key, ssamp_idx, hist, P.W, (uint32_t)kmax_level, mode);
    else
      k_classify_count<kCStages><<<grid_c, kPartThreads, smem_c, e.stream>>>(
          st, segs, src, ssamp_key, ssamp_idx, hist, P.W, (uint32_t)kmax_level, mode);
  }
  const int scan_grid = (int)((P.hist_cap + kScanTile - 1) / kScanTile);
  {
    Scope sc(e, nm[5]);
    k_scan_reduce<<<scan_grid > 0 ? scan_grid : 1, 1024, 0, e.stream>>>(st, hist, block_sums);
  }
  {
    Scope sc(e, nm[6]);
    k_scan_sums<<<1, 1024, 0, e.stream>>>(st, block_sums);
  }
  {
    Scope sc(e, nm[7]);
    k_scan_down<<<scan_grid > 0 ? scan_grid : 1, 1024, 0, e.stream>>>(st, hist, block_sums);
  }
  if (units) {
    launch_scatter_units(e, P, st, segs, src, hist, dst, (uint32_t)kmax_level, unmap_out, nm[8]);
  } else if (atomics) {
    launch_scatter_atomic(e, P, st, segs, src, hist, dst, (uint32_t)kmax_level, unmap_out, nm[8]);
  } else {
    Scope sc(e, nm[8]);
    if (P.warp_direct)
      k_scatter_wd<<<grid_wd_s, kPartThreads, smem_wd, e.stream>>>(
          st, segs, src, ssamp_key, ssamp_idx, hist, dst, P.W, (uint32_t)kmax_level, unmap_out,
          mode);
    else if (wide && stable)
      k_scatter<512, 4096, true>
          <<<grid_for(P.chunk_cap, 1,
                      sms * wide_scatter_blocks_per_sm((uint32_t)kmax_level, mode, true)),
             512, scatter_smem_bytes((uint32_t)kmax_level, mode, 16, 4096), e.stream>>>(
              st, segs, src, ssamp_key, ssamp_idx, hist, dst, P.W, (uint32_t)kmax_level,
              unmap_out, mode);
    else if (wide)
      k_scatter<512, 4096, false>
          <<<grid_for(P.chunk_cap, 1,
                      sms * wide_scatter_blocks_per_sm((uint32_t)kmax_level, mode, false)),
             512, scatter_smem_bytes((uint32_t)kmax_level, mode, 16, 4096, false), e.stream>>>(
              st, segs, src, ssamp_key, ssamp_idx, hist, dst, P.W, (uint32_t)kmax_level,
              unmap_out, mode);
    else if (stable)
      k_scatter<kPartThreads, 2048, true>
          <<<grid_s, kPartThreads, scatter_smem_bytes((uint32_t)kmax_level, mode, kPartWarps, 2048),
             e.stream>>>(st, segs, src, ssamp_key, ssamp_idx, hist, dst, P.W,
                         (uint32_t)kmax_level, unmap_out, mode);
    else
      k_scatter<kPartThreads, 2048, false>
          <<<grid_s, kPartThreads,
             scatter_smem_bytes((uint32_t)kmax_level, mode, kPartWarps, 2048, false),
             e.stream>>>(st, segs, src, ssamp_key, ssamp_idx, hist, dst, P.W,
                         (uint32_t)kmax_level, unmap_out, mode);
  }
  {
    Scope sc(e, nm[9]);
    k_collect<<<grid_for(P.bucket_cap, 256, sms * 8), 256, 0, e.stream>>>(
        st, segs, ssamp_key, hist, list_out, par_in ^ 1, items, P, dst_where, last_level,
        emit_final, offsets_out);
  }
}

}  // namespace rsort
