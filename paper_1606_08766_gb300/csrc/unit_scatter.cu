// unit_scatter.cu -- the classify and scatter passes of a stable partition
// level (the data exchange of Appendix "Robust Multi-Level Sample Sort",
// MPI_Alltoallv in the paper, a stable scatter through HBM here) with the
// bucket of every element computed once and its output written in whole
// sectors.
//
// k_classify_ids   classifies every element of a chunk once (splitters in
//                  shared memory, the same classifiers as every other level)
//                  and stores its bucket id (16 bits) beside the per-chunk
//                  bucket histogram.  Keys stream through 16-byte loads (two
//                  keys each) straight into registers.
//
// k_scatter_units  reads keys and stored bucket ids of 4096-element sub-tiles
//                  (registers, the next sub-tile's loads in flight while the
//                  current one is processed), ranks every element among the
//                  elements of its bucket (warp order, then lane order: input
//                  order, so buckets keep input order), counting-sorts the
//                  sub-tile into shared memory, and writes every bucket's run
//                  in whole UNITS of 8 elements -- 64 bytes of keys and 32
//                  bytes of positions, aligned in the output -- each stored by
//                  8 consecutive lanes of one warp instruction, so every output
//                  sector is written whole and once.  A bucket's incomplete
//                  last unit (at most 7 elements) waits in a per-bucket carry
//                  area in shared memory and goes out with the bucket's next
//                  elements.  Only the first and last unit of a bucket in a
//                  chunk, shared with the neighbouring chunks' ranges, are
//                  written in part.
//
// The carry area holds 7 (key, position) slots per bucket, so the scatter
// serves levels with at most kUnitMaxK buckets.
#include "async_copy.cuh"
#include "bulk_copy.cuh"
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

constexpr int kUnit = 8;    // elements per output unit
constexpr int kCarry = 7;   // carry slots per bucket (kUnit - 1)

// Streaming loads of data read once: no L1 allocation, L2 evict-first.
__device__ __forceinline__ void ld_stream_v2(uint64_t& a, uint64_t& b, const uint64_t* p,
                                             uint64_t pol) {
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
      : "=l"(a), "=l"(b)
      : "l"(p), "l"(pol));
}
__device__ __forceinline__ uint64_t ld_stream_u64(const uint64_t* p, uint64_t pol) {
  uint64_t v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ld_stream_u16(const uint16_t* p, uint64_t pol) {
  unsigned short v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return v;
}

// Key bits as the level stores them: conv 1 maps float64 patterns to the
// order map, 2 maps them back, 0 leaves them.
__device__ __forceinline__ uint64_t conv_key(uint64_t k, int conv) {
  return conv == 1 ? f64_to_ordered(k) : (conv == 2 ? ordered_to_f64(k) : k);
}

// ---------------------------------------------------------------------------
// Classify with stored bucket ids
// ---------------------------------------------------------------------------
constexpr int kCiPairs = 4;  // 16-byte loads (two keys) per thread per step
// steps ahead of the current one whose keys are asked into L2 (0 or 1: none;
// the next step's keys are already in registers)
constexpr int kCiPrefetch = 2;

// VEC: the key array is 16-byte aligned (pairs are read by 16-byte loads);
// MAP: the keys are float64 bit patterns, mapped to the order map on load.
template <int NT, bool VEC, bool MAP>
__global__ void __launch_bounds__(NT, 3)
k_classify_ids(const DevState* st, const LevelSeg* segs, Src src, const uint64_t* ssk,
               const uint32_t* ssi, uint32_t* hist, uint32_t kmax, int mode) {
  constexpr int R = 2 * kCiPairs;  // keys per thread per step
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Splitters sp;
  uint32_t* cnt;
  {
    unsigned char* p = smem_raw;
    const size_t Kp = next_pow2_u32(kmax);
    sp.mode = mode & 1;
    sp.ntb = (mode >> 1) & 1;
    sp.tree = nullptr;
    sp.tbl = nullptr;
    if (sp.mode == 0) {
      sp.tree = (uint64_t*)p;
      p += Kp * 8;
    } else {
      sp.tbl = (uint32_t*)p;
      p += (size_t)4 << table_bits_for((uint32_t)Kp);
    }
    sp.key = (uint64_t*)p; p += (size_t)kmax * 8;
    sp.idx = (uint32_t*)p; p += (size_t)kmax * 4;
    cnt = (uint32_t*)p; p += (size_t)kmax * 4;
    sp.rend = (uint16_t*)p;
  }
  const uint64_t pol = l2_evict_first_policy();
  const uint64_t total = st->total_chunks;
  const uint32_t G = st->cur_nseg;
  const int lane = threadIdx.x & 31;
  uint32_t cur_g = 0xffffffffu;
  for (uint64_t c = blockIdx.x; c < total; c += gridDim.x) {
    const uint32_t g = find_seg(segs, G, c, [](const LevelSeg& x) { return x.chunk_off; });
    const LevelSeg sg = segs[g];
    __syncthreads();
    if (g != cur_g) {
      load_splitters<NT>(sg, ssk, ssi, sp);
      cur_g = g;
    }
    for (uint32_t b = threadIdx.x; b < sg.k; b += NT) cnt[b] = 0;
    __syncthreads();
    const uint64_t cl = c - sg.chunk_off;
    const uint64_t cs = sg.start + cl * sg.W;
    const uint64_t ce = umin64(cs + sg.W, sg.start + sg.m);
    // pairs start at the even position at or below cs (16-byte aligned when
    // the key array is).  VEC: every pair wholly before ce is read by one
    // 16-byte load, from a position clamped into that range (pairs past it
    // read a valid pair and discard it), so the loop has no load branch; an
    // odd chunk end's last key is handled after the loop.  Otherwise every
    // key is read by its own checked load.
    const uint64_t ps = cs & ~1ull;
    const uint64_t npairs = VEC ? (ce - ps) >> 1 : (ce - ps + 1) >> 1;
    auto load = [&](uint64_t p0, uint64_t (&x)[R]) {
#pragma unroll
      for (int r = 0; r < kCiPairs; ++r) {
        const uint64_t j = p0 + (uint64_t)r * NT + threadIdx.x;
        if constexpr (VEC) {
          uint64_t a, b;
          ld_stream_v2(a, b, src.key + ps + 2 * (j < npairs ? j : npairs - 1), pol);
          x[2 * r] = j < npairs ? a : 0;
          x[2 * r + 1] = j < npairs ? b : 0;
        } else {
          const uint64_t pos = ps + 2 * j;
          x[2 * r] = x[2 * r + 1] = 0;
          if (j < npairs) {
            x[2 * r] = ld_stream_u64(src.key + pos, pol);
            if (pos + 1 < ce) x[2 * r + 1] = ld_stream_u64(src.key + pos + 1, pol);
          }
        }
      }
    };
    // one thread asks L2 for the keys of the step starting at pair p0
    auto prefetch = [&](uint64_t p0) {
      if (kCiPrefetch < 2 || threadIdx.x != 0 || p0 >= npairs) return;
      const uint64_t a = umax64(ps + 2 * p0, cs);
      const uint64_t e = umin64(ps + 2 * (p0 + (uint64_t)NT * kCiPairs), ce);
      prefetch_l2_range(src.key + a, src.key + e);
    };
    for (int d = 2; d < kCiPrefetch; ++d) prefetch((uint64_t)d * NT * kCiPairs);
    uint64_t x[R], xn[R];
    if (npairs > 0) load(0, x);
    for (uint64_t p0 = 0; p0 < npairs; p0 += (uint64_t)NT * kCiPairs) {
      prefetch(p0 + (uint64_t)kCiPrefetch * NT * kCiPairs);
      load(p0 + (uint64_t)NT * kCiPairs, xn);
      uint64_t key[R];
#pragma unroll
      for (int e = 0; e < R; ++e) key[e] = MAP ? f64_to_ordered(x[e]) : x[e];
      uint32_t bk[R];
      // positions are read only on a key tie, and only inside the chunk (a
      // padding slot's result is discarded)
      // (each thread's elements come in pairs of consecutive positions)
      auto pos_at = [&](int e) {
        return ps + 2 * (p0 + (uint64_t)(e >> 1) * NT + threadIdx.x) + (e & 1);
      };
      auto valid = [&](int e) {
        const uint64_t pos = pos_at(e);
        return (p0 + (uint64_t)(e >> 1) * NT + threadIdx.x) < npairs && pos >= cs && pos < ce;
      };
      classify_batch_pairs<R>(key, bk, [&](int e) {
        if (!valid(e)) return 0u;
        const uint64_t pos = pos_at(e);
        return src.idx ? src.idx[pos] : (uint32_t)(pos - sg.start);
      }, [&](int e) { return valid(e) && src.idx == nullptr; }, sp);
      // a step whose pairs all lie inside the chunk stores them whole
      const bool whole = ps == cs && p0 + (uint64_t)NT * kCiPairs <= npairs &&
                         ps + 2 * (p0 + (uint64_t)NT * kCiPairs) <= ce;
      // runs of one bucket across the warp (duplicate-heavy inputs) take one
      // atomic per warp and slot; otherwise one atomic per key
      const uint32_t b0 = __shfl_sync(0xffffffffu, bk[0], 0);
      const bool skewed = __popc(__ballot_sync(0xffffffffu, bk[0] == b0)) > 8;
      uint32_t vmask = 0;  // valid elements of the step
#pragma unroll
      for (int r = 0; r < kCiPairs; ++r) {
        const uint64_t j = p0 + (uint64_t)r * NT + threadIdx.x;
        const uint64_t pos = ps + 2 * j;
        const bool v0 = whole || (j < npairs && pos >= cs && pos < ce);
        const bool v1 = whole || (j < npairs && pos + 1 < ce);
        if (whole || (v0 && v1)) {
          *reinterpret_cast<uint32_t*>(src.bid + pos) = bk[2 * r] | (bk[2 * r + 1] << 16);
        } else if (v0) {
          src.bid[pos] = (uint16_t)bk[2 * r];
        } else if (v1) {
          src.bid[pos + 1] = (uint16_t)bk[2 * r + 1];
        }
        vmask |= ((v0 ? 1u : 0u) | (v1 ? 2u : 0u)) << (2 * r);
      }
      if (!skewed) {
#pragma unroll
        for (int e = 0; e < R; ++e)
          if ((vmask >> e) & 1u) atomicAdd(&cnt[bk[e]], 1u);
      } else {
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const bool v = (vmask >> e) & 1u;
          const uint32_t bl = __shfl_sync(0xffffffffu, bk[e], 0);
          if (__all_sync(0xffffffffu, v && bk[e] == bl)) {
            if (lane == 0) atomicAdd(&cnt[bl], 32u);
          } else if (v) {
            atomicAdd(&cnt[bk[e]], 1u);
          }
        }
      }
#pragma unroll
      for (int e = 0; e < R; ++e) x[e] = xn[e];
    }
    // VEC: an odd chunk end's last key (the pair it starts would read one key
    // past the chunk)
    if (VEC && threadIdx.x == 0 && ((ce - ps) & 1) && ce - 1 >= cs) {
      const uint64_t pos = ce - 1;
      const uint64_t raw = ld_stream_u64(src.key + pos, pol);
      uint64_t k1[1] = {MAP ? f64_to_ordered(raw) : raw};
      uint32_t b1[1];
      classify_batch<1>(k1, b1, [&](int) {
        return src.idx ? src.idx[pos] : (uint32_t)(pos - sg.start);
      }, sp);
      src.bid[pos] = (uint16_t)b1[0];
      atomicAdd(&cnt[b1[0]], 1u);
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < sg.k; b += NT)
      hist[sg.hist_off + (uint64_t)b * sg.nunits + cl] = cnt[b];
  }
}

// ---------------------------------------------------------------------------
// The same classify pass with its keys staged by bulk copies: one thread
// keeps a ring of kCbStages shared-memory stages of kCbStageKeys keys filled
// through the tensor memory accelerator (cp.async.bulk, completed on one
// mbarrier per stage), running ahead across the CTA's chunks, so every SM
// has up to 2 x 4 x 16 KB of loads in flight without holding registers for
// them.  A stage starts at an even position (16-byte aligned when the key
// array is) and ends at an even one; a chunk's odd last key is read directly.
// ---------------------------------------------------------------------------
constexpr int kCbStageKeys = 2048;
constexpr int kCbStages = 4;

__host__ __device__ inline size_t classify_bulk_smem_bytes(size_t common) {
  return ((common + 127) & ~(size_t)127) + (size_t)kCbStages * kCbStageKeys * 8 +
         (size_t)kCbStages * 16;
}

// Warp-specialised: NC consumer threads classify, one producer warp (the
// last) streams the stages.  Per stage a "full" barrier (one arrival with the
// expected bytes) and an "empty" barrier (one arrival per consumer warp);
// there is no block barrier inside a chunk.  Every wait is bounded: a wait
// that gives up raises kErrWait, the CTA drains its copies and returns.
template <int NC>
__global__ void __launch_bounds__(NC + 32, 2)
k_classify_bulk(DevState* st, const LevelSeg* segs, Src src, const uint64_t* ssk,
                const uint32_t* ssi, uint32_t* hist, uint32_t kmax, int mode, size_t common) {
  constexpr int NT = NC + 32;
  constexpr int NCW = NC / 32;         // consumer warps
  constexpr int SK = kCbStageKeys;
  constexpr int NST = kCbStages;
  constexpr int PER = SK / (2 * NC);   // key pairs per consumer thread per stage
  constexpr int R = 2 * PER;
  static_assert(PER * 2 * NC == SK, "a stage is whole pairs per consumer thread");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Splitters sp;
  uint32_t* cnt;
  {
    unsigned char* p = smem_raw;
    const size_t Kp = next_pow2_u32(kmax);
    sp.mode = mode & 1;
    sp.ntb = (mode >> 1) & 1;
    sp.tree = nullptr;
    sp.tbl = nullptr;
    if (sp.mode == 0) {
      sp.tree = (uint64_t*)p;
      p += Kp * 8;
    } else {
      sp.tbl = (uint32_t*)p;
      p += (size_t)4 << table_bits_for((uint32_t)Kp);
    }
    sp.key = (uint64_t*)p; p += (size_t)kmax * 8;
    sp.idx = (uint32_t*)p; p += (size_t)kmax * 4;
    cnt = (uint32_t*)p; p += (size_t)kmax * 4;
    sp.rend = (uint16_t*)p;
  }
  uint64_t* stage = (uint64_t*)(smem_raw + ((common + 127) & ~(size_t)127));
  uint64_t* full = stage + (size_t)NST * SK;
  uint64_t* empty = full + NST;
  __shared__ uint32_t s_abort;
  const uint64_t pol = l2_evict_first_policy();
  const uint64_t total = st->total_chunks;
  const uint32_t G = st->cur_nseg;
  const uint32_t tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const bool producer = warp == NCW;
  if (tid == 0) {
    for (int b = 0; b < NST; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], NCW);
    }
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  uint32_t next = 0;   // stages issued (producer) / consumed (consumers) so far
  uint32_t cur_g = 0xffffffffu;
  for (uint64_t c = blockIdx.x; c < total; c += gridDim.x) {
    const uint32_t g = find_seg(segs, G, c, [](const LevelSeg& x) { return x.chunk_off; });
    const LevelSeg sg = segs[g];
    if (__syncthreads_or(s_abort != 0)) break;
    if (g != cur_g) {
      load_splitters<NT>(sg, ssk, ssi, sp);
      cur_g = g;
    }
    for (uint32_t b = tid; b < sg.k; b += NT) cnt[b] = 0;
    __syncthreads();
    const uint64_t cl = c - sg.chunk_off;
    const uint64_t cs = sg.start + cl * sg.W;
    const uint64_t ce = umin64(cs + sg.W, sg.start + sg.m);
    const uint64_t ps = cs & ~1ull, pe = ce & ~1ull;
    const uint32_t nstg = pe > ps ? (uint32_t)((pe - ps + SK - 1) / SK) : 0u;
    if (producer) {
      if (lane == 0) {
        for (uint32_t s = 0; s < nstg; ++s, ++next) {
          const uint32_t buf = next % NST, use = next / NST;
          if (use > 0 && !mbar_wait_bounded(&empty[buf], (use - 1) & 1u, kBulkWaitPolls)) {
            atomicOr(&s_abort, 1u);
            break;
          }
          const uint64_t a = ps + (uint64_t)s * SK;
          const uint64_t b = umin64(a + SK, pe);
          fence_proxy_async_smem();
          bulk_copy_g2s(stage + (size_t)buf * SK, src.key + a, (uint32_t)((b - a) * 8),
                        &full[buf], pol);
        }
      }
      next = __shfl_sync(0xffffffffu, next, 0);
    } else {
      auto count = [&](bool v, uint32_t b) {
        const uint32_t bl = __shfl_sync(0xffffffffu, b, 0);
        if (__all_sync(0xffffffffu, v && b == bl)) {
          if (lane == 0) atomicAdd(&cnt[bl], 32u);
        } else if (v) {
          atomicAdd(&cnt[b], 1u);
        }
      };
      for (uint32_t s = 0; s < nstg; ++s, ++next) {
        const uint32_t buf = next % NST, use = next / NST;
        const bool ok = mbar_wait_bounded(&full[buf], use & 1u, kBulkWaitPolls);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lane == 0) atomicOr(&s_abort, 1u);
          break;
        }
        const uint64_t a = ps + (uint64_t)s * SK;
        const uint64_t b = umin64(a + SK, pe);
        const uint64_t* stg = stage + (size_t)buf * SK;
        uint64_t key[R];
#pragma unroll
        for (int r = 0; r < PER; ++r) {
          const uint32_t j = r * NC + tid;
          key[2 * r] = key[2 * r + 1] = 0;
          if (a + 2 * j < b) {
            const uint4 v = *reinterpret_cast<const uint4*>(stg + 2 * j);
            key[2 * r] = ((uint64_t)v.y << 32) | v.x;
            key[2 * r + 1] = ((uint64_t)v.w << 32) | v.z;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[buf]);  // this warp is done with the stage
#pragma unroll
        for (int e = 0; e < R; ++e) key[e] = src.map_f64 ? f64_to_ordered(key[e]) : key[e];
        uint32_t bk[R];
        classify_batch<R>(key, bk, [&](int e) {
          const uint64_t pos = a + 2 * ((uint64_t)(e >> 1) * NC + tid) + (e & 1);
          if (pos < cs || pos >= ce) return 0u;
          return src.idx ? src.idx[pos] : (uint32_t)(pos - sg.start);
        }, sp);
#pragma unroll
        for (int r = 0; r < PER; ++r) {
          const uint64_t pos = a + 2 * ((uint64_t)r * NC + tid);
          const bool v0 = pos < b && pos >= cs;
          const bool v1 = pos + 1 < b;
          if (v0 && v1) {
            *reinterpret_cast<uint32_t*>(src.bid + pos) = bk[2 * r] | (bk[2 * r + 1] << 16);
          } else if (v1) {
            src.bid[pos + 1] = (uint16_t)bk[2 * r + 1];
          }
          count(v0, bk[2 * r]);
          count(v1, bk[2 * r + 1]);
        }
      }
      // the consumer warps agree on the stage count (an abort ends them early)
    }
    __syncthreads();
    if (s_abort) break;
    // an odd chunk end: its last key is read directly
    if ((ce & 1) && ce - 1 >= cs && tid == 0) {
      uint64_t x[1] = {load_key(src, ce - 1)};
      uint32_t bk[1];
      classify_batch<1>(x, bk, [&](int) {
        return src.idx ? src.idx[ce - 1] : (uint32_t)(ce - 1 - sg.start);
      }, sp);
      src.bid[ce - 1] = (uint16_t)bk[0];
      atomicAdd(&cnt[bk[0]], 1u);
    }
    __syncthreads();
    for (uint32_t b = tid; b < sg.k; b += NT)
      hist[sg.hist_off + (uint64_t)b * sg.nunits + cl] = cnt[b];
  }
  __syncthreads();
  if (s_abort) {
    if (tid == 0) atomicOr(&st->error, kErrWait);
    // copies still in flight must land before the CTA's shared memory goes:
    // the producer waits for the phases of the last stages it issued (a
    // landed one answers at once)
    if (producer && lane == 0) {
      const uint32_t from = next > (uint32_t)NST ? next - NST : 0u;
      for (uint32_t i = from; i < next; ++i)
        mbar_wait_bounded(&full[i % NST], (i / NST) & 1u, kBulkWaitPolls);
    }
  }
}

// ---------------------------------------------------------------------------
// Scatter in whole units
// ---------------------------------------------------------------------------
// The stable scatter keeps per-warp counters and winner slots (512 threads,
// 4096-element sub-tiles); the unordered one needs one counter per bucket,
// and the room that frees holds longer sub-tiles (more elements per thread).
constexpr int kUsThreads = 512;        // stable
constexpr int kUsItems = 8;
constexpr int kUsThreadsAny = 512;     // unordered (6144-element sub-tiles)
constexpr int kUsItemsAny = 12;
// sub-tiles ahead whose bytes are asked into L2 when a sub-tile starts (0:
// none): with 1, the next sub-tile's register loads, issued after this one's
// placement, find their bytes on the way (measured at 2^28 keys: distance 1
// 2.23 -> 2.08 ms, 2 -> 2.12, 3 -> 2.18)
constexpr int kUsPrefetch = 1;
// a bucket with at most this many whole units in a sub-tile writes their
// records itself; more (skewed inputs) send the sub-tile through the unit
// marks and a block max-scan instead
constexpr int kUsDirectUnits = 16;
// bits of the per-bucket meta word
constexpr int kMetaUnitShift = 14;     // sorted slot + 8 below (14 bits)
constexpr int kMetaCarryShift = 25;    // first unit (11 bits) below
constexpr int kMetaPhShift = 28;       // carry count (3 bits) below, phantoms (3 bits)
// bits of the second word of a per-unit record (the first is the output
// position of the unit's slot 0)
constexpr int kRecFirstShift = 14;     // sorted slot of slot 0 + 8 (14 bits) below
constexpr int kRecBucketShift = 20;    // carry count, phantoms (3 + 3 bits) below

__host__ __device__ inline uint32_t us_max_units(uint32_t kmax, uint32_t st) {
  return (st + kCarry * kmax) / kUnit + 1;
}

__host__ __device__ inline size_t us_smem_bytes(uint32_t kmax, uint32_t nt, uint32_t it,
                                                bool stable) {
  const uint32_t nw = nt / 32, st = nt * it;
  size_t b = 0;
  b += (size_t)st * 8;                           // sorted keys
  b += (size_t)kmax * kCarry * 8;                // carried keys
  b += (size_t)us_max_units(kmax, st) * 8;       // per-unit records
  b += (size_t)st * 4;                           // sorted positions
  b += (size_t)kmax * kCarry * 4;                // carried positions
  b += (size_t)kmax * 8;                         // per-bucket obase + meta
  b += (size_t)(kmax + 1) * 4;                   // sbase
  b += stable ? (size_t)nw * cnt_stride(kmax) * 2 : (size_t)kmax * 4;  // counters
  b += (size_t)us_max_units(kmax, st) * 2 + 2;   // unit -> bucket
  b += stable ? (size_t)nw * kmax : 0;           // per-warp winner slots
  return (b + 15) & ~(size_t)15;
}

// Exclusive max-scan of one u32 per thread over the block (NT % 32 == 0);
// sm holds NT/32 words.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_max_u32(uint32_t v, uint32_t* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = max(x, y);
  }
  if (lane == 31) sm[w] = x;
  __syncthreads();
  uint32_t pre = 0;
  for (int q = 0; q < w; ++q) pre = max(pre, sm[q]);
  const uint32_t y = __shfl_up_sync(0xffffffffu, x, 1);
  const uint32_t excl = max(pre, lane > 0 ? y : 0u);
  __syncthreads();
  return excl;
}

// Ranks every valid element (bucket id != 0xffffffff) of a thread's IT among
// the elements of its bucket in the sub-tile, in no particular order, by
// shared-memory atomics on the bucket counters cnt.  Atomics on one word
// serialise, so runs of one bucket (duplicate-heavy inputs, where the copies
// of a key fill a bucket by position) are ranked per warp: a warp whose
// whole window lies in one bucket takes one atomic; a window where lane 0's
// bucket holds more than 8 lanes of the first round takes one atomic per
// distinct bucket and round; otherwise every element takes its own.
template <int IT>
__device__ __forceinline__ void rank_by_atomics(const uint32_t (&bid)[IT], uint32_t (&rank)[IT],
                                                uint32_t* cnt, int lane, uint32_t ltmask) {
  const uint32_t b0 = __shfl_sync(0xffffffffu, bid[0], 0);
  bool same = b0 != 0xffffffffu;
#pragma unroll
  for (int r = 0; r < IT; ++r) same = same && bid[r] == b0;
  if (__all_sync(0xffffffffu, same)) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&cnt[b0], 32u * IT);
    base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
    for (int r = 0; r < IT; ++r) rank[r] = base + r * 32 + lane;
  } else if (__popc(__ballot_sync(0xffffffffu, bid[0] == b0)) > 8) {
#pragma unroll
    for (int r = 0; r < IT; ++r) {
      const uint32_t b = bid[r];
      const uint32_t peers = __match_any_sync(0xffffffffu, b);
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if (b != 0xffffffffu && lane == leader) base = atomicAdd(&cnt[b], __popc(peers));
      rank[r] = __shfl_sync(0xffffffffu, base, leader) + __popc(peers & ltmask);
    }
  } else {
#pragma unroll
    for (int r = 0; r < IT; ++r)
      if (bid[r] != 0xffffffffu) rank[r] = atomicAdd(&cnt[bid[r]], 1u);
  }
}

// HAS_IDX: the level reads stored positions (deeper levels); otherwise the
// position is implicit (level 1: offset in the segment).
// STABLE: elements of a bucket keep input order (ranks from per-warp counters
// and a prefix over the warps); otherwise (a full sort's level 1, whose
// buckets the in-SM sort orders by (key, position) anyway) every element takes
// its rank from one shared-memory atomic on its bucket's counter.
// auto_order: level 1 with its order decided on the device; the kernel
// returns at once unless the decision (l1_auto_ordered) is its own form.
template <int NT, int IT, bool HAS_IDX, bool STABLE>
__global__ void __launch_bounds__(NT, 1)
k_scatter_units(const DevState* st, const LevelSeg* segs, Src src, const uint32_t* hist_scan,
                Dst dst, uint32_t kmax, int conv, uint32_t aoff, bool auto_order) {
  if (auto_order && l1_auto_ordered(st) != STABLE) return;
  constexpr int NW = NT / 32;
  constexpr int ST = NT * IT;
  static_assert(ST + kUnit < (1 << kMetaUnitShift), "sorted slots fit the meta word");
  static_assert(((ST + kCarry * kUnitMaxK) / kUnit) < (1 << (kMetaCarryShift - kMetaUnitShift)),
                "unit indices fit the meta word");
  static_assert(ST + kUnit < (1 << kRecFirstShift) && kUnitMaxK <= (1 << (32 - kRecBucketShift)),
                "sorted slots and buckets fit the unit record");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* p = smem_raw;
  uint64_t* skey = (uint64_t*)p; p += (size_t)ST * 8;
  uint64_t* ckey = (uint64_t*)p; p += (size_t)kmax * kCarry * 8;
  const uint32_t umax = us_max_units(kmax, ST);
  // per whole unit of the sub-tile: its output position, and the sorted slot
  // of its slot 0 + 8 | (carry count | phantoms << 3) << 14 | bucket << 20
  // (carry count and phantoms only in a bucket's first unit)
  uint2* urec = (uint2*)p; p += (size_t)umax * 8;
  uint32_t* sidx = (uint32_t*)p; p += (size_t)ST * 4;
  uint32_t* cidx = (uint32_t*)p; p += (size_t)kmax * kCarry * 4;
  // per-bucket state (two flat word arrays, so that both the bucket-ordered
  // and the interleaved phases touch consecutive words):
  //   obase  output position of the bucket's current unit start (mod 2^32)
  //   meta   sorted slot of that unit's first slot + 8 (14 bits; the unit
  //          may begin with up to 7 carried slots) | first unit in the unit
  //          list << 14 (11 bits) | carry count << 25 | phantoms << 28
  uint32_t* obase = (uint32_t*)p; p += (size_t)kmax * 4;
  uint32_t* meta = (uint32_t*)p; p += (size_t)kmax * 4;
  uint32_t* sbase = (uint32_t*)p; p += (size_t)(kmax + 1) * 4;
  const uint32_t kst = cnt_stride(kmax);
  uint16_t* wcnt = (uint16_t*)p;
  p += STABLE ? (size_t)NW * kst * 2 : (size_t)kmax * 4;
  uint16_t* unit_b = (uint16_t*)p; p += (size_t)umax * 2 + 2;
  uint8_t* wwin = (uint8_t*)p;
  __shared__ uint64_t scan_sm[NW];
  __shared__ uint32_t max_sm[NW];
  __shared__ uint32_t s_big;  // some bucket has more than kUsDirectUnits units
  if (threadIdx.x == 0) s_big = 0;

  const uint64_t pol = l2_evict_first_policy();
  const uint64_t total = st->total_chunks;
  const uint32_t G = st->cur_nseg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t tid = threadIdx.x;
  const uint32_t ltmask = lanemask_lt();
  uint16_t* my_cnt = wcnt + (size_t)warp * kst;
  uint8_t* my_win = wwin + (size_t)warp * kmax;
  uint32_t* ucnt = reinterpret_cast<uint32_t*>(wcnt);  // unordered: one counter per bucket
  for (uint32_t u = tid; u < umax; u += NT) unit_b[u] = 0;
  if (!STABLE)
    for (uint32_t b = tid; b < kmax; b += NT) ucnt[b] = 0;

  for (uint64_t c = blockIdx.x; c < total; c += gridDim.x) {
    const uint32_t g = find_seg(segs, G, c, [](const LevelSeg& x) { return x.chunk_off; });
    const LevelSeg sg = segs[g];
    const uint32_t k = sg.k;
    const int nbits = k > 32 ? 5 : (int)ceil_log2_dev(k);
    const uint64_t cl = c - sg.chunk_off;
    const uint64_t cs = sg.start + cl * sg.W;
    const uint64_t ce = umin64(cs + sg.W, sg.start + sg.m);
    const uint64_t nst = (ce - cs + ST - 1) / ST;
    // buckets handled by this thread in the per-bucket phases
    const uint32_t per = (k + NT - 1) / NT;
    const uint32_t bb0 = min(tid * per, k);
    const uint32_t bb1 = min(bb0 + per, k);
    __syncthreads();  // the previous chunk is done with every shared array
    // output state of every bucket: the chunk's first position p0, the unit
    // start at or below it (units start at positions = aoff mod 8) and the
    // slots before p0 in that unit (phantoms: held, never written)
    for (uint32_t b = tid; b < k; b += NT) {
      const uint32_t p0 = (uint32_t)(hist_scan[sg.hist_off + (uint64_t)b * sg.nunits + cl] +
                                     sg.delta);
      const uint32_t a = (p0 - aoff) & (kUnit - 1);
      obase[b] = p0 - a;
      meta[b] = (a << kMetaCarryShift) | (a << kMetaPhShift);
    }
    const uint32_t q0 = (uint32_t)warp * (IT * 32) + lane;
    uint64_t key[IT];
    uint32_t idx[IT], bid[IT];
    auto load = [&](uint64_t s, uint64_t (&kk)[IT], uint32_t (&ii)[IT], uint32_t (&bb)[IT]) {
      const uint64_t b0 = cs + s * ST;
#pragma unroll
      for (int r = 0; r < IT; ++r) {
        const uint64_t pos = b0 + q0 + r * 32;
        kk[r] = 0;
        ii[r] = 0;
        bb[r] = 0xffffffffu;
        if (s < nst && pos < ce) {
          kk[r] = ld_stream_u64(src.key + pos, pol);
          if (HAS_IDX) ii[r] = ld_stream_u32(src.idx + pos, pol);
          bb[r] = ld_stream_u16(src.bid + pos, pol);
        }
      }
    };
    // one thread asks L2 for sub-tile s's keys, positions and bucket ids
    auto prefetch = [&](uint64_t s) {
      if (kUsPrefetch == 0 || tid != 0 || s >= nst) return;
      const uint64_t a = cs + s * ST, e = umin64(a + ST, ce);
      prefetch_l2_range(src.key + a, src.key + e);
      if (HAS_IDX) prefetch_l2_range(src.idx + a, src.idx + e);
      prefetch_l2_range(src.bid + a, src.bid + e);
    };
    for (int d = 1; d < kUsPrefetch; ++d) prefetch(d);
    load(0, key, idx, bid);
    for (uint64_t s = 0; s < nst; ++s) {
      prefetch(s + kUsPrefetch);
      // -- 1. rank every element among its bucket's elements of this warp
      //    (stable: earlier rounds, then lower lanes), or of the sub-tile
      //    (unordered: a shared-memory atomic)
      uint32_t lrank[IT];
      if constexpr (!STABLE) {
        rank_by_atomics<IT>(bid, lrank, ucnt, lane, ltmask);
      } else {
      for (uint32_t q = lane; q < (k + 1) / 2; q += 32) ((uint32_t*)my_cnt)[q] = 0;
      __syncwarp();
      // a warp whose whole window lies in one bucket (runs of copies of a
      // key) ranks its elements by their place in the window
      const uint32_t b0 = __shfl_sync(0xffffffffu, bid[0], 0);
      bool same = b0 != 0xffffffffu;
#pragma unroll
      for (int r = 0; r < IT; ++r) same = same && bid[r] == b0;
      if (__all_sync(0xffffffffu, same)) {
#pragma unroll
        for (int r = 0; r < IT; ++r) lrank[r] = r * 32 + lane;
        if (lane == 0) my_cnt[b0] = (uint16_t)(32 * IT);
        __syncwarp();
      } else {
#pragma unroll
      for (int r = 0; r < IT; ++r) {
        const uint32_t b = bid[r];
        const bool v = b != 0xffffffffu;
        // peers = the lanes holding the same bucket: up to 32 buckets by
        // ballots over the bucket bits; beyond, every lane writes its lane id
        // to the warp's slot of its bucket and the id that stayed there (one
        // per distinct bucket) is compared instead
        uint32_t w = b;
        if (k > 32) {
          if (v) my_win[b] = (uint8_t)lane;
          __syncwarp();
          w = v ? my_win[b] : 0u;
          __syncwarp();
        }
        uint32_t peers = __ballot_sync(0xffffffffu, v);
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
      }  // mixed window
      }  // STABLE
      __syncthreads();  // (A) every warp's counts are in
      // -- 2. per bucket: exclusive prefix over the warps' counts (in place),
      //    the bucket's elements t in this sub-tile, its virtual run
      //    (carry + t) and the whole units u of that run; then one block scan
      //    of (u, t) places every bucket's elements in the sorted sub-tile and
      //    its units in the unit list, and a bucket with few units writes
      //    their records
      uint32_t loc_t = 0, loc_u = 0;
      if constexpr (!STABLE) {
        for (uint32_t b = bb0; b < bb1; ++b) {
          const uint32_t t = ucnt[b];
          ucnt[b] = 0;  // ready for the next sub-tile (its atomics follow barriers)
          const uint32_t u = (((meta[b] >> kMetaCarryShift) & 7u) + t) / kUnit;
          sbase[b] = t | (u << 16);
          loc_t += t;
          loc_u += u;
        }
      } else {
        uint32_t b = bb0;
        for (; (per & 1) == 0 && b + 1 < bb1; b += 2) {
          uint32_t tot2 = 0;
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            uint32_t* cw = reinterpret_cast<uint32_t*>(wcnt + (size_t)w * kst + b);
            const uint32_t cnt2 = *cw;
            *cw = tot2;
            tot2 = __vadd2(tot2, cnt2);
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t t = h ? (tot2 >> 16) : (tot2 & 0xffffu);
            const uint32_t u = (((meta[b + h] >> kMetaCarryShift) & 7u) + t) / kUnit;
            sbase[b + h] = t | (u << 16);
            loc_t += t;
            loc_u += u;
          }
        }
        for (; b < bb1; ++b) {
          uint32_t t = 0;
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            const uint32_t cnt = wcnt[(size_t)w * kst + b];
            wcnt[(size_t)w * kst + b] = (uint16_t)t;
            t += cnt;
          }
          const uint32_t u = (((meta[b] >> kMetaCarryShift) & 7u) + t) / kUnit;
          sbase[b] = t | (u << 16);
          loc_t += t;
          loc_u += u;
        }
      }
      uint64_t tot;
      const uint64_t ex =
          block_excl_scan_u64<NT>(((uint64_t)loc_u << 32) | loc_t, &tot, scan_sm);
      {
        uint32_t run_t = (uint32_t)ex, run_u = (uint32_t)(ex >> 32);
        bool big = false;
        for (uint32_t b = bb0; b < bb1; ++b) {
          const uint32_t tu = sbase[b], t = tu & 0xffffu, u = tu >> 16;
          const uint32_t m = meta[b];
          const uint32_t cb = (m >> kMetaCarryShift) & 7u;
          sbase[b] = run_t;
          meta[b] = (m & (0x3fu << kMetaCarryShift)) | (run_u << kMetaUnitShift) |
                    (run_t + kUnit - cb);
          if (u > (uint32_t)kUsDirectUnits) {
            big = true;
          } else if (u) {
            const uint32_t ob = obase[b];
            const uint32_t qv = run_t + kUnit - cb;
            urec[run_u] = make_uint2(ob, qv | (((m >> kMetaCarryShift) & 0x3fu) << kRecFirstShift) |
                                             (b << kRecBucketShift));
            for (uint32_t d = 1; d < u; ++d)
              urec[run_u + d] = make_uint2(ob + kUnit * d, (qv + kUnit * d) | (b << kRecBucketShift));
          }
          run_t += t;
          run_u += u;
        }
        if (big) s_big = 1u;
      }
      const uint32_t U = (uint32_t)(tot >> 32);
      if (tid == 0) sbase[k] = (uint32_t)tot;
      __syncthreads();  // (B) bucket bases and unit marks are in
      // -- 3. if a bucket had too many units to write their records: the
      //    bucket of every unit (marks carry bucket + 1 at a bucket's first
      //    unit; an inclusive max-scan fills the rest) and every unit's record
      //    (the marks are cleared for the next sub-tile); then the sub-tile
      //    counting-sorted by bucket into shared memory
      if (s_big) {
        for (uint32_t b = bb0; b < bb1; ++b) {
          const uint32_t m = meta[b];
          const uint32_t uu = (((m >> kMetaCarryShift) & 7u) + sbase[b + 1] - sbase[b]) / kUnit;
          if (uu) unit_b[(m >> kMetaUnitShift) & 0x7ffu] = (uint16_t)(b + 1);
        }
        __syncthreads();
        const uint32_t upt = (U + NT - 1) / NT;
        const uint32_t u0 = min(tid * upt, U), u1 = min(u0 + upt, U);
        uint32_t m = 0;
        for (uint32_t u = u0; u < u1; ++u) m = max(m, (uint32_t)unit_b[u]);
        uint32_t run = block_excl_max_u32<NT>(m, max_sm);
        for (uint32_t u = u0; u < u1; ++u) {
          run = max(run, (uint32_t)unit_b[u]);
          unit_b[u] = 0;
          const uint32_t b = run - 1, mb = meta[b];
          const uint32_t d = u - ((mb >> kMetaUnitShift) & 0x7ffu);  // unit of the bucket's run
          const uint32_t first = d == 0 ? (mb >> kMetaCarryShift) & 0x3fu : 0u;
          urec[u] = make_uint2(obase[b] + kUnit * d,
                               ((mb & ((1u << kMetaUnitShift) - 1)) + kUnit * d) |
                                   (first << kRecFirstShift) | (b << kRecBucketShift));
        }
      }
      const uint32_t pos0 = (uint32_t)(cs + s * ST - sg.start) + q0;  // implicit positions
#pragma unroll
      for (int r = 0; r < IT; ++r) {
        const uint32_t b = bid[r];
        if (b != 0xffffffffu) {
          const uint32_t q = sbase[b] + (STABLE ? (uint32_t)my_cnt[b] : 0u) + lrank[r];
          skey[q] = conv_key(key[r], conv);
          sidx[q] = HAS_IDX ? idx[r] : pos0 + r * 32;
        }
      }
      __syncthreads();  // (C) the sorted sub-tile and the unit buckets are in
      if (tid == 0) s_big = 0;
      // the next sub-tile's loads go out now, into the same registers, and
      // land while this one is written
      load(s + 1, key, idx, bid);
      // -- 4. whole units out: 8 consecutive lanes store one unit (slots
      //    before the carry count come from the carry area, phantoms are
      //    skipped); one record lookup per slot
      for (uint32_t e = tid; e < U * kUnit; e += NT) {
        const uint32_t u = e / kUnit, j = e % kUnit;
        const uint2 rc = urec[u];
        const uint32_t cb = (rc.y >> kRecFirstShift) & 7u;
        const uint32_t ph = (rc.y >> (kRecFirstShift + 3)) & 7u;
        uint64_t kv;
        uint32_t iv;
        if (j < cb) {
          const uint32_t cq = (rc.y >> kRecBucketShift) * kCarry + j;
          kv = ckey[cq];
          iv = cidx[cq];
        } else {
          const uint32_t q = (rc.y & ((1u << kRecFirstShift) - 1)) - kUnit + j;
          kv = skey[q];
          iv = sidx[q];
        }
        if (j >= ph) {
          dst.key[rc.x + j] = kv;
          dst.idx[rc.x + j] = iv;
        }
      }
      __syncthreads();  // (D) carry slots are read
      // -- 5. the incomplete last unit of every bucket becomes its carry
      //    (buckets interleaved over the threads, so that neighbouring lanes
      //    touch neighbouring carry rows; copies unrolled and predicated)
      for (uint32_t b = tid; b < k; b += NT) {
        const uint32_t m = meta[b];
        const uint32_t cb = (m >> kMetaCarryShift) & 7u;
        const uint32_t qb = (m & ((1u << kMetaUnitShift) - 1)) - kUnit;  // sorted slot of run slot 0
        const uint32_t L = cb + (sbase[b + 1] - sbase[b]), u = L / kUnit, nc = L % kUnit;
        // run slots [first, L) become carry slots [first - shift, L - shift)
        const uint32_t first = u == 0 ? cb : kUnit * u;
        const uint32_t shift = kUnit * u;
        {
          uint64_t ck[kCarry];
#pragma unroll
          for (int j = 0; j < kCarry; ++j)
            if (first + j < L) ck[j] = skey[qb + first + j];
#pragma unroll
          for (int j = 0; j < kCarry; ++j)
            if (first + j < L) ckey[b * kCarry + first + j - shift] = ck[j];
        }
        {
          uint32_t ci[kCarry];
#pragma unroll
          for (int j = 0; j < kCarry; ++j)
            if (first + j < L) ci[j] = sidx[qb + first + j];
#pragma unroll
          for (int j = 0; j < kCarry; ++j)
            if (first + j < L) cidx[b * kCarry + first + j - shift] = ci[j];
        }
        const uint32_t ph = u == 0 ? ((m >> kMetaPhShift) & 7u) : 0u;
        obase[b] += shift;
        meta[b] = (nc << kMetaCarryShift) | (ph << kMetaPhShift);
      }
    }
    // the chunk's last, incomplete unit of every bucket (the rest of its
    // sectors belongs to the next chunk's range)
    for (uint32_t b = tid; b < k; b += NT) {
      const uint32_t m = meta[b], ob = obase[b];
      const uint32_t cb = (m >> kMetaCarryShift) & 7u, ph = (m >> kMetaPhShift) & 7u;
      for (uint32_t j = ph; j < cb; ++j) {
        dst.key[ob + j] = ckey[b * kCarry + j];
        dst.idx[ob + j] = cidx[b * kCarry + j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Scatter of an unordered level (a full sort's levels after the first): the
// in-SM sort orders (key, position) pairs, so elements of a bucket may leave
// in any order.  Every element takes its rank from one shared-memory atomic
// on its bucket's counter -- no per-warp tables, no carries (a bucket's run
// per sub-tile is long at these fan-outs) -- so the kernel is small enough
// for several CTAs per SM to hide each other's latency.
// ---------------------------------------------------------------------------
constexpr int kSaThreads = 256;
constexpr int kSaItems = 8;
constexpr int kSaTile = kSaThreads * kSaItems;  // 2048 elements per sub-tile

__host__ __device__ inline size_t sa_smem_bytes(uint32_t kmax) {
  return (size_t)kSaTile * (8 + 4 + 2) + (size_t)kmax * 12;
}

template <int NT, bool HAS_IDX>
__global__ void __launch_bounds__(NT, 4)
k_scatter_atomic(const DevState* st, const LevelSeg* segs, Src src, const uint32_t* hist_scan,
                 Dst dst, uint32_t kmax, int conv) {
  constexpr int IT = kSaItems;
  constexpr int ST = NT * IT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* p = smem_raw;
  uint64_t* skey = (uint64_t*)p; p += (size_t)ST * 8;
  uint32_t* sidx = (uint32_t*)p; p += (size_t)ST * 4;
  uint32_t* cnt = (uint32_t*)p; p += (size_t)kmax * 4;    // counts, then rank bases
  uint32_t* opos = (uint32_t*)p; p += (size_t)kmax * 4;   // running output position
  uint32_t* dlt = (uint32_t*)p; p += (size_t)kmax * 4;    // output position - sorted slot
  uint16_t* sb = (uint16_t*)p;                            // bucket of every sorted slot
  __shared__ uint64_t scan_sm[NT / 32];
  const uint64_t pol = l2_evict_first_policy();
  const uint64_t pol_keep = l2_evict_last_policy();
  const uint64_t total = st->total_chunks;
  const uint32_t G = st->cur_nseg;
  const uint32_t tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const uint32_t q0 = (uint32_t)warp * (IT * 32) + lane;
  for (uint64_t c = blockIdx.x; c < total; c += gridDim.x) {
    const uint32_t g = find_seg(segs, G, c, [](const LevelSeg& x) { return x.chunk_off; });
    const LevelSeg sg = segs[g];
    const uint32_t k = sg.k;
    const uint64_t cl = c - sg.chunk_off;
    const uint64_t cs = sg.start + cl * sg.W;
    const uint64_t ce = umin64(cs + sg.W, sg.start + sg.m);
    const uint32_t per = (k + NT - 1) / NT;
    const uint32_t bb0 = min(tid * per, k), bb1 = min(bb0 + per, k);
    __syncthreads();  // the previous chunk is done with every shared array
    for (uint32_t b = tid; b < k; b += NT) {
      opos[b] = (uint32_t)(hist_scan[sg.hist_off + (uint64_t)b * sg.nunits + cl] + sg.delta);
      cnt[b] = 0;
    }
    for (uint64_t b0 = cs; b0 < ce; b0 += ST) {
      const uint32_t len = (uint32_t)umin64(ST, ce - b0);
      uint64_t key[IT];
      uint32_t idx[IT], bid[IT], rank[IT];
#pragma unroll
      for (int r = 0; r < IT; ++r) {
        const uint32_t q = q0 + r * 32;
        bid[r] = 0xffffffffu;
        if (q < len) {
          key[r] = ld_stream_u64(src.key + b0 + q, pol);
          idx[r] = HAS_IDX ? ld_stream_u32(src.idx + b0 + q, pol)
                           : (uint32_t)(b0 + q - sg.start);
          bid[r] = ld_stream_u16(src.bid + b0 + q, pol);
        }
      }
      __syncthreads();  // (A) counters cleared, previous sub-tile written out
      rank_by_atomics<IT>(bid, rank, cnt, lane, lanemask_lt());
      __syncthreads();  // (B) counts complete
      {
        uint32_t loc = 0;
        for (uint32_t b = bb0; b < bb1; ++b) loc += cnt[b];
        uint64_t tot;
        uint32_t run = (uint32_t)block_excl_scan_u64<NT>(loc, &tot, scan_sm);
        for (uint32_t b = bb0; b < bb1; ++b) {
          const uint32_t t = cnt[b];
          cnt[b] = run;                    // rank base of the bucket in the sub-tile
          dlt[b] = opos[b] - run;          // modulo 2^32: positions are below 2^32
          opos[b] += t;
          run += t;
        }
      }
      __syncthreads();  // (C) bases in place
#pragma unroll
      for (int r = 0; r < IT; ++r) {
        const uint32_t b = bid[r];
        if (b != 0xffffffffu) {
          const uint32_t q = cnt[b] + rank[r];
          skey[q] = conv_key(key[r], conv);
          sidx[q] = idx[r];
          sb[q] = (uint16_t)b;
        }
      }
      __syncthreads();  // (D) sub-tile sorted by bucket
      // runs of ~m/k elements per bucket: the sectors at their ends are
      // completed by the next sub-tile, so the stores ask the L2 to keep
      // them until then
      for (uint32_t q = tid; q < len; q += NT) {
        const uint32_t d = dlt[sb[q]] + q;
        st_keep_u64(dst.key + d, skey[q], pol_keep);
        st_keep_u32(dst.idx + d, sidx[q], pol_keep);
      }
      // counters back to zero for the next sub-tile (bases are no longer read)
      __syncthreads();
      for (uint32_t b = bb0; b < bb1; ++b) cnt[b] = 0;
    }
  }
}

// Dynamic shared memory limit of the unit scatter (0 until set or if refused).
size_t g_us_smem_max = 0;

}  // namespace

size_t classify_ids_smem_bytes(uint32_t kmax, int mode) {
  const size_t Kp = next_pow2_u32(kmax);
  size_t b = (mode & 1) == 0 ? Kp * 8 : ((size_t)4 << table_bits_for((uint32_t)Kp));
  b += (size_t)kmax * (8 + 4 + 4 + 2);
  return (b + 15) & ~(size_t)15;
}

bool unit_scatter_fits(uint32_t kmax) {
  return kmax <= (uint32_t)kUnitMaxK &&
         us_smem_bytes(kmax, kUsThreads, kUsItems, true) <= g_us_smem_max &&
         us_smem_bytes(kmax, kUsThreadsAny, kUsItemsAny, false) <= g_us_smem_max;
}

void set_unit_scatter_attributes() {
  const int ci_smem = (int)umax64(classify_ids_smem_bytes(kMaxK, 0),
                                  classify_ids_smem_bytes(kMaxK, 1));
  cudaFuncSetAttribute(k_classify_ids<256, true, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, ci_smem);
  cudaFuncSetAttribute(k_classify_ids<256, true, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, ci_smem);
  cudaFuncSetAttribute(k_classify_ids<256, false, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, ci_smem);
  cudaFuncSetAttribute(k_classify_ids<256, false, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, ci_smem);
  cudaFuncSetAttribute(k_classify_bulk<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)classify_bulk_smem_bytes(umax64(classify_ids_smem_bytes(kMaxK, 0),
                                                            classify_ids_smem_bytes(kMaxK, 1))));
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  size_t limit = 0;
  if (cudaFuncGetAttributes(&fa, k_scatter_units<kUsThreads, kUsItems, true, true>) == cudaSuccess &&
      (size_t)optin > fa.sharedSizeBytes) {
    limit = (size_t)optin - fa.sharedSizeBytes;
    const size_t need = umax64(us_smem_bytes(kUnitMaxK, kUsThreads, kUsItems, true),
                               us_smem_bytes(kUnitMaxK, kUsThreadsAny, kUsItemsAny, false));
    if (limit > need) limit = need;
    if (cudaFuncSetAttribute(k_scatter_units<kUsThreads, kUsItems, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)limit) != cudaSuccess ||
        cudaFuncSetAttribute(k_scatter_units<kUsThreads, kUsItems, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)limit) != cudaSuccess ||
        cudaFuncSetAttribute(k_scatter_units<kUsThreadsAny, kUsItemsAny, true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)limit) != cudaSuccess ||
        cudaFuncSetAttribute(k_scatter_units<kUsThreadsAny, kUsItemsAny, false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)limit) != cudaSuccess)
      limit = 0;
  }
  g_us_smem_max = limit;
  cudaFuncSetAttribute(k_scatter_atomic<kSaThreads, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa_smem_bytes(kMaxK));
  cudaFuncSetAttribute(k_scatter_atomic<kSaThreads, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa_smem_bytes(kMaxK));
  cudaGetLastError();
}

void launch_classify_ids(const LaunchEnv& e, const LevelParams& P, DevState* st,
                         const LevelSeg* segs, Src src, const uint64_t* ssk, const uint32_t* ssi,
                         uint32_t* hist, uint32_t kmax, int mode, const char* name) {
  if (P.bulk_classify && ((uintptr_t)src.key & 15) == 0) {
    // keys staged by bulk copies (needs a 16-byte aligned key array)
    const size_t common = classify_ids_smem_bytes(kmax, mode);
    const size_t smem = classify_bulk_smem_bytes(common);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_classify_bulk<256>, 256 + 32, smem);
    if (nb < 1) nb = 1;
    const uint64_t grid = umin64(P.chunk_cap, (uint64_t)e.num_sms * nb);
    Scope sc(e, name);
    k_classify_bulk<256><<<(int)(grid ? grid : 1), 256 + 32, smem, e.stream>>>(
        st, segs, src, ssk, ssi, hist, kmax, mode, common);
    return;
  }
  const size_t smem = classify_ids_smem_bytes(kmax, mode);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_classify_ids<256, true, false>, 256,
                                                smem);
  if (nb < 1) nb = 1;
  const uint64_t grid = umin64(P.chunk_cap, (uint64_t)e.num_sms * nb);
  // 16-byte pair loads need a 16-byte aligned key array
  const int vec = ((uintptr_t)src.key & 15) == 0;
  Scope sc(e, name);
  const int g = (int)(grid ? grid : 1);
  if (vec && src.map_f64)
    k_classify_ids<256, true, true><<<g, 256, smem, e.stream>>>(st, segs, src, ssk, ssi, hist,
                                                                kmax, mode);
  else if (vec)
    k_classify_ids<256, true, false><<<g, 256, smem, e.stream>>>(st, segs, src, ssk, ssi, hist,
                                                                 kmax, mode);
  else if (src.map_f64)
    k_classify_ids<256, false, true><<<g, 256, smem, e.stream>>>(st, segs, src, ssk, ssi, hist,
                                                                 kmax, mode);
  else
    k_classify_ids<256, false, false><<<g, 256, smem, e.stream>>>(st, segs, src, ssk, ssi, hist,
                                                                  kmax, mode);
}

void launch_scatter_atomic(const LaunchEnv& e, const LevelParams& P, DevState* st,
                           const LevelSeg* segs, Src src, const uint32_t* hist_scan, Dst dst,
                           uint32_t kmax, int unmap_out, const char* name) {
  const int conv = (src.map_f64 && !unmap_out) ? 1 : ((!src.map_f64 && unmap_out) ? 2 : 0);
  const size_t smem = sa_smem_bytes(kmax);
  int nb = 0;
  if (src.idx)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scatter_atomic<kSaThreads, true>,
                                                  kSaThreads, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scatter_atomic<kSaThreads, false>,
                                                  kSaThreads, smem);
  if (nb < 1) nb = 1;
  const uint64_t grid = umin64(P.chunk_cap, (uint64_t)e.num_sms * nb);
  Scope sc(e, name);
  if (src.idx)
    k_scatter_atomic<kSaThreads, true><<<(int)(grid ? grid : 1), kSaThreads, smem, e.stream>>>(
        st, segs, src, hist_scan, dst, kmax, conv);
  else
    k_scatter_atomic<kSaThreads, false><<<(int)(grid ? grid : 1), kSaThreads, smem, e.stream>>>(
        st, segs, src, hist_scan, dst, kmax, conv);
}

bool atomic_scatter_fits(uint32_t kmax) {
  return kmax <= (uint32_t)kMaxK && sa_smem_bytes(kmax) <= sa_smem_bytes(kMaxK);
}

void launch_scatter_units(const LaunchEnv& e, const LevelParams& P, DevState* st,
                          const LevelSeg* segs, Src src, const uint32_t* hist_scan, Dst dst,
                          uint32_t kmax, int unmap_out, const char* name) {
  const int conv = (src.map_f64 && !unmap_out) ? 1 : ((!src.map_f64 && unmap_out) ? 2 : 0);
  // units start where the output key address is 64-byte aligned
  const uint32_t aoff = (uint32_t)(((64 - ((uintptr_t)dst.key & 63)) & 63) / 8);
  const uint64_t grid = umin64(P.chunk_cap, (uint64_t)e.num_sms);
  Scope sc(e, name);
  const int g = (int)(grid ? grid : 1);
  const size_t smem_s = us_smem_bytes(kmax, kUsThreads, kUsItems, true);
  const size_t smem_a = us_smem_bytes(kmax, kUsThreadsAny, kUsItemsAny, false);
  const bool autoo = P.stable == kOrderAuto;
  if (P.stable == 1 || autoo) {
    if (src.idx)
      k_scatter_units<kUsThreads, kUsItems, true, true><<<g, kUsThreads, smem_s, e.stream>>>(
          st, segs, src, hist_scan, dst, kmax, conv, aoff, autoo);
    else
      k_scatter_units<kUsThreads, kUsItems, false, true><<<g, kUsThreads, smem_s, e.stream>>>(
          st, segs, src, hist_scan, dst, kmax, conv, aoff, autoo);
  }
  // with the order left to the device both forms launch; the one not chosen
  // returns at once
  if (autoo && e.launches) ++*e.launches;
  if (P.stable != 1 || autoo) {
    if (src.idx)
      k_scatter_units<kUsThreadsAny, kUsItemsAny, true, false>
          <<<g, kUsThreadsAny, smem_a, e.stream>>>(st, segs, src, hist_scan, dst, kmax, conv,
                                                   aoff, autoo);
    else
      k_scatter_units<kUsThreadsAny, kUsItemsAny, false, false>
          <<<g, kUsThreadsAny, smem_a, e.stream>>>(st, segs, src, hist_scan, dst, kmax, conv,
                                                   aoff, autoo);
  }
}

}  // namespace rsort
