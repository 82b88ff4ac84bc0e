// median_kernels.cu -- the binary-tree median approximation of Section 3
// ("Approximate Median Selection with a Single Reduction") over a whole key
// array, as one CTA reducing the tree level by level through global scratch.
#include "rsort_internal.cuh"
#include "tree_median.cuh"

namespace rsort {

namespace {

constexpr int kTmThreads = 1024;

template <int K>
__global__ void __launch_bounds__(kTmThreads, 1)
k_tree_median(const uint64_t* keys, uint32_t n, int f64, uint64_t seed, uint32_t leaves,
              unsigned char* scratch, uint64_t* out_pos) {
  uint64_t* bk0 = (uint64_t*)scratch;
  uint64_t* bk1 = bk0 + leaves;
  uint32_t* bp0 = (uint32_t*)(bk1 + leaves);
  uint32_t* bp1 = bp0 + leaves;
  uint8_t* bn0 = (uint8_t*)(bp1 + leaves);
  uint8_t* br0 = bn0 + leaves / 2;
  uint8_t* bn1 = br0 + leaves / 2;
  uint8_t* br1 = bn1 + leaves / 2;
  uint64_t key;
  const uint32_t r = cta_tree_median<K, kTmThreads>(
      [&](uint32_t i, uint64_t& k, uint32_t& pos) {
        const uint64_t raw = keys[i];
        k = f64 ? f64_to_ordered(raw) : raw;
        pos = i;
      },
      n, leaves, seed, bk0, bp0, bn0, br0, bk1, bp1, bn1, br1, &key);
  if (threadIdx.x == 0) *out_pos = r;
}

template <int K>
void launch_k(const LaunchEnv& e, const uint64_t* keys, uint32_t n, int f64, uint64_t seed,
              uint32_t leaves, void* scratch, uint64_t* out) {
  k_tree_median<K><<<1, kTmThreads, 0, e.stream>>>(keys, n, f64, seed, leaves,
                                                   (unsigned char*)scratch, out);
}

}  // namespace

size_t tree_median_scratch_bytes(uint64_t n) {
  const uint64_t leaves = next_pow2_u32((uint32_t)(n > 0 ? n : 1));
  return (size_t)leaves * 24 + (size_t)leaves * 2 + 64;
}

bool launch_tree_median(const LaunchEnv& e, const uint64_t* keys, uint32_t n, int f64,
                        uint32_t k, uint64_t seed, void* scratch, uint64_t* out_pos) {
  const uint32_t leaves = next_pow2_u32(n);
  struct Scope {
    const LaunchEnv& e;
    Scope(const LaunchEnv& env) : e(env) {
      if (e.timer) e.timer->begin("tree_median", e.stream);
    }
    ~Scope() {
      if (e.timer) e.timer->end(e.stream);
      if (e.launches) ++*e.launches;
    }
  } sc(e);
  switch (k) {
    case 2: launch_k<2>(e, keys, n, f64, seed, leaves, scratch, out_pos); return true;
    case 4: launch_k<4>(e, keys, n, f64, seed, leaves, scratch, out_pos); return true;
    case 8: launch_k<8>(e, keys, n, f64, seed, leaves, scratch, out_pos); return true;
    case 16: launch_k<16>(e, keys, n, f64, seed, leaves, scratch, out_pos); return true;
    case 32: launch_k<32>(e, keys, n, f64, seed, leaves, scratch, out_pos); return true;
    default: return false;
  }
}

}  // namespace rsort
