// cta_sort.cuh — stable sort of up to kCtaSortMax (key, value) pairs in one thread block.
//
// The multi-pass device-wide radix sort costs two launches and a memset per 8-bit digit, which
// dominates small sorts (the journeys and runs of one stream window: hundreds to a few
// thousand pairs). Here one block loads the pairs into shared memory, pads to a power of two
// and runs a bitonic network on (key bits [begin_bit, end_bit), input position): positions are
// distinct, so the network yields exactly the stable order, then writes keys and values out.
// The network does O(n log^2 n) work on one SM: above a few thousand pairs the device-wide sort
// is faster, hence the limit.
#pragma once
#include "common.cuh"

namespace cvetl {

constexpr uint32_t kCtaSortMax = 2048;
constexpr int kCtaSortBlock = 1024;

template <typename K>
constexpr size_t cta_sort_smem() {
  return (size_t)kCtaSortMax * (sizeof(K) + 4);
}

// Sorts n <= kCtaSortMax pairs by bits [begin_bit, end_bit) of the key. vin == nullptr means
// value = input position. Launch with one block of kCtaSortBlock threads and
// cta_sort_smem<K>() bytes of dynamic shared memory.
template <typename K>
__global__ void __launch_bounds__(kCtaSortBlock) k_cta_sort(const K* __restrict__ kin,
                                                             const uint32_t* __restrict__ vin, uint32_t n,
                                                             int begin_bit, int end_bit,
                                                             K* __restrict__ kout,
                                                             uint32_t* __restrict__ vout) {
  extern __shared__ __align__(16) unsigned char smem[];
  K* sk = reinterpret_cast<K*>(smem);
  uint32_t* sp = reinterpret_cast<uint32_t*>(sk + kCtaSortMax);
  const uint32_t N = n < 2 ? 2u : (1u << (32 - __clz(n - 1)));
  const int width = end_bit - begin_bit;
  const K mask = width >= (int)(8 * sizeof(K)) ? ~(K)0 : (((K)1 << width) - 1);
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
    sk[i] = i < n ? kin[i] : (K)0;
    sp[i] = i;
  }
  __syncthreads();
  // a < b in (padding last, key bits, position)
  auto less = [&](K ka, uint32_t pa, K kb, uint32_t pb) {
    if (pa >= n) return false;
    if (pb >= n) return true;
    const K a = (ka >> begin_bit) & mask, b = (kb >> begin_bit) & mask;
    return a < b || (a == b && pa < pb);
  };
  for (uint32_t k = 2; k <= N; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
        const uint32_t l = i ^ j;
        if (l <= i) continue;
        const K ka = sk[i], kb = sk[l];
        const uint32_t pa = sp[i], pb = sp[l];
        const bool up = (i & k) == 0;
        if (up ? less(kb, pb, ka, pa) : less(ka, pa, kb, pb)) {
          sk[i] = kb;
          sk[l] = ka;
          sp[i] = pb;
          sp[l] = pa;
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    kout[i] = sk[i];
    vout[i] = vin ? vin[sp[i]] : sp[i];
  }
}

}  // namespace cvetl
