// cta_sort.cuh — stable sort of up to kCtaSortMax (key, value) pairs in one thread block.
//
// The multi-pass device-wide radix sort costs two launches and a memset per 8-bit digit, which
// dominates small sorts (the journeys and runs of one stream window: hundreds to a few
// thousand pairs). Here one block loads the pairs into shared memory and runs an LSD radix sort
// there: it first finds which key bits differ between the pairs (an OR and an AND over the
// keys) and runs a counting pass only for the 8-bit digits that hold such a bit; a digit that is
// the same in every key would leave the order unchanged. Each pass ranks a warp's keys by their
// digits' peer lanes (found by one ballot per digit bit, as in the journey kernel's radix sort),
// sums the warps' digit counts in order, and scatters; every pass is stable, so the result is
// the stable order by the key bits [begin_bit, end_bit), equal keys in input order.
#pragma once
#include "common.cuh"

namespace cvetl {

// Two block sizes: 1,024 threads for up to kCtaSortMax pairs, 256 threads for up to a quarter of
// that (a block's fixed per-pass work, zeroing and summing its warps' digit counters, grows with
// its warps). Each thread ranks kCtaSortPer keys per pass.
constexpr int kCtaSortPer = 4;
constexpr int kCtaSortBlock = 1024;
constexpr int kCtaSortBlockSmall = 256;
constexpr uint32_t kCtaSortMax = kCtaSortPer * kCtaSortBlock;
constexpr uint32_t kCtaSortSmallMax = kCtaSortPer * kCtaSortBlockSmall;

static_assert(kCtaSortBlockSmall % 256 == 0 && kCtaSortBlock % 256 == 0, "a thread per digit and group");

// Two key buffers, two value buffers, and the warps' digit counters (uint16, warp-major).
template <typename K, int NT = kCtaSortBlock>
constexpr size_t cta_sort_smem() {
  return (size_t)kCtaSortPer * NT * 2 * (sizeof(K) + 4) + (size_t)(NT / 32) * 256 * 2;
}

// Sorts n <= kCtaSortPer * NT pairs by bits [begin_bit, end_bit) of the key. vin == nullptr means
// value = input position. Launch with one block of NT threads (256 or 1024) and
// cta_sort_smem<K, NT>() bytes of dynamic shared memory.
template <typename K, int NT>
__global__ void __launch_bounds__(NT) k_cta_sort(const K* __restrict__ kin,
                                                             const uint32_t* __restrict__ vin, uint32_t n,
                                                             int begin_bit, int end_bit,
                                                             K* __restrict__ kout,
                                                             uint32_t* __restrict__ vout) {
  constexpr int kWarps = NT / 32;
  constexpr uint32_t kCap = (uint32_t)kCtaSortPer * NT;
  constexpr int kQ = NT / 256;             // groups of warps whose digit counts one thread sums
  constexpr int kWarpsPerQ = kWarps / kQ;  // 8
  extern __shared__ __align__(16) unsigned char smem[];
  K* ka = reinterpret_cast<K*>(smem);
  K* kb = ka + kCap;
  uint32_t* va = reinterpret_cast<uint32_t*>(kb + kCap);
  uint32_t* vb = va + kCap;
  uint16_t* wcnt = reinterpret_cast<uint16_t*>(vb + kCap);  // [warp][digit]
  __shared__ uint32_t qsum[kQ * 256];  // per group of warps and digit: counts, then offsets
  __shared__ uint32_t base[256];       // first output position of each digit
  __shared__ uint32_t scan[NT / 32 + 1];
  __shared__ K s_or, s_and;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int width = end_bit - begin_bit;
  const K mask = width >= (int)(8 * sizeof(K)) ? ~(K)0 : (((K)1 << width) - 1);
  if (tid == 0) {
    s_or = (K)0;
    s_and = ~(K)0;
  }
  __syncthreads();
  K o = (K)0, a = ~(K)0;
  for (uint32_t i = tid; i < n; i += NT) {
    const K k = kin[i];
    ka[i] = k;
    va[i] = vin ? vin[i] : i;
    const K d = (k >> begin_bit) & mask;
    o |= d;
    a &= d;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    o |= __shfl_xor_sync(0xffffffffu, o, s);
    a &= __shfl_xor_sync(0xffffffffu, a, s);
  }
  if (lane == 0) {
    atomicOr(&s_or, o);
    atomicAnd(&s_and, a);
  }
  __syncthreads();
  const K vary = s_or ^ s_and;  // bits that differ between some two keys
  K *src = ka, *dst = kb;
  uint32_t *vs = va, *vd = vb;
  for (int shift = 0; shift < width; shift += 8) {
    if (((vary >> shift) & (K)255) == (K)0) continue;  // uniform digit: the pass keeps the order
    for (int i = tid; i < kWarps * 256 / 2; i += NT) reinterpret_cast<uint32_t*>(wcnt)[i] = 0u;
    __syncthreads();
    // warp w ranks keys [w * 32 * kCtaSortPer, (w + 1) * 32 * kCtaSortPer), 32 at a time in order
    K key[kCtaSortPer];
    uint32_t val[kCtaSortPer], dg[kCtaSortPer], rank[kCtaSortPer];
#pragma unroll
    for (int r = 0; r < kCtaSortPer; ++r) {
      const uint32_t idx = (uint32_t)(warp * 32 * kCtaSortPer + r * 32 + lane);
      const bool in = idx < n;
      key[r] = in ? src[idx] : (K)0;
      val[r] = in ? vs[idx] : 0u;
      const uint32_t d = in ? (uint32_t)((((key[r] >> begin_bit) & mask) >> shift) & (K)255) : 256u;
      const uint32_t peers = match_label<9>(d);  // d <= 256
      const uint32_t before = in ? (uint32_t)wcnt[warp * 256 + d] : 0u;
      __syncwarp();
      if (in && lane == __ffs(peers) - 1) wcnt[warp * 256 + d] = (uint16_t)(before + __popc(peers));
      __syncwarp();
      dg[r] = d;
      rank[r] = before + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    {  // digit d, group q of the warps: exclusive offsets inside the group, group totals
      const int d = tid & 255, q = tid >> 8;
      uint32_t run = 0;
#pragma unroll
      for (int w = q * kWarpsPerQ; w < (q + 1) * kWarpsPerQ; ++w) {
        const uint32_t c = wcnt[w * 256 + d];
        wcnt[w * 256 + d] = (uint16_t)run;
        run += c;
      }
      qsum[q * 256 + d] = run;
    }
    __syncthreads();
    uint32_t tot = 0;
    if (tid < 256) {
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        const uint32_t a = qsum[q * 256 + tid];
        qsum[q * 256 + tid] = tot;
        tot += a;
      }
    }
    const uint32_t e = block_excl_scan<NT>(tot, scan, nullptr);
    if (tid < 256) base[tid] = e;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kCtaSortPer; ++r) {
      if (dg[r] < 256u) {
        const uint32_t d = dg[r];
        const uint32_t p = base[d] + qsum[(warp / kWarpsPerQ) * 256 + d] + wcnt[warp * 256 + d] + rank[r];
        dst[p] = key[r];
        vd[p] = val[r];
      }
    }
    __syncthreads();
    K* tk = src;
    src = dst;
    dst = tk;
    uint32_t* tv = vs;
    vs = vd;
    vd = tv;
  }
  for (uint32_t i = tid; i < n; i += NT) {
    kout[i] = src[i];
    vout[i] = vs[i];
  }
}

}  // namespace cvetl
