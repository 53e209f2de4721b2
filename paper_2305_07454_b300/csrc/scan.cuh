// scan.cuh — exclusive prefix sum of uint32 counts (reduce tiles, scan tile sums, apply).
#pragma once
#include "common.cuh"

namespace cvetl {
namespace scan {

constexpr int kBlock = 256;
constexpr int kRounds = 16;
constexpr int kTile = kBlock * kRounds;

// n_dev != nullptr (all three passes): the count is read from device memory, n is the upper
// bound the grid covers.
__global__ void __launch_bounds__(kBlock) k_tile_sums(const uint32_t* __restrict__ in, uint32_t n,
                                                      uint32_t* __restrict__ sums,
                                                      const uint32_t* __restrict__ n_dev) {
  __shared__ uint32_t scratch[kBlock / 32];
  if (n_dev) n = min(n, *n_dev);
  uint32_t base = blockIdx.x * kTile, acc = 0;
  for (int r = 0; r < kRounds; ++r) {
    uint32_t i = base + r * kBlock + threadIdx.x;
    if (i < n) acc += in[i];
  }
  uint32_t s = block_sum<kBlock, uint32_t>(acc, scratch);
  if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

// Single block: sums[0..nb) -> exclusive prefix in place; *total = the sum.
__global__ void __launch_bounds__(kBlock) k_scan_sums(uint32_t* sums, uint32_t nb, uint32_t* total) {
  __shared__ uint32_t scratch[kBlock / 32 + 1];
  uint32_t carry = 0;
  for (uint32_t b = 0; b < nb; b += kBlock) {
    uint32_t i = b + threadIdx.x;
    uint32_t v = (i < nb) ? sums[i] : 0u, tot;
    uint32_t e = block_excl_scan<kBlock>(v, scratch, &tot);
    if (i < nb) sums[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kBlock) k_apply(const uint32_t* __restrict__ in, uint32_t n,
                                                  const uint32_t* __restrict__ sums,
                                                  uint32_t* __restrict__ out,
                                                  const uint32_t* __restrict__ n_dev) {
  __shared__ uint32_t scratch[kBlock / 32 + 1];
  if (n_dev) n = min(n, *n_dev);
  if (blockIdx.x * kTile >= n && blockIdx.x > 0) return;
  uint32_t base = blockIdx.x * kTile, carry = sums[blockIdx.x];
  for (int r = 0; r < kRounds; ++r) {
    uint32_t i = base + r * kBlock + threadIdx.x;
    uint32_t v = (i < n) ? in[i] : 0u, tot;
    uint32_t e = block_excl_scan<kBlock>(v, scratch, &tot);
    if (i < n) out[i] = carry + e;
    carry += tot;
  }
}

// Single block for n <= kTile: out = exclusive prefix of in, *total = the sum (one launch).
__global__ void __launch_bounds__(kBlock) k_scan_small(const uint32_t* __restrict__ in, uint32_t n,
                                                       uint32_t* __restrict__ out, uint32_t* total) {
  __shared__ uint32_t scratch[kBlock / 32 + 1];
  uint32_t carry = 0;
  for (uint32_t b = 0; b < n; b += kBlock) {
    const uint32_t i = b + threadIdx.x;
    uint32_t v = (i < n) ? in[i] : 0u, tot;
    const uint32_t e = block_excl_scan<kBlock>(v, scratch, &tot);
    if (i < n) out[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

}  // namespace scan
}  // namespace cvetl
