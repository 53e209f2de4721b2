// radix_sort.cuh — stable LSD radix sort of (key, uint32 value) pairs, one scatter pass per
// 8-bit digit with decoupled look-back (the single-pass "onesweep" scheme of Adinets and
// Merrill, 2022): an up-front histogram pass computes every digit's global counts, then each
// pass counts a 4096-item tile's digits, publishes the counts, looks back over earlier tiles for
// its global offsets, ranks the tile in shared memory and scatters through shared memory so that
// consecutive threads write consecutive addresses.
#pragma once
#include "common.cuh"

namespace cvetl {
namespace rs {

constexpr int kBits = 8;
constexpr int kRadix = 256;
constexpr int kBlock = 256;
constexpr int kIpt = 16;
constexpr int kTile = kBlock * kIpt;  // 4096
constexpr int kWarps = kBlock / 32;
constexpr int kMaxPasses = 8;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 22;  // look-back polls before the tile gives up
constexpr int kLookBack = 4;          // predecessors' status words read per round trip

// The digit of a pass at bit `shift`; dmask keeps only the bits below the sort's end bit (255
// unless the last pass's digit is narrower than 8 bits), so that bits at or above the end bit
// take no part in the order.
template <typename K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift, uint32_t dmask) {
  return (uint32_t)(k >> shift) & dmask;
}

// Mask of the digit at bit `shift` of a sort by bits [.., end_bit).
__host__ __device__ __forceinline__ uint32_t digit_mask(int shift, int end_bit) {
  return (end_bit - shift >= kBits) ? (uint32_t)(kRadix - 1) : ((1u << (end_bit - shift)) - 1u);
}

// Histograms of n_passes digits starting at begin_bit, over bits below end_bit. hist:
// [kMaxPasses][256], zeroed. n_dev != nullptr: the key count is read from device memory (n is
// then an upper bound).
template <typename K>
__global__ void __launch_bounds__(kBlock) k_histogram(const K* __restrict__ keys, uint32_t n,
                                                      int begin_bit, int n_passes, int end_bit,
                                                      uint32_t* __restrict__ hist,
                                                      const uint32_t* __restrict__ n_dev) {
  __shared__ uint32_t sh[kMaxPasses][kRadix];
  if (n_dev) n = min(n, *n_dev);
  for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += kBlock) (&sh[0][0])[i] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * kBlock + threadIdx.x; i < n; i += gridDim.x * kBlock) {
    K k = keys[i];
    for (int p = 0; p < n_passes; ++p) {
      const int shift = begin_bit + kBits * p;
      atomicAdd(&sh[p][digit_of(k, shift, digit_mask(shift, end_bit))], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_passes * kRadix; i += kBlock) {
    uint32_t v = (&sh[0][0])[i];
    if (v) atomicAdd(&hist[i], v);
  }
}

// In place: hist[p][d] -> exclusive prefix over d. One block of 256 threads per pass.
__global__ void __launch_bounds__(kBlock) k_hist_scan(uint32_t* hist) {
  __shared__ uint32_t scratch[kBlock / 32 + 1];
  uint32_t* h = hist + blockIdx.x * kRadix;
  uint32_t v = h[threadIdx.x];
  uint32_t e = block_excl_scan<kBlock>(v, scratch, nullptr);
  h[threadIdx.x] = e;
}

// Exclusive prefix of digit `tid`'s counts over the tiles before `tile` (decoupled look-back):
// the tile's count is already published as an aggregate; the predecessors' status words are
// read four tiles per round trip, aggregates summed until an inclusive prefix is found. A word
// not yet published is polled with a bounded wait (timeout: error bit, prefix left partial).
__device__ __forceinline__ uint32_t look_back(const uint32_t* status, uint32_t tile, int tid, uint32_t* err) {
  uint32_t excl = 0;
  int64_t p = (int64_t)tile - 1;
  bool done = false;
  while (p >= 0 && !done) {
    uint32_t sv[kLookBack];
#pragma unroll
    for (int q = 0; q < kLookBack; ++q)
      sv[q] = (p - q >= 0) ? ld_relaxed_u32(status + (size_t)(p - q) * kRadix + tid) : 0u;
#pragma unroll
    for (int q = 0; q < kLookBack; ++q) {
      if (done || p - q < 0) break;
      uint32_t s = sv[q];
      int spins = 0;
      while ((s & (kFlagAgg | kFlagPre)) == 0) {
        if (++spins > kSpinLimit) break;
        __nanosleep(32);
        s = ld_relaxed_u32(status + (size_t)(p - q) * kRadix + tid);
      }
      if ((s & (kFlagAgg | kFlagPre)) == 0) {
        atomicOr(err, kErrLookbackTimeout);
        done = true;
        break;
      }
      excl += s & kValMask;
      if (s & kFlagPre) done = true;
    }
    p -= kLookBack;
  }
  return excl;
}

// One digit pass over the bits of `dmask` at `shift`. status: [n_tiles][256] words, zeroed;
// tile_ctr zeroed.
// vin == nullptr means value = input position (iota). n_dev != nullptr: the key count is read
// from device memory and the grid covers the upper bound n; tiles are numbered in the order the
// CTAs start, so a tile that starts past the count returns at once (no tile holding keys looks
// back at it).
// A tile loads its keys, prefetches into L2 those of the tile one wave of resident CTAs later
// (numbered 3 per SM past its own: the tile that starts about when this one finishes), then
// counts its warps' digits (the digit's lanes found by ballots, the lowest of them
// adding their number), publishes its counts, looks back for the earlier tiles' totals, then
// ranks its keys in input order, warp by warp (i-major, lane-minor, their global order, so the
// pass is stable), writes them to their tile positions in shared memory and copies the tile
// out digit run by digit run, consecutive threads to consecutive addresses.
template <typename K>
__global__ void __launch_bounds__(kBlock, 3) k_onesweep(const K* __restrict__ kin,
                                                        const uint32_t* __restrict__ vin,
                                                        K* __restrict__ kout,
                                                        uint32_t* __restrict__ vout, uint32_t n,
                                                        int shift, uint32_t dmask,
                                                        const uint32_t* __restrict__ goff,
                                                        uint32_t* status, uint32_t* tile_ctr,
                                                        uint32_t* err, const uint32_t* __restrict__ n_dev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* s_keys = reinterpret_cast<K*>(smem_raw);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(smem_raw + sizeof(K) * kTile);
  __shared__ uint32_t s_wcnt[kWarps][kRadix];  // warp's digit counts, then its first tile positions
  __shared__ uint32_t s_gbase[kRadix];         // output position of tile position 0 per digit
  __shared__ uint32_t s_scan[kBlock / 32 + 1];
  __shared__ uint32_t s_tile;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  for (int i = tid; i < kWarps * kRadix; i += kBlock) (&s_wcnt[0][0])[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t base = tile * kTile;
  if (n_dev) {
    n = min(n, *n_dev);
    if (base >= n && tile > 0) return;
  }
  const uint32_t n_valid = (base < n) ? min((uint32_t)kTile, n - base) : 0u;

  K key[kIpt];
  uint32_t val[kIpt], peers[kIpt];
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    uint32_t idx = base + warp * (32 * kIpt) + i * 32 + lane;
    bool ok = idx < n;
    key[i] = ok ? kin[idx] : ~K(0);
    val[i] = ok ? (vin ? vin[idx] : idx) : 0u;
  }
  {
    // the tile one wave of resident CTAs ahead (3 per SM) into L2 while this one ranks: one
    // prefetch per 128-byte line, inside the arrays
    uint32_t nsm;
    asm("mov.u32 %0, %%nsmid;" : "=r"(nsm));
    const unsigned long long b2 = (unsigned long long)(tile + 3u * nsm) * kTile;
    if (b2 < n) {
      const uint32_t m2 = min((unsigned long long)kTile, n - b2);
      const uint32_t kl = (m2 * (uint32_t)sizeof(K) + 127u) / 128u;
      if ((uint32_t)tid < kl) asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)(kin + b2) + 128u * tid));
      const uint32_t vl = vin ? (m2 * 4u + 127u) / 128u : 0u;
      if ((uint32_t)tid < vl) asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)(vin + b2) + 128u * tid));
    }
  }
  // the warps' digit counts
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    const uint32_t d = digit_of(key[i], shift, dmask);
    peers[i] = match_label<kBits>(d);
    if (lane == __ffs(peers[i]) - 1) atomicAdd(&s_wcnt[warp][d], (uint32_t)__popc(peers[i]));
  }
  __syncthreads();
  // Thread t owns digit t: offsets of the warps inside the digit, the tile's count.
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    uint32_t c = s_wcnt[w][tid];
    s_wcnt[w][tid] = run;
    run += c;
  }
  // Items past n carry key ~0 (the largest digit, dmask) and rank after every valid item of
  // that digit.
  const uint32_t cnt_valid = run - ((tid == (int)dmask) ? (kTile - n_valid) : 0u);
  uint32_t* my_status = status + (size_t)tile * kRadix + tid;
  uint32_t excl = 0;
  if (tile == 0) {
    st_relaxed_u32(my_status, kFlagPre | cnt_valid);
  } else {
    st_relaxed_u32(my_status, kFlagAgg | cnt_valid);
    excl = look_back(status, tile, tid, err);
    st_relaxed_u32(my_status, kFlagPre | (excl + cnt_valid));
  }
  const uint32_t ts = block_excl_scan<kBlock>(run, s_scan, nullptr);
  s_gbase[tid] = goff[tid] + excl - ts;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s_wcnt[w][tid] += ts;
  __syncthreads();
  // ranks in input order; each key goes straight to its tile position
#pragma unroll
  for (int i = 0; i < kIpt; ++i) {
    const uint32_t d = digit_of(key[i], shift, dmask);
    const uint32_t before = s_wcnt[warp][d];
    __syncwarp();
    if (lane == __ffs(peers[i]) - 1) s_wcnt[warp][d] = before + __popc(peers[i]);
    __syncwarp();
    const uint32_t pos = before + __popc(peers[i] & lanemask_lt());
    s_keys[pos] = key[i];
    s_vals[pos] = val[i];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kIpt; ++j) {
    uint32_t p = j * kBlock + tid;
    if (p < n_valid) {
      K k = s_keys[p];
      uint32_t g = s_gbase[digit_of(k, shift, dmask)] + p;
      kout[g] = k;
      vout[g] = s_vals[p];
    }
  }
}

}  // namespace rs
}  // namespace cvetl
