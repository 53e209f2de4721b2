// lattice.cuh — the 8-channel spatio-temporal lattice: per lattice time bin, direction and cell,
// the mean point speed and the number of unique journeys (channels 2d and 2d + 1 of direction
// d), min-max normalised per channel, optionally written densely as [bin][8][row][col].
// (Results: the 5-minute channel images of speed and volume in four cardinal directions;
// Algorithm 2, step 3: direction = heading // dxn_step; Table 3: "Count Unique (Volume)",
// "Normalize".)
#pragma once
#include "common.cuh"
#include "keying.cuh"

namespace cvetl {

struct LatticeParams {
  int64_t bin_ms;
  int32_t n_bins;
  int32_t direction;   // 0 cardinal: floor(((h + 45) mod 360) / 90); 1 quadrant: floor((h mod 360) / 90)
  int32_t rank_bits;   // bits of the journey rank in the sort key
  unsigned long long t_span;     // n_bins * bin_ms (saturated)
  unsigned long long bin_magic;  // ceil(2^64 / bin_ms) (0 for bin_ms = 1)
};

// Direction channel of a heading by the definition, binary64 arithmetic on the float32
// heading; -1 for a non-finite heading. (Out of line: only headings outside the usual range
// take it.)
__device__ __noinline__ int lattice_direction_exact(float heading, int mode) {
  const double h = (double)heading;
  if (!isfinite(h)) return -1;
  double r = fmod(h + (mode == 0 ? 45.0 : 0.0), 360.0);
  if (r < 0.0) r += 360.0;
  if (r >= 360.0) r = 0.0;
  return (int)floor(r / 90.0);
}

// The same for the headings of the usual range by float32 compares. For a cardinal h in
// [-45, 315) (quadrant: [0, 360)), r = h + 45 (h) lies in [0, 360) where the remainder is r
// itself, h + 45 is exact in binary64 wherever it decides a sector, and floor(r / 90) of the
// correctly rounded quotient is the number of the edges 90, 180, 270 that r reaches (a quotient
// just below an integer k never rounds up to k: its distance to k exceeds half an ulp of k), so
// the sector is the number of edges h reaches. A cardinal h in [315, 405) has the remainder
// h + 45 - 360 in [0, 90) (sector 0); one in [-405, -45) has h + 405 (exact: |h| >= 45, so h
// needs no bits below 2^-18), whose sector counts the edges -315, -225, -135 that h reaches.
__device__ __forceinline__ int lattice_direction(float heading, int mode) {
  if (mode == 0) {
    if (heading >= -45.0f && heading < 315.0f)
      return (heading >= 45.0f) + (heading >= 135.0f) + (heading >= 225.0f);
    if (heading >= 315.0f && heading < 405.0f) return 0;
    if (heading >= -405.0f && heading < -45.0f)
      return (heading >= -315.0f) + (heading >= -225.0f) + (heading >= -135.0f);
  } else if (heading >= 0.0f && heading < 360.0f) {
    return (heading >= 90.0f) + (heading >= 180.0f) + (heading >= 270.0f);
  }
  return lattice_direction_exact(heading, mode);
}

// Sort key of every row: (lattice key << rank_bits) | journey rank for a kept row that has a
// lattice position, all-ones otherwise (sorted last); the speed is the sort's payload. Dropped
// kept rows are counted. Four rows per thread per iteration: their columns and their journeys'
// ranks are loaded before any of them is keyed, so the loads overlap.
constexpr int kLatRows = 4;
__global__ void __launch_bounds__(256) k_lattice_keys(const uint32_t* __restrict__ row_slot,
                                                      const uint32_t* __restrict__ slot_rank,
                                                      const int64_t* __restrict__ ts,
                                                      const double* __restrict__ lat,
                                                      const double* __restrict__ lon,
                                                      const float* __restrict__ heading, uint32_t n,
                                                      const float* __restrict__ spd, GridParams g,
                                                      LatticeParams lp, unsigned long long* __restrict__ keys,
                                                      uint32_t* __restrict__ vals,
                                                      unsigned long long* n_dropped) {
  __shared__ unsigned long long scratch[8];
  unsigned long long dropped = 0;
  const uint32_t step = gridDim.x * blockDim.x * kLatRows;
  for (uint32_t i0 = blockIdx.x * blockDim.x * kLatRows + threadIdx.x; i0 < n; i0 += step) {
    uint32_t slot[kLatRows], rank[kLatRows];
    float hd[kLatRows], sp[kLatRows];
    double la[kLatRows], lo[kLatRows];
    int64_t t[kLatRows];
#pragma unroll
    for (int u = 0; u < kLatRows; ++u) {
      const uint32_t i = i0 + u * blockDim.x;
      const bool in = i < n;
      slot[u] = in ? row_slot[i] : kKeyInvalid;
      hd[u] = in ? heading[i] : 0.0f;
      sp[u] = in ? spd[i] : 0.0f;
      la[u] = in ? lat[i] : 0.0;
      lo[u] = in ? lon[i] : 0.0;
      t[u] = in ? ts[i] : 0;
    }
#pragma unroll
    for (int u = 0; u < kLatRows; ++u) rank[u] = (slot[u] != kKeyInvalid) ? slot_rank[slot[u]] : 0u;
#pragma unroll
    for (int u = 0; u < kLatRows; ++u) {
      const uint32_t i = i0 + u * blockDim.x;
      if (i >= n) break;
      unsigned long long k = ~0ull;
      if (slot[u] != kKeyInvalid) {
        const int d = lattice_direction(hd[u], lp.direction);
        const int r = grid_index(la[u], g.row_thr, g.n_rows, g.lat_min_f, g.inv_cell_f);
        const int c = grid_index(lo[u], g.col_thr, g.n_cols, g.lon_min_f, g.inv_cell_f);
        const unsigned long long off = (unsigned long long)t[u] - (unsigned long long)g.t0_ms;
        if (d < 0 || r < 0 || c < 0 || t[u] < g.t0_ms || off >= lp.t_span) {
          ++dropped;
        } else {
          const unsigned long long b = (lp.t_span <= 0xFFFFFFFFull)
                                           ? (lp.bin_magic ? __umul64hi(lp.bin_magic, off) : off)
                                           : off / (unsigned long long)lp.bin_ms;
          const unsigned long long lk =
              ((b * 4ull + (unsigned long long)d) * (unsigned long long)g.n_rows + (unsigned long long)r) *
                  (unsigned long long)g.n_cols + (unsigned long long)c;
          k = (lk << lp.rank_bits) | (unsigned long long)rank[u];
        }
      }
      keys[i] = k;
      vals[i] = __float_as_uint(sp[u]);  // the sort's payload: the speed, read in lattice order
    }
  }
  const unsigned long long s = block_sum<256, unsigned long long>(dropped, scratch);
  if (threadIdx.x == 0 && s) atomicAdd(n_dropped, s);
}

// Segment heads of the sorted keys (a key whose cell differs from its predecessor's) counted
// per tile of kLatTile keys: thread t of the block takes keys [16t, 16t + 16) of its tile.
constexpr int kLatPer = 16;
constexpr int kLatTile = 256 * kLatPer;

__device__ __forceinline__ uint32_t lat_heads(const unsigned long long* __restrict__ skey, uint32_t m,
                                              int rank_bits, uint32_t i0, uint32_t& mask) {
  unsigned long long prev = i0 ? (skey[i0 - 1] >> rank_bits) : ~0ull;
  mask = 0;
  if (i0 + kLatPer <= m) {  // 16 keys in four 32-byte loads
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(skey + i0);
#pragma unroll
    for (int v = 0; v < kLatPer / 2; ++v) {
      const ulonglong2 kk = __ldg(p + v);
      const unsigned long long a = kk.x >> rank_bits, b = kk.y >> rank_bits;
      mask |= (i0 + 2 * v == 0 || a != prev ? 1u : 0u) << (2 * v);
      mask |= (b != a ? 1u : 0u) << (2 * v + 1);
      prev = b;
    }
  } else {
    for (int u = 0; u < kLatPer && i0 + u < m; ++u) {
      const unsigned long long a = skey[i0 + u] >> rank_bits;
      mask |= (i0 + u == 0 || a != prev ? 1u : 0u) << u;
      prev = a;
    }
  }
  return (uint32_t)__popc(mask);
}

__global__ void __launch_bounds__(256) k_lattice_tile_heads(const unsigned long long* __restrict__ skey, uint32_t m,
                                                            int rank_bits, uint32_t* __restrict__ tile_cnt) {
  __shared__ uint32_t scratch[8];
  const uint32_t i0 = blockIdx.x * kLatTile + threadIdx.x * kLatPer;
  uint32_t mask, c = 0;
  if (i0 < m) c = lat_heads(skey, m, rank_bits, i0, mask);
  const uint32_t tot = block_sum<256, uint32_t>(c, scratch);
  if (threadIdx.x == 0) tile_cnt[blockIdx.x] = tot;
}

// Cell starts: the q-th segment head's position at start[q], and start[K] = m. The tile's heads
// are numbered from its offset (the exclusive scan of the tile counts) in key order.
__global__ void __launch_bounds__(256) k_lattice_tile_starts(const unsigned long long* __restrict__ skey, uint32_t m,
                                                             int rank_bits, const uint32_t* __restrict__ tile_off,
                                                             const uint32_t* __restrict__ K,
                                                             uint32_t* __restrict__ start) {
  __shared__ uint32_t scratch[256 / 32 + 1];
  const uint32_t i0 = blockIdx.x * kLatTile + threadIdx.x * kLatPer;
  uint32_t mask = 0, c = 0;
  if (i0 < m) c = lat_heads(skey, m, rank_bits, i0, mask);
  uint32_t o = tile_off[blockIdx.x] + block_excl_scan<256>(c, scratch, nullptr);
  while (mask) {
    start[o++] = i0 + (uint32_t)(__ffs(mask) - 1);
    mask &= mask - 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) start[*K] = m;
}

struct LatticeOut {
  uint32_t* key;
  int32_t *bin, *dxn, *row, *col;
  uint32_t* count;
  double* sum;
  float* mean;
  uint32_t* volume;
  float *mean_norm, *volume_norm;
};

__device__ __forceinline__ uint32_t ord_f32(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_ord_f32(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u ^ 0x80000000u) : ~u);
}

// Sort keys of the cells by length, longest first (ties by cell).
__global__ void k_lattice_len_keys(const uint32_t* __restrict__ start, const uint32_t* __restrict__ Kp,
                                   unsigned long long* __restrict__ lkey) {
  const uint32_t K = *Kp;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < K; q += gridDim.x * blockDim.x)
    lkey[q] = ((unsigned long long)(0xFFFFFFFFu - (start[q + 1] - start[q])) << 32) | q;
}

// One thread per lattice cell: its points in (journey, row) order give the count, the speed sum
// in that order (binary64, one add per point as defined), the mean and the unique journeys; the
// channel extremes go to chan[0..7] (min) and chan[8..15] (max) as order-preserving words.
// Cells are taken in the order `order` (longest first), so that the lanes of a warp fold
// cells of about the same length; each cell's own points keep their order.
__global__ void k_lattice_fold(const unsigned long long* __restrict__ skey, const uint32_t* __restrict__ sspd,
                               const uint32_t* __restrict__ start, const uint32_t* __restrict__ order,
                               const uint32_t* __restrict__ Kp, int rank_bits, int32_t n_rows, int32_t n_cols,
                               LatticeOut o, uint32_t* __restrict__ chan) {
  // channel extremes of this block's cells, merged into chan once per block (the 16 words of
  // chan would otherwise take four contended global atomics per cell)
  __shared__ uint32_t s_chan[16];
  if (threadIdx.x < 16) s_chan[threadIdx.x] = threadIdx.x < 8 ? 0xFFFFFFFFu : 0u;
  __syncthreads();
  const uint32_t K = *Kp;
  const unsigned long long rmask = (1ull << rank_bits) - 1;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < K; w += gridDim.x * blockDim.x) {
    const uint32_t q = order ? order[w] : w;
    const uint32_t e0 = start[q], e1 = start[q + 1];
    const unsigned long long lk = skey[e0] >> rank_bits;
    uint32_t vol = 0;
    double sum = 0.0;
    unsigned long long prev_rank = ~0ull;
    // the cell's entries four at a time: the loads first (independent), then the sum in order
    for (uint32_t e4 = e0; e4 < e1; e4 += 4) {
      uint32_t sv[4];
      unsigned long long kv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = e4 + u < e1;
        sv[u] = in ? sspd[e4 + u] : 0u;
        kv[u] = in ? skey[e4 + u] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (e4 + u >= e1) break;
        const float sp = __uint_as_float(sv[u]);
        sum += f32_to_f64_exact(((sv[u] & 0x7FFFFFFFu) == 0) ? 0.0f : sp);
        const unsigned long long rk = kv[u] & rmask;
        vol += (rk != prev_rank) ? 1u : 0u;
        prev_rank = rk;
      }
    }
    const uint32_t cnt = e1 - e0;
    const uint32_t key = (uint32_t)lk, cells = (uint32_t)n_rows * (uint32_t)n_cols;
    const int d = (int)((key / cells) % 4u);
    const float mean = (float)(sum / (double)cnt);
    o.key[q] = key;
    o.bin[q] = (int32_t)(key / (cells * 4u));
    o.dxn[q] = d;
    o.row[q] = (int32_t)((key % cells) / (uint32_t)n_cols);
    o.col[q] = (int32_t)(key % (uint32_t)n_cols);
    o.count[q] = cnt;
    o.sum[q] = sum;
    o.mean[q] = mean;
    o.volume[q] = vol;
    atomicMin(&s_chan[2 * d], ord_f32(mean));
    atomicMax(&s_chan[8 + 2 * d], ord_f32(mean));
    atomicMin(&s_chan[2 * d + 1], ord_f32((float)vol));
    atomicMax(&s_chan[8 + 2 * d + 1], ord_f32((float)vol));
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    if (s_chan[threadIdx.x] != 0xFFFFFFFFu) atomicMin(&chan[threadIdx.x], s_chan[threadIdx.x]);
  } else if (threadIdx.x < 16) {
    if (s_chan[threadIdx.x] != 0u) atomicMax(&chan[threadIdx.x], s_chan[threadIdx.x]);
  }
}

// Min-max normalisation per channel and, when dense != nullptr, the dense tensor
// [n_bins][8][n_rows][n_cols] (zeroed beforehand; channels of the normalised values when
// normalized, of the raw values otherwise).
__global__ void k_lattice_norm(uint32_t K, const uint32_t* __restrict__ chan, LatticeOut o, int32_t n_rows,
                               int32_t n_cols, float* __restrict__ dense, int normalized) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < K; q += gridDim.x * blockDim.x) {
    const int d = o.dxn[q];
    const float mn0 = from_ord_f32(chan[2 * d]), mx0 = from_ord_f32(chan[8 + 2 * d]);
    const float mn1 = from_ord_f32(chan[2 * d + 1]), mx1 = from_ord_f32(chan[8 + 2 * d + 1]);
    const float mean = o.mean[q], vol = (float)o.volume[q];
    const float mn = (mx0 > mn0) ? (mean - mn0) / (mx0 - mn0) : 0.0f;
    const float vn = (mx1 > mn1) ? (vol - mn1) / (mx1 - mn1) : 0.0f;
    o.mean_norm[q] = mn;
    o.volume_norm[q] = vn;
    if (dense) {
      const size_t plane = (size_t)n_rows * (size_t)n_cols;
      const size_t at = ((size_t)o.bin[q] * 8u + (size_t)(2 * d)) * plane + (size_t)o.row[q] * (size_t)n_cols +
                        (size_t)o.col[q];
      dense[at] = normalized ? mn : mean;
      dense[at + plane] = normalized ? vn : vol;
    }
  }
}

}  // namespace cvetl
