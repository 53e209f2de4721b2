// cells.cuh — load stage: runs sorted by (key, first sorted position) are folded into the
// cell x bin table (count, sum, min, max, mean), in a fixed order.
#pragma once
#include "common.cuh"
#include "keying.cuh"

namespace cvetl {

// R_dev != nullptr (here and in k_cell_write): the run count is read from device memory and R
// is the upper bound the grid covers.
__global__ void k_cell_heads(const unsigned long long* __restrict__ skey, uint32_t R,
                             uint32_t* __restrict__ head, const uint32_t* __restrict__ R_dev) {
  if (R_dev) R = min(R, *R_dev);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x)
    head[i] = (i == 0 || (skey[i] >> 32) != (skey[i - 1] >> 32)) ? 1u : 0u;
}

struct CellOut {
  uint32_t* key;
  int32_t *row, *col, *bin;
  uint32_t* count;
  double *sum, *mean;
  float *min, *max;
  uint32_t* volume;  // unique journeys (batch mode)
};

// Rank of the journey whose sorted points contain position pos (joff: J ascending offsets).
__device__ __forceinline__ uint32_t journey_of(const uint32_t* __restrict__ joff, uint32_t J, uint32_t pos) {
  uint32_t lo = 0, hi = J;  // last offset <= pos
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (joff[mid] <= pos) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_cell_write(const unsigned long long* __restrict__ skey,
                             const uint32_t* __restrict__ sidx, uint32_t R,
                             const uint32_t* __restrict__ head, const uint32_t* __restrict__ cidx,
                             const uint32_t* __restrict__ run_cnt, const double* __restrict__ run_sum,
                             const float* __restrict__ run_min, const float* __restrict__ run_max,
                             int32_t n_rows, int32_t n_cols, Batch bt,
                             CellOut o, const uint32_t* __restrict__ R_dev,
                             const uint32_t* __restrict__ joff, uint32_t J) {
  if (R_dev) R = min(R, *R_dev);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) {
    if (!head[i]) continue;
    const uint32_t key = (uint32_t)(skey[i] >> 32);
    uint32_t cnt = 0, vol = 0, prev_j = 0xFFFFFFFFu;
    double sum = 0.0;
    float mn = run_min[sidx[i]], mx = run_max[sidx[i]];
    // runs of a key come by first sorted position, so one journey's runs are adjacent
    for (uint32_t m = i; m < R && (uint32_t)(skey[m] >> 32) == key; ++m) {
      uint32_t r = sidx[m];
      cnt += run_cnt[r];
      sum += run_sum[r];
      mn = fminf(mn, run_min[r]);
      mx = fmaxf(mx, run_max[r]);
      if (o.volume) {
        const uint32_t jr = journey_of(joff, J, (uint32_t)skey[m]);
        vol += jr != prev_j;
        prev_j = jr;
      }
    }
    const uint32_t c = cidx[i];
    uint32_t lkey = key;  // a batch reports each instance's own keys
    int32_t nr = n_rows, nc = n_cols;
    if (bt.n_inst) {
      const int q = inst_of_key(bt, key);
      lkey = key - bt.inst[q].key_off;
      nr = bt.inst[q].n_rows;
      nc = bt.inst[q].n_cols;
    }
    const uint32_t cells = (uint32_t)nr * (uint32_t)nc;
    o.key[c] = lkey;
    o.bin[c] = (int32_t)(lkey / cells);
    o.row[c] = (int32_t)((lkey % cells) / (uint32_t)nc);
    o.col[c] = (int32_t)(lkey % (uint32_t)nc);
    o.count[c] = cnt;
    o.sum[c] = sum;
    o.mean[c] = sum / (double)cnt;
    o.min[c] = mn;
    o.max[c] = mx;
    if (o.volume) o.volume[c] = vol;
  }
}

// First journey rank and first cell row of each batch instance (out[i], out[kMaxInst + i]), by
// binary search over the sorted journey keys (order-preserving keys of (instance, id)) and the
// sorted run keys ((key << 32) | position; an instance's first run heads its first cell).
// One thread per instance.
__global__ void k_inst_begins(const unsigned long long* __restrict__ jkey, uint32_t J,
                              const unsigned long long* __restrict__ rkey, uint32_t R,
                              const uint32_t* __restrict__ R_dev, const uint32_t* __restrict__ cidx,
                              const uint32_t* __restrict__ K_dev, Batch bt, uint32_t* __restrict__ out) {
  if (R_dev) R = min(R, *R_dev);
  const int i = threadIdx.x;
  if (i >= bt.n_inst) return;
  const unsigned long long jk = ((unsigned long long)i << kInstShift) ^ kSign64;
  uint32_t lo = 0, hi = J;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (jkey[mid] < jk) lo = mid + 1;
    else hi = mid;
  }
  out[i] = lo;
  const unsigned long long ck = (unsigned long long)bt.inst[i].key_off << 32;
  lo = 0;
  hi = R;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (rkey[mid] < ck) lo = mid + 1;
    else hi = mid;
  }
  out[kMaxInst + i] = lo < R ? cidx[lo] : *K_dev;
}

}  // namespace cvetl
