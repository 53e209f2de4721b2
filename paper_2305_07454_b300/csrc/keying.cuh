// keying.cuh — the grid / time-bin key of Algorithm 2 (row, column and bin by floor division,
// unrolled into one positional index), shared by the kernels that key points: the scatter of
// the batch path and the append of the stream path.
#pragma once
#include "common.cuh"

namespace cvetl {

// cosine table entry: {lat0 = k * 0.01, cos(lat0 deg), sin(lat0 deg) * pi/180, unused}
struct __align__(32) CosEntry {
  double lat0, c0, s0r, pad;
};

struct GridParams {
  const unsigned long long* row_thr;  // n_rows + 1 ordered thresholds (see keying below)
  const unsigned long long* col_thr;  // n_cols + 1
  float lat_min_f, lon_min_f, inv_cell_f;
  int32_t n_rows, n_cols, n_bins;
  int64_t t0_ms, bin_ms;
  unsigned long long t_span;  // n_bins * bin_ms, saturated
  float v_stop;
  double radius_m;
  const CosEntry* cos_tab;  // k = -9000..9000
  double asin_c1, asin_c2, asin_c3;  // 2R, 2R/6, 2R*3/40: d = sqrt(h) (c1 + h (c2 + h c3))
  double dist_k;                     // 2R pi/360: distance per degree of sqrt(m) (binary64 series)
};

// ---------------------------------------------------------------- keying (Algorithm 2)
// row = floor(RN(RN(lat - lat_min) / cell)) is a non-decreasing function of lat, so it is
// fixed by the smallest binary64 value at which it reaches each k (computed once on the host
// with the binary64 formula itself). The device compares order-preserving bit patterns with
// that table: no floating-point division, bit-exact with the binary64 definition. A float
// estimate from the double's leading bits picks the table entry; one or two compares fix it.
__device__ __forceinline__ float leading_f32(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  uint32_t hi = (uint32_t)(b >> 32);
  uint32_t sign = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7FF);
  if (e < 1023 - 126) return __int_as_float((int)sign);
  if (e > 1023 + 127) return __int_as_float((int)(sign | 0x7F800000u));
  uint32_t mant = ((hi & 0xFFFFFu) << 3) | (uint32_t)((b >> 29) & 7u);
  return __int_as_float((int)(sign | ((uint32_t)(e - 1023 + 127) << 23) | mant));
}

__device__ __forceinline__ int grid_index(double x, const unsigned long long* __restrict__ thr,
                                          int n, float xmin_f, float inv_f) {
  unsigned long long u = ord_f64(x);
  if (u < __ldg(&thr[0]) || u >= __ldg(&thr[n])) return -1;
  int r = __float2int_rd((leading_f32(x) - xmin_f) * inv_f);
  r = max(0, min(n - 1, r));
  while (r > 0 && u < __ldg(&thr[r])) --r;
  while (r < n - 1 && u >= __ldg(&thr[r + 1])) ++r;
  return r;
}

// bin = floor((ts - t0) / bin_ms) when 0 <= bin < n_bins, else -1 (exact integer arithmetic).
__device__ __forceinline__ int time_bin(int64_t ts, const GridParams& g) {
  if (ts < g.t0_ms) return -1;
  unsigned long long off = (unsigned long long)ts - (unsigned long long)g.t0_ms;
  if (off >= g.t_span) return -1;
  if (g.t_span <= 0xFFFFFFFFull) return (int)((uint32_t)off / (uint32_t)g.bin_ms);
  return (int)(off / (unsigned long long)g.bin_ms);
}

__device__ __forceinline__ uint32_t cell_key(double lat, double lon, int64_t ts, const GridParams& g) {
  int r = grid_index(lat, g.row_thr, g.n_rows, g.lat_min_f, g.inv_cell_f);
  int c = grid_index(lon, g.col_thr, g.n_cols, g.lon_min_f, g.inv_cell_f);
  int b = time_bin(ts, g);
  if (r < 0 || c < 0 || b < 0) return kKeyInvalid;
  return ((uint32_t)b * (uint32_t)g.n_rows + (uint32_t)r) * (uint32_t)g.n_cols + (uint32_t)c;
}

}  // namespace cvetl
