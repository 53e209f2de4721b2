// keying.cuh — the grid / time-bin key of Algorithm 2 (row, column and bin by floor division,
// unrolled into one positional index), computed per point by the journey kernel (batch and
// stream paths) and, with a direction channel, by the lattice.
#pragma once
#include "common.cuh"

namespace cvetl {

// cosine table entry: {lat0 = k * 0.01, cos(lat0 deg), sin(lat0 deg) * pi/180} in binary64 and
// the last two rounded to float32 (for the float32 form)
struct __align__(32) CosEntry {
  double lat0, c0, s0r;
  float c0f, s0rf;
};

struct GridParams {
  const unsigned long long* row_thr;  // n_rows + 1 ordered thresholds (see keying below)
  const unsigned long long* col_thr;  // n_cols + 1
  float lat_min_f, lon_min_f, inv_cell_f;
  int32_t n_rows, n_cols, n_bins;
  int64_t t0_ms, bin_ms;
  unsigned long long t_span;  // n_bins * bin_ms, saturated
  unsigned long long bin_magic;  // ceil(2^64 / bin_ms) (0 for bin_ms = 1): see bin_of
  float v_stop;
  double radius_m;
  const CosEntry* cos_tab;  // k = -9000..9000
  double asin_c1, asin_c2, asin_c3;  // 2R, 2R/6, 2R*3/40: d = sqrt(h) (c1 + h (c2 + h c3))
  double dist_k;                     // 2R pi/360: distance per degree of sqrt(m) (binary64 series)
  float dist_kh, dist_kl;            // dist_k as a float32 pair (the leading float, the rest)
};

// ---------------------------------------------------------------- keying (Algorithm 2)
// row = floor(RN(RN(lat - lat_min) / cell)) is a non-decreasing function of lat, so it is
// fixed by the smallest binary64 value at which it reaches each k (computed once on the host
// with the binary64 formula itself). The device compares order-preserving bit patterns with
// that table: no floating-point division, bit-exact with the binary64 definition. A float
// estimate from the double's leading bits picks the table entry; one or two compares fix it.
__device__ __forceinline__ float leading_f32(double x) {
  uint64_t b = dbits(x);
  uint32_t hi = (uint32_t)(b >> 32);
  uint32_t sign = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7FF);
  if (e < 1023 - 126) return __int_as_float((int)sign);
  if (e > 1023 + 127) return __int_as_float((int)(sign | 0x7F800000u));
  uint32_t mant = ((hi & 0xFFFFFu) << 3) | (uint32_t)((b >> 29) & 7u);
  return __int_as_float((int)(sign | ((uint32_t)(e - 1023 + 127) << 23) | mant));
}

// Threshold i of a table in global memory (read-only path) or in shared memory (kShared).
template <bool kShared>
__device__ __forceinline__ unsigned long long thr_at(const unsigned long long* __restrict__ thr, int i) {
  if constexpr (kShared) return thr[i];
  else return __ldg(thr + i);
}

// n >= 1. The cell is the r with thr[r] <= u < thr[r + 1]; both bounds of the estimate are
// loaded together, and a step past either end of the table means off the grid.
template <bool kShared = false>
__device__ __forceinline__ int grid_index(double x, const unsigned long long* __restrict__ thr,
                                          int n, float xmin_f, float inv_f) {
  const unsigned long long u = ord_f64(x);
  int r = __float2int_rd((leading_f32(x) - xmin_f) * inv_f);
  r = max(0, min(n - 1, r));
  unsigned long long lo = thr_at<kShared>(thr, r), hi = thr_at<kShared>(thr, r + 1);
  while (u < lo) {
    if (r == 0) return -1;
    --r;
    hi = lo;
    lo = thr_at<kShared>(thr, r);
  }
  while (u >= hi) {
    if (r == n - 1) return -1;
    ++r;
    lo = hi;
    hi = thr_at<kShared>(thr, r + 1);
  }
  return r;
}

// floor(off / bin_ms) for off < t_span. Below 2^32 by one multiply-high with c = ceil(2^64 / d):
// floor(x / d) = floor(c x / 2^64) for every 32-bit x and 32-bit d (Lemire, Kaser and Kurz,
// "Faster remainder by direct computation", 2019, with 64-bit fractions for 32-bit words).
__device__ __forceinline__ uint32_t bin_of(unsigned long long off, const GridParams& g) {
  if (g.t_span <= 0xFFFFFFFFull) return g.bin_magic ? (uint32_t)__umul64hi(g.bin_magic, off) : (uint32_t)off;
  return (uint32_t)(off / (unsigned long long)g.bin_ms);
}

// bin = floor((ts - t0) / bin_ms) when 0 <= bin < n_bins, else -1 (exact integer arithmetic).
__device__ __forceinline__ int time_bin(int64_t ts, const GridParams& g) {
  if (ts < g.t0_ms) return -1;
  unsigned long long off = (unsigned long long)ts - (unsigned long long)g.t0_ms;
  if (off >= g.t_span) return -1;
  return (int)bin_of(off, g);
}

// The key on the grid of g, with its threshold tables at row_thr and col_thr (g's own, or a
// copy of them in shared memory with kShared).
template <bool kShared = false>
__device__ __forceinline__ uint32_t cell_key(double lat, double lon, int64_t ts, const GridParams& g,
                                             const unsigned long long* __restrict__ row_thr,
                                             const unsigned long long* __restrict__ col_thr) {
  int r = grid_index<kShared>(lat, row_thr, g.n_rows, g.lat_min_f, g.inv_cell_f);
  int c = grid_index<kShared>(lon, col_thr, g.n_cols, g.lon_min_f, g.inv_cell_f);
  int b = time_bin(ts, g);
  if (r < 0 || c < 0 || b < 0) return kKeyInvalid;
  return ((uint32_t)b * (uint32_t)g.n_rows + (uint32_t)r) * (uint32_t)g.n_cols + (uint32_t)c;
}

// ---------------------------------------------------------------- batches of instances
// A batch holds up to kMaxInst instances (days x regions), each with its own grid origin and
// size and its own day, processed together: rows are concatenated, a journey is identified by
// (instance, id) packed as (instance << 58) + (id + 2^57) (ids within [-2^57, 2^57)), and each
// instance's keys are offset into one 32-bit key space, so every kernel makes one pass over all
// instances and the results come out instance by instance.
constexpr int kMaxInst = 32;  // CVETL_MAX_INSTANCES
constexpr int kInstShift = 58;
constexpr long long kIdBias = 1ll << 57;

struct BatchInst {
  const unsigned long long* row_thr;  // the instance's n_rows + 1 thresholds
  const unsigned long long* col_thr;  // n_cols + 1
  float lat_min_f, lon_min_f;
  int32_t n_rows, n_cols;
  int64_t t0_ms;
  uint32_t row_begin;  // first row of the instance in the concatenated columns
  uint32_t key_off;    // first key of the instance in the concatenated key space
  uint32_t group_begin;  // first group of the instance's rows (groups of kScatterRows rows, per instance)
};

// A batch's instance columns read in place (device batches): instance k's own arrays.
struct BatchCols {
  const int64_t *jid, *ts;
  const double *lat, *lon;
  const float* spd;
};

struct Batch {
  int n_inst;              // 0: one instance described by GridParams
  const BatchInst* inst;   // n_inst entries, ascending row_begin and key_off
  const BatchCols* cols;   // n_inst entries when the instances' columns are read in place, else null
                           // (the batch's rows are then concatenated in the context's columns)
};

// last instance whose row_begin (or key_off) is <= v
__device__ __forceinline__ int inst_of_row(const Batch& b, uint32_t row) {
  int lo = 0, hi = b.n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&b.inst[mid].row_begin) <= row) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
// The columns batch row i is read from and its index there: the concatenated columns `all`,
// or its instance's own columns (instance k from inst_of_row).
struct RowCols {
  const int64_t *jid, *ts;
  const double *lat, *lon;
  const float* spd;
};
__device__ __forceinline__ uint32_t row_cols(const Batch& b, const RowCols& all, uint32_t i, int k, RowCols& c) {
  if (!b.cols) {
    c = all;
    return i;
  }
  const BatchCols* q = b.cols + k;
  c.jid = reinterpret_cast<const int64_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&q->jid)));
  c.ts = reinterpret_cast<const int64_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&q->ts)));
  c.lat = reinterpret_cast<const double*>(__ldg(reinterpret_cast<const unsigned long long*>(&q->lat)));
  c.lon = reinterpret_cast<const double*>(__ldg(reinterpret_cast<const unsigned long long*>(&q->lon)));
  c.spd = reinterpret_cast<const float*>(__ldg(reinterpret_cast<const unsigned long long*>(&q->spd)));
  return i - __ldg(&b.inst[k].row_begin);
}

// Row i's timestamp (from its instance's own column when the batch is read in place).
__device__ __forceinline__ int64_t row_ts(const int64_t* __restrict__ ts, const Batch& b, uint32_t i) {
  if (!b.cols) return ts[i];
  RowCols c;
  const uint32_t r = row_cols(b, RowCols{}, i, inst_of_row(b, i), c);
  return c.ts[r];
}

// last instance whose first row group is <= g
__device__ __forceinline__ int inst_of_group(const Batch& b, uint32_t g) {
  int lo = 0, hi = b.n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&b.inst[mid].group_begin) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int inst_of_key(const Batch& b, uint32_t key) {
  int lo = 0, hi = b.n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&b.inst[mid].key_off) <= key) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool composite_id(int inst, int64_t jid, uint64_t* out) {
  if (jid < -kIdBias || jid >= kIdBias) return false;
  *out = ((uint64_t)inst << kInstShift) + (uint64_t)(jid + kIdBias);
  return true;
}
__device__ __forceinline__ int64_t composite_jid(uint64_t cid) {
  return (int64_t)(cid & ((1ull << kInstShift) - 1)) - kIdBias;
}

// The key of a row of instance bi, offset into the batch's key space.
__device__ __forceinline__ uint32_t batch_cell_key(double lat, double lon, int64_t ts, const GridParams& g,
                                                   const BatchInst& bi) {
  const int r = grid_index(lat, bi.row_thr, bi.n_rows, bi.lat_min_f, g.inv_cell_f);
  const int c = grid_index(lon, bi.col_thr, bi.n_cols, bi.lon_min_f, g.inv_cell_f);
  if (r < 0 || c < 0 || ts < bi.t0_ms) return kKeyInvalid;
  const unsigned long long off = (unsigned long long)ts - (unsigned long long)bi.t0_ms;
  if (off >= g.t_span) return kKeyInvalid;
  const int b = (int)bin_of(off, g);
  return bi.key_off + ((uint32_t)b * (uint32_t)bi.n_rows + (uint32_t)r) * (uint32_t)bi.n_cols + (uint32_t)c;
}

// The key of a point: of the single instance described by g (bi == nullptr) or of batch
// instance *bi.
__device__ __forceinline__ uint32_t point_key(double lat, double lon, int64_t ts, const GridParams& g,
                                              const BatchInst* bi) {
  return bi ? batch_cell_key(lat, lon, ts, g, *bi) : cell_key(lat, lon, ts, g, g.row_thr, g.col_thr);
}

}  // namespace cvetl
