// journey.cuh — one CTA per journey: order the journey's bucket by (timestamp, row index),
// then walk it in sorted order computing per-point kinematics and the Algorithm 2 key, the
// journey summary, and the runs of equal cell x bin keys that feed the load stage.
#pragma once
#include "common.cuh"

namespace cvetl {

constexpr int kJBlock = 256;   // threads per journey CTA
constexpr int kJCap = 4096;    // records sorted in shared memory in one piece

struct GridParams {
  const unsigned long long* row_thr;  // n_rows + 1 ordered thresholds (see keying below)
  const unsigned long long* col_thr;  // n_cols + 1
  float lat_min_f, lon_min_f, inv_cell_f;
  int32_t n_rows, n_cols, n_bins;
  int64_t t0_ms, bin_ms;
  unsigned long long t_span;  // n_bins * bin_ms, saturated
  float v_stop;
  double radius_m;
};

struct JourneyOut {
  // journey table, indexed by rank
  int64_t *n, *off, *start_ts, *end_ts, *duration, *dwell;
  double *dist, *slat, *slon, *elat, *elon;
  // per-point columns at sorted positions (all NULL unless materialised)
  uint32_t* perm;
  double* d;
  float *vhat, *accel;
  int64_t* dwell_pt;
  uint32_t* key;
  uint8_t* flags;
  // cell runs
  unsigned long long* run_sortkey;  // (key << 32) | sorted position of the run's first point
  uint32_t* run_cnt;
  double* run_sum;
  float *run_min, *run_max;
  uint32_t run_cap;
};

struct __align__(16) Elem {
  unsigned long long t;  // order-preserving timestamp
  uint32_t idx;          // extracted-row index (tie-break)
  uint32_t pos;          // position inside the journey's bucket
};

__device__ __forceinline__ bool elem_less(const Elem& a, const Elem& b) {
  return a.t < b.t || (a.t == b.t && a.idx < b.idx);
}

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

// ---------------------------------------------------------------- kinematics
// Haversine distance on a sphere of radius R; coordinates differenced in degrees first.
__device__ __forceinline__ double haversine_m(double la1, double lo1, double la2, double lo2, double R) {
  const double rad = 0.017453292519943295;  // pi / 180
  double dphi = (la2 - la1) * rad, dlam = (lo2 - lo1) * rad;
  double s1 = sin(0.5 * dphi), s2 = sin(0.5 * dlam);
  double h = s1 * s1 + cos(la1 * rad) * cos(la2 * rad) * (s2 * s2);
  double r = fmin(sqrt(h), 1.0);
  return 2.0 * R * asin(r);
}

// ---------------------------------------------------------------- in-CTA sorting
__device__ __forceinline__ void bitonic_smem(Elem* E, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += kJBlock) {
        int ixj = i ^ j;
        if (ixj > i) {
          Elem a = E[i], b = E[ixj];
          bool up = (i & k) == 0;
          if (up ? elem_less(b, a) : elem_less(a, b)) {
            E[i] = b;
            E[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void load_elems(Elem* E, const Rec* __restrict__ R, int base, int m, int P) {
  for (int i = threadIdx.x; i < P; i += kJBlock) {
    Elem e;
    if (i < m) {
      const Rec* r = R + base + i;
      e.t = (unsigned long long)r->ts ^ kSign64;
      e.idx = r->idx;
      e.pos = (uint32_t)(base + i);
    } else {
      e.t = ~0ull;
      e.idx = 0xFFFFFFFFu;
      e.pos = 0xFFFFFFFFu;
    }
    E[i] = e;
  }
  __syncthreads();
}

// Number of items taken from A among the first d outputs of merge(A, B).
__device__ __forceinline__ int merge_path(const Elem* A, int la, const Elem* B, int lb, int d) {
  int lo = max(0, d - lb), hi = min(d, la);
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (elem_less(A[mid], B[d - 1 - mid])) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Sorts a journey larger than kJCap: shared-memory bitonic sort of kJCap chunks, then rounds
// of CTA-wide merge-path merges between two global scratch buffers. Returns the buffer
// holding the sorted elements.
__device__ const Elem* sort_big(Elem* E, const Rec* __restrict__ R, int n, Elem* A, Elem* B) {
  for (int c0 = 0; c0 < n; c0 += kJCap) {
    int m = min(kJCap, n - c0);
    int P = 1;
    while (P < m) P <<= 1;
    load_elems(E, R, c0, m, P);
    bitonic_smem(E, P);
    for (int i = threadIdx.x; i < m; i += kJBlock) A[c0 + i] = E[i];
    __syncthreads();
  }
  Elem *src = A, *dst = B;
  for (int L = kJCap; L < n; L <<= 1) {
    for (int a0 = 0; a0 < n; a0 += 2 * L) {
      int la = min(L, n - a0);
      int lb = max(0, min(L, n - a0 - la));
      int total = la + lb;
      const Elem* SA = src + a0;
      const Elem* SB = SA + la;
      int d0 = (int)((long long)total * threadIdx.x / kJBlock);
      int d1 = (int)((long long)total * (threadIdx.x + 1) / kJBlock);
      int i = merge_path(SA, la, SB, lb, d0), j = d0 - i;
      for (int o = d0; o < d1; ++o) {
        if (i < la && (j >= lb || elem_less(SA[i], SB[j]))) dst[a0 + o] = SA[i++];
        else dst[a0 + o] = SB[j++];
      }
    }
    __syncthreads();
    Elem* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

// ---------------------------------------------------------------- the journey kernel
__device__ __forceinline__ void emit_run(const JourneyOut& o, DevState* st, uint32_t key, uint32_t cnt,
                                         double sum, float mn, float mx, uint32_t start) {
  uint32_t i = atomicAdd(&st->n_runs, 1u);
  if (i >= o.run_cap) {
    atomicOr(&st->err, kErrCapacity);
    return;
  }
  o.run_sortkey[i] = ((unsigned long long)key << 32) | start;
  o.run_cnt[i] = cnt;
  o.run_sum[i] = sum;
  o.run_min[i] = mn;
  o.run_max[i] = mx;
}

__global__ void __launch_bounds__(kJBlock) k_journeys(const Rec* __restrict__ rec,
                                                      const uint32_t* __restrict__ jn,
                                                      const uint32_t* __restrict__ joff, uint32_t J,
                                                      Elem* scrA, Elem* scrB, GridParams g,
                                                      JourneyOut o, DevState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Elem* E = reinterpret_cast<Elem*>(smem_raw);
  __shared__ int64_t e_ts[kJBlock / 32 + 1];
  __shared__ double e_lat[kJBlock / 32 + 1], e_lon[kJBlock / 32 + 1];
  __shared__ float e_spd[kJBlock / 32 + 1];
  __shared__ uint32_t s_key[kJBlock];
  __shared__ float s_spd[kJBlock];
  __shared__ uint32_t c_key, c_cnt, c_start, o_key, o_cnt, o_start;
  __shared__ double c_sum, o_sum;
  __shared__ float c_min, c_max, o_min, o_max;
  __shared__ double red_d[kJBlock / 32];
  __shared__ long long red_i[kJBlock / 32];
  __shared__ int64_t s_first_ts, s_last_ts;
  __shared__ double s_first_lat, s_first_lon, s_last_lat, s_last_lon;

  const uint32_t j = blockIdx.x;
  if (j >= J) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = (int)jn[j];
  const uint32_t off = joff[j];
  const Rec* R = rec + off;

  // 1. order the bucket by (timestamp, row index)
  const Elem* sorted;
  if (n <= kJCap) {
    int P = 1;
    while (P < n) P <<= 1;
    load_elems(E, R, 0, n, P);
    bitonic_smem(E, P);
    sorted = E;
  } else {
    if (tid == 0) atomicAdd(&st->n_big, 1u);
    sorted = sort_big(E, R, n, scrA + off, scrB + off);
  }

  if (tid == 0) {
    c_key = kKeyInvalid;
    o_key = kKeyInvalid;
    c_cnt = 0;
  }
  double dist = 0.0;
  long long dwell_sum = 0, n_dup = 0, n_off = 0;
  __syncthreads();

  // 2. walk the sorted journey, 256 points at a time
  for (int s0 = 0; s0 < n; s0 += kJBlock) {
    const int k = s0 + tid;
    const bool active = k < n;
    Rec cur;
    if (active) cur = R[sorted[k].pos];
    else {
      cur.ts = 0; cur.lat = 0.0; cur.lon = 0.0; cur.spd = 0.0f; cur.idx = 0;
    }
    // predecessor: the previous lane, or the previous warp's last lane, or the last point of
    // the previous slice (e_*[0])
    int64_t p_ts = __shfl_up_sync(0xffffffffu, cur.ts, 1);
    double p_lat = __shfl_up_sync(0xffffffffu, cur.lat, 1);
    double p_lon = __shfl_up_sync(0xffffffffu, cur.lon, 1);
    float p_spd = __shfl_up_sync(0xffffffffu, cur.spd, 1);
    if (lane == 31) {
      e_ts[warp + 1] = cur.ts;
      e_lat[warp + 1] = cur.lat;
      e_lon[warp + 1] = cur.lon;
      e_spd[warp + 1] = cur.spd;
    }
    __syncthreads();
    if (lane == 0) {
      p_ts = e_ts[warp];
      p_lat = e_lat[warp];
      p_lon = e_lon[warp];
      p_spd = e_spd[warp];
    }
    const uint32_t prevc = c_key;
    uint8_t fl = 0;
    double d = 0.0;
    float vh = 0.0f, ac = 0.0f;
    int64_t dw = 0;
    uint32_t key = kKeyInvalid;
    if (active) {
      if (k == 0) {
        fl |= kFStart;
        s_first_ts = cur.ts;
        s_first_lat = cur.lat;
        s_first_lon = cur.lon;
      } else {
        int64_t dt = (int64_t)((unsigned long long)cur.ts - (unsigned long long)p_ts);
        if (dt == 0) fl |= kFDup;
        d = haversine_m(p_lat, p_lon, cur.lat, cur.lon, g.radius_m);
        if (dt > 0) {
          double dts = (double)dt / 1000.0;
          vh = (float)(d / dts * 3.6);
          ac = (float)((((double)cur.spd - (double)p_spd) / 3.6) / dts);
        }
        if (p_spd < g.v_stop && cur.spd < g.v_stop) {
          fl |= kFStop;
          dw = dt;
        }
      }
      key = cell_key(cur.lat, cur.lon, cur.ts, g);
      if (key == kKeyInvalid) fl |= kFOffgrid;
      if (k == n - 1) {
        s_last_ts = cur.ts;
        s_last_lat = cur.lat;
        s_last_lon = cur.lon;
      }
      if (o.perm) {
        const uint32_t gp = off + (uint32_t)k;
        o.perm[gp] = cur.idx;
        o.d[gp] = d;
        o.vhat[gp] = vh;
        o.accel[gp] = ac;
        o.dwell_pt[gp] = dw;
        o.key[gp] = key;
        o.flags[gp] = fl;
      }
    }
    s_key[tid] = key;
    s_spd[tid] = cur.spd;
    // journey partial sums, in a fixed order
    double sd = block_sum<kJBlock, double>(d, red_d);
    long long sw = block_sum<kJBlock, long long>((long long)dw, red_i);
    long long sdup = block_sum<kJBlock, long long>((fl & kFDup) ? 1 : 0, red_i);
    long long soff = block_sum<kJBlock, long long>((active && key == kKeyInvalid) ? 1 : 0, red_i);
    if (tid == 0) {
      dist += sd;
      dwell_sum += sw;
      n_dup += sdup;
      n_off += soff;
    }
    // (block_sum ends with __syncthreads, so s_key / s_spd are visible here)
    // runs of equal valid keys: the carried run first (thread 0), then runs starting here
    if (tid == 0 && prevc != kKeyInvalid) {
      if (s_key[0] == prevc) {
        int e = 0;
        while (e < kJBlock && s_key[e] == prevc) {
          float v = s_spd[e];
          c_cnt += 1;
          c_sum += (double)v;
          c_min = fminf(c_min, v);
          c_max = fmaxf(c_max, v);
          ++e;
        }
        if (e < kJBlock) {
          emit_run(o, st, c_key, c_cnt, c_sum, c_min, c_max, c_start);
          c_key = kKeyInvalid;
        }
      } else {
        emit_run(o, st, c_key, c_cnt, c_sum, c_min, c_max, c_start);
        c_key = kKeyInvalid;
      }
    }
    const uint32_t mk = s_key[tid];
    const bool head = mk != kKeyInvalid && (tid == 0 ? mk != prevc : mk != s_key[tid - 1]);
    if (head) {
      int e = tid;
      uint32_t cnt = 0;
      double sum = 0.0;
      float mn = s_spd[tid], mx = s_spd[tid];
      while (e < kJBlock && s_key[e] == mk) {
        float v = s_spd[e];
        cnt += 1;
        sum += (double)v;
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
        ++e;
      }
      const uint32_t start = off + (uint32_t)(s0 + tid);
      if (e < kJBlock) {
        emit_run(o, st, mk, cnt, sum, mn, mx, start);
      } else {  // open at the slice end: becomes the carried run
        o_key = mk;
        o_cnt = cnt;
        o_sum = sum;
        o_min = mn;
        o_max = mx;
        o_start = start;
      }
    }
    __syncthreads();
    if (tid == 0 && o_key != kKeyInvalid) {
      c_key = o_key;
      c_cnt = o_cnt;
      c_sum = o_sum;
      c_min = o_min;
      c_max = o_max;
      c_start = o_start;
      o_key = kKeyInvalid;
    }
    if (tid == kJBlock - 1) {  // last point of this slice, for the next slice's first lane
      e_ts[0] = cur.ts;
      e_lat[0] = cur.lat;
      e_lon[0] = cur.lon;
      e_spd[0] = cur.spd;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (c_key != kKeyInvalid) emit_run(o, st, c_key, c_cnt, c_sum, c_min, c_max, c_start);
    o.n[j] = n;
    o.off[j] = off;
    o.start_ts[j] = s_first_ts;
    o.end_ts[j] = s_last_ts;
    o.duration[j] = (int64_t)((unsigned long long)s_last_ts - (unsigned long long)s_first_ts);
    o.dist[j] = dist;
    o.dwell[j] = dwell_sum;
    o.slat[j] = s_first_lat;
    o.slon[j] = s_first_lon;
    o.elat[j] = s_last_lat;
    o.elon[j] = s_last_lon;
    if (n_dup) atomicAdd(&st->n_dup, (unsigned long long)n_dup);
    if (n_off) atomicAdd(&st->n_offgrid, (unsigned long long)n_off);
  }
}

}  // namespace cvetl
