// journey.cuh — one CTA per journey: order the journey's bucket by (timestamp, row index),
// then walk it in sorted order computing per-point kinematics and the Algorithm 2 key, the
// journey summary, and the runs of equal cell x bin keys that feed the load stage.
#pragma once
#include "common.cuh"
#include "keying.cuh"

namespace cvetl {

// Two launch shapes of the journey kernel: 256 threads take journeys of any length; 64 threads
// take journeys of up to 512 points, with four times as many journeys resident per SM (a short
// journey leaves most of a 256-thread CTA idle through its sort and stitch barriers).
template <int NT>
struct JShape;
template <>
struct JShape<256> {
  static constexpr int kCap = 4096;     // records sorted in shared memory in one piece
  static constexpr int kEChunk = 2048;  // (timestamp, row) pairs sorted per shared-memory chunk (fallback)
  static constexpr int kRunBuf = 512;   // closed runs staged in shared memory
  static constexpr int kMinBlocks = 3;
};
// 512 threads (the staged sort of journeys of 4097-8192 points): the general sort's shape for its
// fallback when a time bucket is crowded (keys of up to 4096 points in shared memory, the
// (timestamp, row) pair sort above that)
template <>
struct JShape<512> {
  static constexpr int kCap = 4096;
  static constexpr int kEChunk = 4096;
  static constexpr int kRunBuf = 512;
  static constexpr int kMinBlocks = 1;
};
template <>
struct JShape<64> {
  static constexpr int kCap = 512;
  static constexpr int kEChunk = 256;
  static constexpr int kRunBuf = 128;
  static constexpr int kMinBlocks = 12;
};
constexpr int kJBlock = 256;   // threads per journey CTA (the shape for journeys of any length)
constexpr int kJSmallBlock = 64;
constexpr int kJCap = JShape<kJBlock>::kCap;
constexpr int kJSmallMax = JShape<kJSmallBlock>::kCap;  // longest journey of the 64-thread shape
constexpr int kBucketsBig = 12288;  // time buckets for journeys above kJCap (counters in shared memory)
static_assert(kJSmallBlock % 32 == 0 && kJBlock % kJSmallBlock == 0, "walk ranges: whole warps");

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
  int64_t* stop_ms;  // time since the current stop began
  float* accel_v;    // acceleration from the implied speeds
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

// ---------------------------------------------------------------- kinematics
// Haversine distance on a sphere of radius R; coordinates differenced in degrees first.
// General form with the CUDA math library (used for large steps).
__device__ __forceinline__ double haversine_m(double la1, double lo1, double la2, double lo2, double R) {
  const double rad = 0.017453292519943295;  // pi / 180
  double dphi = (la2 - la1) * rad, dlam = (lo2 - lo1) * rad;
  double s1 = sin(0.5 * dphi), s2 = sin(0.5 * dlam);
  double h = s1 * s1 + cos(la1 * rad) * cos(la2 * rad) * (s2 * s2);
  double r = fmin(sqrt(h), 1.0);
  return 2.0 * R * asin(r);
}

// ---------------------------------------------------------------- in-CTA sorting
template <int NT>
__device__ __forceinline__ void bitonic_smem(Elem* E, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += NT) {
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

template <int NT>
__device__ __forceinline__ void load_elems(Elem* E, const Rec* __restrict__ R, int base, int m, int P) {
  for (int i = threadIdx.x; i < P; i += NT) {
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

// Sorts a journey by (timestamp, row) pairs: shared-memory bitonic sort of kEChunk chunks, then rounds
// of CTA-wide merge-path merges between two global scratch buffers. Returns the buffer
// holding the sorted elements.
template <int NT>
__device__ const Elem* sort_big(Elem* E, const Rec* __restrict__ R, int n, Elem* A, Elem* B) {
  constexpr int kEChunk = JShape<NT>::kEChunk;
  for (int c0 = 0; c0 < n; c0 += kEChunk) {
    int m = min(kEChunk, n - c0);
    int P = 1;
    while (P < m) P <<= 1;
    load_elems<NT>(E, R, c0, m, P);
    bitonic_smem<NT>(E, P);
    for (int i = threadIdx.x; i < m; i += NT) A[c0 + i] = E[i];
    __syncthreads();
  }
  Elem *src = A, *dst = B;
  for (int L = kEChunk; L < n; L <<= 1) {
    for (int a0 = 0; a0 < n; a0 += 2 * L) {
      int la = min(L, n - a0);
      int lb = max(0, min(L, n - a0 - la));
      int total = la + lb;
      const Elem* SA = src + a0;
      const Elem* SB = SA + la;
      int d0 = (int)((long long)total * threadIdx.x / NT);
      int d1 = (int)((long long)total * (threadIdx.x + 1) / NT);
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

// ---------------------------------------------------------------- binary64 haversine, fast path
// For the sub-second steps of a journey the half-angles x = dphi/2 and y = dlambda/2 (radians)
// are tiny. With K = pi/360, u = dphi^2, v = dlambda^2 (degrees) and C = cos(lat1) cos(lat2),
// and |dphi|, |dlambda| < 0.0229 deg (|x|, |y| < 2e-4 rad, steps under ~2.5 km):
//   sin^2(x) = x^2 (1 - x^2/3) + O(x^6)            (dropped term < 2x^4/45 < 1e-16 relative)
//   h = sin^2 x + C sin^2 y = K^2 m (1 + eC - q),  m = u + C v,  q = K^2 (u^2 + C v^2) / (3m)
//   asin(s) = s (1 + h/6 + 3h^2/40) + O(s^7)
//   cos(lat0 + e) = c0 - s0 E - c0 E^2/2 + s0 E^3/6 + O(E^4), E = e pi/180, lat0 the nearest
//                   0.01 deg (|E| < 8.8e-5, dropped terms < 3e-18); eC collects the E^2, E^3
//                   terms of both cosines relative to C v / m
//   sqrt(m) = s sqrt(1 + r / s^2) = s (1 + p/2 + 3p^2/8) + O(p^3),  p = r / m,
//             s = sqrt_f32(m) correctly rounded,  r = m - s^2 (|p| <= 2^-23)
// so d = 2R asin(sqrt h) = 2R K s (1 + ds)(1 + dr) with
//   ds = p/2 + 3p^2/8,  dr = (eC - q)/2 + h/6 + 3h^2/40   (|ds| < 6e-8, |dr| < 2e-8).
// The coordinate differences and the cosine c0 - s0 e are binary64 (the differences are exact
// for nearby points); each is then split into a float32 pair h + l (48 significand bits) and
// the products, m, the residual r and the scaling by 2R K are evaluated as float32 pairs with
// error-free products (fmaf) and sums; the pair 2R K s (1 + ds + dr) is added up once in
// binary64. Each pair step has a relative error of a few 2^-48 and the small corrections ds,
// dr are float32 (below 5e-15 relative on d): d is within about 1e-14 of the haversine of the
// same binary64 inputs, as close as the all-binary64 evaluation of the series.
// That is 5 binary64 operations per point (cosine 2, differences 2, the final sum) on a part
// that runs about 1.7 of them per clock per SM against 128 float32 operations; the journey sum
// is kept in integer fixed point and the implied speed rounded to float32 by integer
// operations. Larger steps take the general formula through the CUDA math library.
constexpr double kRad = 0.017453292519943295;  // pi / 180
constexpr float kRadF = 0.017453292519943295f;
constexpr float kK2F = 7.615435494667714e-5f;  // (pi/360)^2
constexpr double kTinyDeg = 0.0229;           // |dphi|, |dlambda| below this take the series

// float -> double by the bit layout, exact for normal floats and zero (denormals read as zero),
// without a conversion instruction on the binary64 pipe.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t ex = (b >> 23) & 0xFFu;
  if (ex == 0) return __hiloint2double((int)(b & 0x80000000u), 0);
  const uint32_t hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// A value as the unevaluated sum h + l of two float32 (|l| <= ulp(h)).
struct F2 {
  float h, l;
};

// x = h + l by integer operations on the bit pattern: h the leading 24 significand bits of x
// rounded to nearest (ties up), l the rest rounded to float32 (|l| <= ulp(h) / 2, a relative
// error below 2^-48; exact when x has at most 48 significand bits), for finite
// 2^-74 <= |x| < 2^64; smaller x give h = l = 0.
__device__ __forceinline__ F2 split_f64(double x) {
  const unsigned long long b = dbits(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo32 = (uint32_t)b, ex = (hi >> 20) & 0x7FFu;
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t low29 = lo32 & 0x1FFFFFFFu;  // the bits below h's, in units of 2^(ex - 1075)
  const uint32_t up = low29 >> 28;            // the rest is at least half a unit of h
  const uint32_t hb = (sign | ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo32 >> 29)) + up;
  const float lo = __int2float_rn((int)low29 - (int)(up << 29)) * __uint_as_float((ex - 948u) << 23);
  const bool ok = ex >= 949u;
  F2 r;
  r.h = ok ? __uint_as_float(hb) : 0.0f;
  r.l = ok ? __uint_as_float(__float_as_uint(lo) ^ sign) : 0.0f;
  return r;
}

// Float32-pair steps with error-free products (the rounding error of a.h b.h by fmaf); the
// intrinsics keep the compiler from fusing a product that a later step takes as rounded.
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  F2 r;
  r.h = __fmul_rn(a.h, b.h);
  r.l = fmaf(a.l, b.l, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -r.h))));
  return r;
}
__device__ __forceinline__ F2 f2_sq(F2 a) {
  F2 r;
  r.h = __fmul_rn(a.h, a.h);
  r.l = fmaf(a.l, a.l, fmaf(a.h + a.h, a.l, fmaf(a.h, a.h, -r.h)));
  return r;
}
__device__ __forceinline__ F2 f2_add_pos(F2 a, F2 b) {  // a + b for a, b >= 0 (fast two-sum)
  const float big = fmaxf(a.h, b.h), small = fminf(a.h, b.h);
  F2 r;
  r.h = __fadd_rn(big, small);
  r.l = __fadd_rn(__fsub_rn(small, __fsub_rn(r.h, big)), __fadd_rn(a.l, b.l));
  return r;
}
__device__ __forceinline__ F2 f2_norm(F2 a) {  // the same value with |l| <= ulp(h) / 2
  F2 r;
  r.h = __fadd_rn(a.h, a.l);
  r.l = __fsub_rn(a.l, __fsub_rn(r.h, a.h));
  return r;
}

// cosine of a latitude: the binary64 value c0 - s0 E as a float32 pair, and the float32
// relative correction of the E^2 and E^3 terms
struct Cos64 {
  float h, l, eps;
};

__device__ __forceinline__ Cos64 cos64(double lat, const CosEntry* __restrict__ tab) {
  int k = __float2int_rn(leading_f32(lat) * 100.0f);
  k = max(-9000, min(9000, k));
  const double2* p = reinterpret_cast<const double2*>(tab + (k + 9000));
  const double2 t0 = __ldg(p), t1 = __ldg(p + 1);  // {lat0, cos}, {sin * pi/180, float32 copies}
  const double e = lat - t0.x;                      // degrees
  const F2 c2 = split_f64(fma(-t1.x, e, t0.y));
  Cos64 c;
  c.h = c2.h;
  c.l = c2.l;
  const unsigned long long cs = dbits(t1.y);  // {cos, sin * pi/180} rounded to float32
  const float c0f = __uint_as_float((uint32_t)cs), s0rf = __uint_as_float((uint32_t)(cs >> 32));
  const float ef = leading_f32(e), E = ef * kRadF;
  // -c0 E^2/2 + s0 E^3/6 = E^2 (s0r e / 6 - c0 / 2), relative to the value
  c.eps = __fdividef(E * E * fmaf(s0rf * ef, 1.0f / 6.0f, -0.5f * c0f), c.h);
  return c;
}

// |x| < kTinyDeg on the bit patterns (an integer compare, not a binary64 one; NaN fails).
__device__ __forceinline__ bool tiny_deg(double x) {
  return (dbits(x) & 0x7FFFFFFFFFFFFFFFull) < 0x3F977318FC504817ull;  // 0.0229
}

// A binary64 distance with its float32 rounding (the implied speed's input).
struct D64 {
  double d;
  float f;
  __device__ D64(int = 0) : d(0.0), f(0.0f) {}
  __device__ D64(double x, float xf) : d(x), f(xf) {}
  __device__ explicit operator double() const { return d; }
};

__device__ __forceinline__ float to_f32(double x) { return f64_to_f32_rn(x); }
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(const D64& x) { return x.f; }

__device__ __forceinline__ D64 haversine64(double la1, double lo1, const Cos64& c1, double la2,
                                              double lo2, const Cos64& c2, const GridParams& g) {
  const double dp = la2 - la1, dl = lo2 - lo1;  // exact for nearby points
  if (tiny_deg(dp) && tiny_deg(dl)) {
    const F2 dpp = split_f64(dp), dlp = split_f64(dl);
    const F2 u = f2_sq(dpp), v = f2_sq(dlp);
    const F2 C = f2_mul(F2{c1.h, c1.l}, F2{c2.h, c2.l});
    const F2 m = f2_norm(f2_add_pos(u, f2_mul(C, v)));
    const float mf = m.h;
    if (mf >= 1e-30f) {
      const float s = __fsqrt_rn(mf);
      const float t = __fmul_rn(s, s), te = fmaf(s, s, -t);  // s^2 = t + te
      const float r = __fadd_rn(__fsub_rn(mf, t), __fsub_rn(m.l, te));  // m - s^2 (mf - t exact)
      const float uf = u.h, vf = v.h, Cvf = c1.h * c2.h * vf;
      const float inv_m = __frcp_rn(mf);
      const float q = (kK2F / 3.0f) * fmaf(Cvf, vf, uf * uf) * inv_m;
      const float eC = Cvf * (c1.eps + c2.eps) * inv_m;
      const float hf = kK2F * mf;
      const float p = r * inv_m;
      const float ds = p * fmaf(0.375f, p, 0.5f);
      const float dr = fmaf(0.5f, eC - q, hf * fmaf(hf, 0.075f, 1.0f / 6.0f));
      const float delta = fmaf(ds, dr, ds + dr);
      const float dh = __fmul_rn(g.dist_kh, s);
      float dlo = fmaf(g.dist_kl, s, fmaf(g.dist_kh, s, -dh));
      dlo = fmaf(dh, delta, dlo);
      // exact: the pair spans under 53 bits; its float32 rounding is that of the sum
      return D64((double)dh + (double)dlo, __fadd_rn(dh, dlo));
    }
    if (((dbits(dp) | dbits(dl)) << 1) == 0) return D64();
  }
  const double x = haversine_m(la1, lo1, la2, lo2, g.radius_m);
  return D64(x, f64_to_f32_rn(x));
}

// ---------------------------------------------------------------- CTA-wide radix sort
// Stable LSD radix sort of n 64-bit keys (8-bit digits over bits [0, nbits)) by one CTA.
// A and B are shared memory for n <= kJCap (one tile), else global scratch (a journey's scratch stays in
// L2 while its CTA works on it). Ranking inside a 4096-key tile takes each digit's peer lanes
// (one ballot per digit bit) and their count below the lane, as the device-wide sort does; multi-tile passes add a digit histogram and carry running offsets
// from tile to tile in order, which keeps the sort stable.
constexpr int kRTile = 16 * kJBlock;  // keys ranked per tile: 16 per thread
constexpr int kBucketLoads = 8;        // keys or timestamps a thread reads at once in a counting pass

struct SortSmem {
  uint16_t wcnt[kJBlock / 32][256];
  uint32_t run[256];
  uint32_t scan[kJBlock / 32 + 1];
};

// static shared memory of the in-CTA sorts: the radix sort's with 256 threads, the bucket sort's
// scan scratch alone with 64
template <int NT>
struct JSort {
  struct Smem {
    uint32_t scan[NT / 32 + 1];
  };
};
template <>
struct JSort<kJBlock> {
  typedef SortSmem Smem;
};

__device__ unsigned long long* cta_radix_sort(unsigned long long* A, unsigned long long* B, int n,
                                              int nbits, SortSmem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool one_tile = n <= kRTile;
  for (int shift = 0; shift < nbits; shift += 8) {
    if (!one_tile) {
      sm.run[tid] = 0;
      __syncthreads();
      for (int i0 = tid; i0 < n; i0 += kJBlock * kBucketLoads) {  // keys read kBucketLoads at a time
        unsigned long long a[kBucketLoads];
#pragma unroll
        for (int u = 0; u < kBucketLoads; ++u) a[u] = i0 + u * kJBlock < n ? A[i0 + u * kJBlock] : 0ull;
#pragma unroll
        for (int u = 0; u < kBucketLoads; ++u)
          if (i0 + u * kJBlock < n) atomicAdd(&sm.run[(uint32_t)(a[u] >> shift) & 255u], 1u);
      }
      __syncthreads();
      uint32_t v = sm.run[tid];
      uint32_t e = block_excl_scan<kJBlock>(v, sm.scan, nullptr);
      sm.run[tid] = e;
      __syncthreads();
    }
    for (int t0 = 0; t0 < n; t0 += kRTile) {
      const int m = min(kRTile, n - t0);
      for (int i = tid; i < (kJBlock / 32) * 256; i += kJBlock) (&sm.wcnt[0][0])[i] = 0;
      __syncthreads();
      unsigned long long key[16];
      uint32_t rank[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int idx = warp * 512 + i * 32 + lane;
        key[i] = (idx < m) ? A[t0 + idx] : ~0ull;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const uint32_t d = (uint32_t)(key[i] >> shift) & 255u;
        const uint32_t peers = match_label<8>(d);
        const uint32_t before = sm.wcnt[warp][d];
        __syncwarp();
        if (lane == (__ffs(peers) - 1)) sm.wcnt[warp][d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        rank[i] = before + __popc(peers & lanemask_lt());
      }
      __syncthreads();
      uint32_t cnt = 0;
#pragma unroll
      for (int w = 0; w < kJBlock / 32; ++w) {
        const uint32_t c = sm.wcnt[w][tid];
        sm.wcnt[w][tid] = (uint16_t)cnt;
        cnt += c;
      }
      const uint32_t cnt_valid = cnt - ((tid == 255) ? (uint32_t)(kRTile - m) : 0u);
      uint32_t base;
      if (one_tile) base = block_excl_scan<kJBlock>(cnt, sm.scan, nullptr);
      else base = sm.run[tid];
      __syncthreads();
      sm.run[tid] = base;  // this tile's first output position per digit
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int idx = warp * 512 + i * 32 + lane;
        if (idx < m) {
          const uint32_t d = (uint32_t)(key[i] >> shift) & 255u;
          B[sm.run[d] + sm.wcnt[warp][d] + rank[i]] = key[i];
        }
      }
      __syncthreads();
      if (!one_tile) {
        sm.run[tid] = base + cnt_valid;
        __syncthreads();
      }
    }
    unsigned long long* t = A;
    A = B;
    B = t;
  }
  return A;
}

// Counting sort of a journey's keys by a monotone time bucket, then insertion sort inside each
// bucket (up to four or eight keys: loaded together and put in order by a 5- or 19-step
// network), equal timestamps (always in one bucket) ordered by extracted-row index. Timestamps of a journey are spread almost evenly over its span (regular sampling),
// so with about one bucket per point the buckets hold a few keys each and the sort is O(n).
// bucket(t) = min(nb - 1, floor(float(t) * nb / (span + 1))) is non-decreasing in t, so the
// buckets' concatenation is in key order once each bucket is sorted. Returns false when some
// bucket holds more than kMaxBucket keys (then the caller uses the radix sort). cnt: nb
// counters in shared memory. The sorted keys end in B.
constexpr int kMaxBucket = 48;

// Bucket of a time offset t in [0, span]: a journey spanning under 2^32 ms (any real one)
// converts through 32 bits, which gives the same float as the 64-bit conversion.
__device__ __forceinline__ int time_bucket(unsigned long long t, bool narrow, float scale, int nb) {
  const float f = narrow ? __uint2float_rz((uint32_t)t) : u64_to_f32_rz_rare(t);
  return min(nb - 1, (int)(f * scale));
}

// The keys are rebuilt from the journey's records on each pass (the records stay in L2), so
// that only the output buffer B takes shared memory.
__device__ __forceinline__ unsigned long long rec_key(const Rec* __restrict__ R, int i,
                                                      unsigned long long tmin, int pos_bits) {
  return ((((unsigned long long)R[i].ts ^ kSign64) - tmin) << pos_bits) | (unsigned long long)i;
}

__device__ __forceinline__ void cswap(unsigned long long& a, unsigned long long& b) {
  const unsigned long long x = min(a, b), y = max(a, b);
  a = x;
  b = y;
}

template <int NT>
__device__ bool cta_bucket_sort_rec(const Rec* __restrict__ R, unsigned long long tmin, int pos_bits,
                                    unsigned long long* B, int n, unsigned long long span,
                                    uint32_t* cnt, int nb, uint32_t* scan_scratch, int* flag) {
  const int tid = threadIdx.x;
  const float scale = (float)nb / ((float)span + 1.0f);
  const bool narrow = span <= 0xFFFFFFFFull;
  for (int i = tid; i < nb; i += NT) cnt[i] = 0;
  __syncthreads();
  // the records' timestamps are read kBucketLoads at a time (independent loads in flight)
  for (int i0 = tid; i0 < n; i0 += NT * kBucketLoads) {
    unsigned long long t[kBucketLoads];
#pragma unroll
    for (int u = 0; u < kBucketLoads; ++u) {
      const int i = i0 + u * NT;
      t[u] = i < n ? (unsigned long long)R[i].ts : 0ull;
    }
#pragma unroll
    for (int u = 0; u < kBucketLoads; ++u)
      if (i0 + u * NT < n) atomicAdd(&cnt[time_bucket((t[u] ^ kSign64) - tmin, narrow, scale, nb)], 1u);
  }
  __syncthreads();
  const int chunk = (nb + NT - 1) / NT;
  const int c0 = min(nb, tid * chunk), c1 = min(nb, c0 + chunk);
  uint32_t sum = 0, mx = 0;
  for (int i = c0; i < c1; ++i) {
    sum += cnt[i];
    mx = max(mx, cnt[i]);
  }
  if (tid == 0) *flag = 0;
  uint32_t base = block_excl_scan<NT>(sum, scan_scratch, nullptr);
  if (mx > (uint32_t)kMaxBucket) *flag = 1;
  for (int i = c0; i < c1; ++i) {
    const uint32_t v = cnt[i];
    cnt[i] = base;
    base += v;
  }
  __syncthreads();
  if (*flag) return false;
  for (int i0 = tid; i0 < n; i0 += NT * kBucketLoads) {
    unsigned long long t[kBucketLoads];
#pragma unroll
    for (int u = 0; u < kBucketLoads; ++u) {
      const int i = i0 + u * NT;
      t[u] = i < n ? (unsigned long long)R[i].ts : 0ull;
    }
#pragma unroll
    for (int u = 0; u < kBucketLoads; ++u) {
      const int i = i0 + u * NT;
      if (i < n) {
        const unsigned long long d = (t[u] ^ kSign64) - tmin;
        B[atomicAdd(&cnt[time_bucket(d, narrow, scale, nb)], 1u)] = (d << pos_bits) | (unsigned long long)i;
      }
    }
  }
  __syncthreads();
  // Each bucket in key order, then equal timestamps (which share a bucket) by extracted-row
  // index, as fix_ties does for the other sorts.
  const unsigned long long pmask = (1ull << pos_bits) - 1;
  for (int b = tid; b < nb; b += NT) {
    const int lo = b ? (int)cnt[b - 1] : 0, hi = (int)cnt[b];
    if (hi - lo <= 1) continue;
    if (hi - lo <= 4) {  // up to four keys: loaded together, sorted in registers
      unsigned long long v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = lo + q < hi ? B[lo + q] : ~0ull;
      cswap(v[0], v[1]);
      cswap(v[2], v[3]);
      cswap(v[0], v[2]);
      cswap(v[1], v[3]);
      cswap(v[1], v[2]);
      bool tie = false;
#pragma unroll
      for (int q = 0; q < 3; ++q) tie |= lo + q + 1 < hi && (v[q] >> pos_bits) == (v[q + 1] >> pos_bits);
      if (tie) {  // odd-even transposition by (timestamp, row index)
        uint32_t x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = lo + q < hi ? R[v[q] & pmask].idx : 0xFFFFFFFFu;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = r & 1; q < 3; q += 2)
            if ((v[q] >> pos_bits) == (v[q + 1] >> pos_bits) && x[q] > x[q + 1]) {
              const unsigned long long tv = v[q];
              v[q] = v[q + 1];
              v[q + 1] = tv;
              const uint32_t tx = x[q];
              x[q] = x[q + 1];
              x[q + 1] = tx;
            }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (lo + q < hi) B[lo + q] = v[q];
      continue;
    }
    if (hi - lo <= 8) {  // up to eight keys: Batcher's 19-step network in registers
      unsigned long long v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = lo + q < hi ? B[lo + q] : ~0ull;
      cswap(v[0], v[1]); cswap(v[2], v[3]); cswap(v[4], v[5]); cswap(v[6], v[7]);
      cswap(v[0], v[2]); cswap(v[1], v[3]); cswap(v[4], v[6]); cswap(v[5], v[7]);
      cswap(v[1], v[2]); cswap(v[5], v[6]);
      cswap(v[0], v[4]); cswap(v[1], v[5]); cswap(v[2], v[6]); cswap(v[3], v[7]);
      cswap(v[2], v[4]); cswap(v[3], v[5]);
      cswap(v[1], v[2]); cswap(v[3], v[4]); cswap(v[5], v[6]);
      bool tie = false;
#pragma unroll
      for (int q = 0; q < 7; ++q) tie |= lo + q + 1 < hi && (v[q] >> pos_bits) == (v[q + 1] >> pos_bits);
      if (tie) {  // odd-even transposition by (timestamp, row index)
        uint32_t x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = lo + q < hi ? R[v[q] & pmask].idx : 0xFFFFFFFFu;
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int q = r & 1; q < 7; q += 2)
            if ((v[q] >> pos_bits) == (v[q + 1] >> pos_bits) && x[q] > x[q + 1]) {
              const unsigned long long tv = v[q];
              v[q] = v[q + 1];
              v[q + 1] = tv;
              const uint32_t tx = x[q];
              x[q] = x[q + 1];
              x[q + 1] = tx;
            }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (lo + q < hi) B[lo + q] = v[q];
      continue;
    }
    bool tie = false;
    for (int i = lo + 1; i < hi; ++i) {
      const unsigned long long v = B[i];
      int q = i - 1;
      while (q >= lo && B[q] > v) {
        B[q + 1] = B[q];
        --q;
      }
      B[q + 1] = v;
    }
    for (int i = lo + 1; i < hi; ++i) tie |= (B[i - 1] >> pos_bits) == (B[i] >> pos_bits);
    if (tie) {  // insertion by (timestamp, row index)
      for (int i = lo + 1; i < hi; ++i) {
        const unsigned long long v = B[i];
        const uint32_t vi = R[v & pmask].idx;
        int q = i - 1;
        while (q >= lo && (B[q] >> pos_bits) == (v >> pos_bits) && R[B[q] & pmask].idx > vi) {
          B[q + 1] = B[q];
          --q;
        }
        B[q + 1] = v;
      }
    }
  }
  __syncthreads();
  return true;
}

// Keys are ((ts - tmin) << pos_bits) | slot. Points with equal timestamps are ordered by the
// slot (arbitrary) here; reorder each such group by extracted-row index.
template <int NT>
__device__ void fix_ties(unsigned long long* K, int n, int pos_bits, const Rec* __restrict__ R) {
  const unsigned long long mask = (1ull << pos_bits) - 1;
  for (int k = threadIdx.x; k < n; k += NT) {
    const unsigned long long t = K[k] >> pos_bits;
    const bool lead = (k + 1 < n && (K[k + 1] >> pos_bits) == t) && (k == 0 || (K[k - 1] >> pos_bits) != t);
    if (lead) {
      int e = k + 1;
      while (e < n && (K[e] >> pos_bits) == t) ++e;
      for (int i = k + 1; i < e; ++i) {  // insertion sort by row index
        const unsigned long long v = K[i];
        const uint32_t vi = R[v & mask].idx;
        int q = i - 1;
        while (q >= k && R[K[q] & mask].idx > vi) {
          K[q + 1] = K[q];
          --q;
        }
        K[q + 1] = v;
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- the journey kernel
// Speed sums of a run: compensated float32 pairs (Neumaier's variant of Kahan summation; the
// error stays below ~2^-45 relative for runs of any practical length), folded into binary64
// once per run.
__device__ __forceinline__ void fsum_add(float& s, float& c, float v) {
  const float t = s + v;
  c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
  s = t;
}

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

__device__ __forceinline__ int bits_for(unsigned long long v) { return v ? 64 - __clzll(v) : 0; }

// ---------------------------------------------------------------- the two arithmetic forms
// Binary64 form: the distance is evaluated in binary64 throughout (haversine_fast above).
// Float32 form: the coordinates are differenced in binary64 (exact for nearby points) and
// rounded to float32; the bulk of the haversine, the cosines and the per-point arithmetic run
// in float32; the journey distance is summed in compensated float32 pairs. Keys, counts and
// the order are the same integer computation in both forms.
constexpr float kHalfRadF = 0.0087266462599716f;  // pi / 360

__device__ __forceinline__ float haversine_f32(double la1, double lo1, float c1, double la2, double lo2,
                                               float c2, const GridParams& g) {
  const float a = leading_f32(la2 - la1) * kHalfRadF;
  const float b = leading_f32(lo2 - lo1) * kHalfRadF;
  const float R2 = (float)g.asin_c1;
  if (fabsf(a) < 1e-2f && fabsf(b) < 1e-2f) {
    // sin^2 x = x^2 (1 - x^2/3) + O(x^6); asin s = s (1 + h/6 + 3 h^2/40) + O(s^7), h = s^2
    const float a2 = a * a, b2 = b * b;
    const float h = fmaf(c1 * c2, b2 * fmaf(b2, -1.0f / 3.0f, 1.0f), a2 * fmaf(a2, -1.0f / 3.0f, 1.0f));
    const float s = sqrtf(h);
    return R2 * s * fmaf(h, fmaf(h, 0.075f, 1.0f / 6.0f), 1.0f);
  }
  const float sa = sinf(a), sb = sinf(b);
  return R2 * asinf(fminf(1.0f, sqrtf(fmaf(c1 * c2, sb * sb, sa * sa))));
}

struct Fp64Form {
  typedef Cos64 Cos;
  typedef D64 Dist;
  // the per-point rates (implied speed, acceleration): float32 quotients by the fast division
  // (within 2 ulp, far inside the rates' 1e-6 tolerance)
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ Cos64 cosine(double lat, const GridParams& g) {
    return cos64(lat, g.cos_tab);
  }
  static __device__ __forceinline__ D64 distance(double la1, double lo1, const Cos64& c1, double la2,
                                                 double lo2, const Cos64& c2, const GridParams& g) {
    return haversine64(la1, lo1, c1, la2, lo2, c2, g);
  }
  // A lane's distance sum in 128-bit fixed point (units of 2^-64 m), off the binary64 pipe: each
  // distance is truncated to a multiple of 2^-64 m (under 5.5e-20 m lost per point) and the sums
  // are exact, so they do not depend on the order of their terms. Distances are non-negative and
  // below 2^63 m.
  struct Acc {
    unsigned long long lo = 0, hi = 0;
    __device__ __forceinline__ void add(const D64& x) { add(x.d); }
    __device__ __forceinline__ void add(double d) {
      const unsigned long long b = dbits(d);
      const int e = (int)((b >> 52) & 0x7FFull);
      const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const int sh = e - 1011;  // d * 2^64 = m * 2^sh
      unsigned long long vlo, vhi;
      if (sh > 0 && sh < 64) {  // 2^-11 m <= d < 2^52 m
        vhi = m >> (64 - sh);
        vlo = m << sh;
      } else if (e == 0 || sh <= -64) {  // zero, or below 2^-64 m
        vhi = 0;
        vlo = 0;
      } else if (sh <= 0) {
        vhi = 0;
        vlo = m >> (-sh);
      } else {
        vhi = m << min(sh - 64, 10);
        vlo = 0;
      }
      add_fixed(vlo, vhi);
    }
    __device__ __forceinline__ void add_fixed(unsigned long long vlo, unsigned long long vhi) {
      const unsigned long long nlo = lo + vlo;
      hi += vhi + (nlo < lo ? 1ull : 0ull);
      lo = nlo;
    }
    // hi + lo 2^-64, within one unit in the last place
    __device__ __forceinline__ double value() const {
      return (double)hi + __ull2double_rn(lo) * 5.421010862427522e-20;
    }
    // the warp's total (valid in lane 0): the lanes' sums added exactly, then rounded
    __device__ __forceinline__ double warp_total() const {
      Acc a = *this;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        a.add_fixed(__shfl_down_sync(0xffffffffu, a.lo, o), __shfl_down_sync(0xffffffffu, a.hi, o));
      return a.value();
    }
  };
};

struct Fp32Form {
  typedef float Cos;
  typedef float Dist;
  // the per-point rates by the fast float32 division (within 2 ulp)
  static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  // cos(lat) from the nearest 0.01-degree table point: c0 - s0 E (E the offset in radians, under
  // 8.8e-5; the dropped E^2 term is below 4e-9 relative)
  static __device__ __forceinline__ float cosine(double lat, const GridParams& g) {
    const float lf = leading_f32(lat);
    const int k = max(-9000, min(9000, __float2int_rn(lf * 100.0f)));
    const float2 cs = __ldg(reinterpret_cast<const float2*>(&g.cos_tab[k + 9000].c0f));
    return fmaf(-cs.y, lf - (float)k * 0.01f, cs.x);
  }
  static __device__ __forceinline__ float distance(double la1, double lo1, float c1, double la2,
                                                   double lo2, float c2, const GridParams& g) {
    return haversine_f32(la1, lo1, c1, la2, lo2, c2, g);
  }
  struct Acc {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float d) { fsum_add(s, c, d); }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
    // the warp's total (valid in lane 0), by a fixed shuffle tree
    __device__ __forceinline__ double warp_total() const { return warp_sum(value()); }
  };
};

// device-resident state of every journey seen so far, indexed by its slot in the journey hash
struct JState {
  int64_t *n, *start_ts, *end_ts, *dwell;
  double *dist, *slat, *slon;
  // last finalised point: the predecessor of the journey's next point
  int64_t* l_ts;
  double *l_lat, *l_lon;
  float* l_spd;
  uint32_t* l_key;
  // run of equal keys still open at the last finalised point
  uint32_t *r_cnt;
  float *r_s, *r_c, *r_mn, *r_mx;
};

// Run fragments a thread hands to the stitch at the end of the walk.
struct RunPart {
  uint32_t key, cnt, start;
  float s, c, mn, mx;
};

__device__ __forceinline__ void run_add(RunPart& r, float v) {
  r.cnt += 1;
  fsum_add(r.s, r.c, v);
  r.mn = fminf(r.mn, v);
  r.mx = fmaxf(r.mx, v);
}
__device__ __forceinline__ void run_merge(RunPart& r, const RunPart& q) {
  r.cnt += q.cnt;
  fsum_add(r.s, r.c, q.s);
  r.c += q.c;
  r.mn = fminf(r.mn, q.mn);
  r.mx = fmaxf(r.mx, q.mx);
}

template <int NT>
struct StitchSmem {
  RunPart pre[NT];  // run continuing from the previous thread's range (cnt 0: none)
  RunPart suf[NT];  // run open at the end of the range
  uint8_t has[NT];  // the thread had points
  uint8_t cont[NT]; // the whole range continued the previous thread's run
};

// Closed runs are staged in shared memory (the bucket counters' space, free once the journey
// is sorted) and written out with one global allocation per journey; a journey with more runs
// than the buffer holds emits the rest directly.
struct __align__(8) RunSlot {
  float s, c;  // compensated speed sum, folded into binary64 at the copy-out (not in the walk)
  uint32_t key, cnt, start;
  float mn, mx;
  uint32_t pad;
};

// Dynamic shared memory of the journey kernel: the sort keys of a journey of up to kCap points,
// then its kCap bucket counters; once the journey is sorted the run buffer takes the counters'
// space (and the stitch arrays the keys'). Journeys above kCap (256 threads only) keep their
// keys in global scratch and use the whole space for kBucketsBig counters.
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
template <int NT>
__host__ __device__ constexpr int jrunbuf_off() {
  return cmax(cmax(JShape<NT>::kCap * 8, JShape<NT>::kEChunk * 16), (int)sizeof(StitchSmem<NT>));
}
template <int NT>
__host__ __device__ constexpr int jsmem() {
  return cmax(JShape<NT>::kCap * 12, jrunbuf_off<NT>() + JShape<NT>::kRunBuf * (int)sizeof(RunSlot));
}
constexpr int kJSmem = jsmem<kJBlock>();
constexpr int kJSmallSmem = jsmem<kJSmallBlock>();
static_assert(kJSmem == kJCap * 12, "journey kernel shared memory as sized for 256 threads");
static_assert(kBucketsBig * 4 <= kJSmem, "bucket counters must fit the dynamic shared memory");
static_assert(JShape<kJSmallBlock>::kCap * 12 <= kJSmallSmem, "keys and counters must fit");

template <int NT>
__device__ __forceinline__ void run_put(RunSlot* buf, uint32_t* nbuf, const JourneyOut& o, DevState* st,
                                        const RunPart& r) {
  if (r.key == kKeyInvalid || r.cnt == 0) return;
  const uint32_t i = atomicAdd(nbuf, 1u);
  if (i < (uint32_t)JShape<NT>::kRunBuf) {
    RunSlot& q = buf[i];
    q.s = r.s;
    q.c = r.c;
    q.key = r.key;
    q.cnt = r.cnt;
    q.start = r.start;
    q.mn = r.mn;
    q.mx = r.mx;
  } else {
    emit_run(o, st, r.key, r.cnt, (double)r.s + (double)r.c, r.mn, r.mx, r.start);
  }
}

// ---- stitching the threads' run fragments in parallel
// Thread t of the walk acts on the run left open before its range as one of two maps:
// continue (its whole range has the open run's key: open <- open + X) or reset (emit
// open + X, then open <- S, the run open at the end of its range). Maps compose
// associatively (continue.continue = continue with X1 + X2; continue.reset = reset with
// X1 + X2; reset.continue = reset with S1 + X2; reset.reset = reset keeping X1, S2, the run
// S1 + X2 in between being emitted by its owner), so one warp scans them: each lane folds
// nr / 32 consecutive walk ranges (nr = 64 or 256), an exclusive warp scan gives each lane its
// incoming open run, and each lane then replays its ranges, emitting as the serial order would.
__device__ __forceinline__ RunPart run_empty() {
  return RunPart{kKeyInvalid, 0u, 0u, 0.f, 0.f, __int_as_float(0x7F800000), __int_as_float((int)0xFF800000u)};
}

__device__ __forceinline__ RunPart rp_merge(RunPart a, const RunPart& b) {
  if (b.cnt == 0) return a;
  if (a.cnt == 0) return b;
  run_merge(a, b);
  return a;
}

struct RunMap {
  uint32_t reset;
  RunPart X, S;
};

__device__ __forceinline__ RunMap map_then(RunMap f, const RunMap& g) {
  if (!g.reset) {
    if (!f.reset) f.X = rp_merge(f.X, g.X);
    else f.S = rp_merge(f.S, g.X);
    return f;
  }
  RunMap r;
  r.reset = 1u;
  r.X = f.reset ? f.X : rp_merge(f.X, g.X);
  r.S = g.S;
  return r;
}

__device__ __forceinline__ RunPart shfl_up_rp(const RunPart& r, int d) {
  RunPart o;
  o.key = __shfl_up_sync(0xffffffffu, r.key, d);
  o.cnt = __shfl_up_sync(0xffffffffu, r.cnt, d);
  o.start = __shfl_up_sync(0xffffffffu, r.start, d);
  o.s = __shfl_up_sync(0xffffffffu, r.s, d);
  o.c = __shfl_up_sync(0xffffffffu, r.c, d);
  o.mn = __shfl_up_sync(0xffffffffu, r.mn, d);
  o.mx = __shfl_up_sync(0xffffffffu, r.mx, d);
  return o;
}

__device__ __forceinline__ RunMap shfl_up_map(const RunMap& f, int d) {
  RunMap o;
  o.reset = __shfl_up_sync(0xffffffffu, f.reset, d);
  o.X = shfl_up_rp(f.X, d);
  o.S = shfl_up_rp(f.S, d);
  return o;
}

// Called by warp 0 only, over the nr walk ranges (a multiple of 32). Returns, in lane 31, the
// run open after the journey's last point.
template <int NT>
__device__ RunPart stitch_runs(const StitchSmem<NT>& ss, int nr, const RunPart& init, RunSlot* buf,
                               uint32_t* nbuf, const JourneyOut& o, DevState* st) {
  const int kPer = nr / 32;
  const int lane = threadIdx.x & 31, t0 = lane * kPer;
  RunMap f{0u, run_empty(), run_empty()};
#pragma unroll 1
  for (int t = t0; t < t0 + kPer; ++t) {
    if (!ss.has[t]) continue;
    const RunMap g{ss.cont[t] ? 0u : 1u, ss.pre[t], ss.suf[t]};
    f = map_then(f, g);
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const RunMap q = shfl_up_map(f, d);
    if (lane >= d) f = map_then(q, f);
  }
  RunMap ex = shfl_up_map(f, 1);
  if (lane == 0) ex = RunMap{0u, run_empty(), run_empty()};
  RunPart open = ex.reset ? ex.S : rp_merge(init, ex.X);
#pragma unroll 1
  for (int t = t0; t < t0 + kPer; ++t) {
    if (!ss.has[t]) continue;
    if (ss.cont[t]) {
      open = rp_merge(open, ss.pre[t]);
    } else {
      run_put<NT>(buf, nbuf, o, st, rp_merge(open, ss.pre[t]));
      open = ss.suf[t];
    }
  }
  return open;
}

// The journey's bucket R[0..n) in (timestamp, row index) order: either the sorted keys K
// (((ts - tmin) << pos_bits) | bucket position; position = K[k] & pmask) or, when the keys do not
// fit 64 bits or a 64-thread CTA meets crowded buckets, the sorted (timestamp, row) pairs E.
struct JSorted {
  const unsigned long long* K;
  const Elem* E;
  unsigned long long pmask;
  __device__ __forceinline__ uint32_t pos(int k) const { return K ? (uint32_t)(K[k] & pmask) : E[k].pos; }
};

// Sorts one journey by the whole CTA (every thread calls it). Uses the dynamic shared memory
// (keys of up to kCap points and their bucket counters) and, above kCap, the journey's slice of
// the global scratch scrA / scrB. Ends with a barrier.
template <int NT>
__device__ __forceinline__ JSorted journey_sort(const Rec* __restrict__ R, int n, uint32_t off, Elem* scrA,
                                                Elem* scrB, DevState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kCap = JShape<NT>::kCap;
  __shared__ typename JSort<NT>::Smem ssort;
  __shared__ unsigned long long s_tmin, s_tmax;
  __shared__ int s_flag;
  const int tid = threadIdx.x, lane = tid & 31;
  const bool small = n <= kCap;  // always, with 64 threads
  // 1. order the bucket by (timestamp, row index)
  // 1a. range of the timestamps (as order-preserving keys)
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int i = tid; i < n; i += NT) {
    const unsigned long long t = (unsigned long long)R[i].ts ^ kSign64;
    lo = min(lo, t);
    hi = max(hi, t);
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o2));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o2));
  }
  if (tid == 0) {
    s_tmin = ~0ull;
    s_tmax = 0ull;
  }
  __syncthreads();
  if (lane == 0) {
    atomicMin(&s_tmin, lo);
    atomicMax(&s_tmax, hi);
  }
  __syncthreads();
  const unsigned long long tmin = s_tmin;
  const int pos_bits = max(1, bits_for((unsigned long long)(n > 1 ? n - 1 : 1)));
  const int nbits = pos_bits + bits_for(s_tmax - tmin);
  // keyed: the sort keys below fit 64 bits and the journey was sorted by them; otherwise it is
  // sorted as (timestamp, row) pairs
  bool keyed = nbits <= 64;
  const unsigned long long* sortedK = nullptr;
  const Elem* sortedE = nullptr;
  if (keyed) {
    // 1b. keys ((ts - tmin) << pos_bits) | slot: counting sort by time bucket into shared memory
    // (global scratch above kCap); when buckets are crowded, a radix sort through global scratch
    // (256 threads) or the pair sort (64 threads); ties by row index
    unsigned long long* KB = small ? reinterpret_cast<unsigned long long*>(smem_raw)
                                   : reinterpret_cast<unsigned long long*>(scrB + off);
    uint32_t* cnt = small ? reinterpret_cast<uint32_t*>(smem_raw + kCap * sizeof(unsigned long long))
                          : reinterpret_cast<uint32_t*>(smem_raw);
    const int nb = small ? max(1, n) : min(n, kBucketsBig);
    unsigned long long* K = nullptr;
    bool ties_done = false;  // the time-bucket sort orders equal timestamps by row index itself
    if (n <= kBucketsBig * 8 &&
        cta_bucket_sort_rec<NT>(R, tmin, pos_bits, KB, n, s_tmax - tmin, cnt, nb, ssort.scan, &s_flag)) {
      K = KB;
      ties_done = true;
    } else if constexpr (NT == kJBlock) {
      unsigned long long* GA = reinterpret_cast<unsigned long long*>(scrA + off);
      unsigned long long* GB = reinterpret_cast<unsigned long long*>(scrB + off);
      for (int i = tid; i < n; i += NT) GA[i] = rec_key(R, i, tmin, pos_bits);
      __syncthreads();
      K = cta_radix_sort(GA, GB, n, nbits, ssort);
    } else {
      keyed = false;
    }
    if (keyed) {
      if (!ties_done) fix_ties<NT>(K, n, pos_bits, R);
      sortedK = K;
    }
  }
  if (!keyed) {
    // timestamps spanning more than 2^(64 - pos_bits) ms (counted), or crowded buckets with
    // 64 threads: compare (timestamp, row) pairs
    if (tid == 0 && nbits > 64) atomicAdd(&st->n_big, 1u);
    sortedE = sort_big<NT>(reinterpret_cast<Elem*>(smem_raw), R, n, scrA + off, scrB + off);
  }
  __syncthreads();
  return JSorted{sortedK, sortedE, (1ull << pos_bits) - 1};
}


// One journey (rank j) by the whole CTA. Ends with every thread past its last shared-memory use
// of this journey except the run copy-out (the caller synchronises before the next journey).
template <class Form, int NT>
__device__ __forceinline__ void journey_one(uint32_t j, const Rec* __restrict__ rec,
                                            const uint32_t* __restrict__ jn,
                                            const uint32_t* __restrict__ joff, Elem* scrA, Elem* scrB,
                                            const GridParams& g, const Batch& bt, const JourneyOut& o,
                                            DevState* st,
                                            const uint32_t* __restrict__ jslot, const JState& js) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kRunBuf = JShape<NT>::kRunBuf;
  __shared__ double red_d[NT / 32];
  __shared__ long long red_i[3][NT / 32];
  __shared__ int64_t s_first_ts, s_last_ts;
  __shared__ double s_first_lat, s_first_lon, s_last_lat, s_last_lon;
  __shared__ float s_last_spd;
  __shared__ uint32_t s_last_key;
  __shared__ uint32_t s_nbuf, s_base;
  __shared__ RunPart s_open;
  constexpr int kRunBufOff = jrunbuf_off<NT>();
  RunSlot* rbuf = reinterpret_cast<RunSlot*>(smem_raw + kRunBufOff);

  const int tid = threadIdx.x, lane = tid & 31;
  const int n = (int)jn[j];
  const uint32_t off = joff[j];
  const Rec* R = rec + off;
  // the grid and day the journey's points are keyed on (a journey lies in one batch instance)
  const BatchInst* bi = bt.n_inst ? bt.inst + inst_of_row(bt, R[0].idx) : nullptr;
  // stream mode: the journey continues from its state (last point, open run, running sums)
  const bool stream = js.n != nullptr;
  const uint32_t slot = stream ? jslot[j] : 0u;
  const bool has_prev = stream && js.n[slot] > 0;

  if (tid == 0) s_nbuf = 0u;
  // 1. order the bucket by (timestamp, row index)
  const JSorted srt = journey_sort<NT>(R, n, off, scrA, scrB, st);
  const bool keyed = srt.K != nullptr;
  const unsigned long long* sortedK = srt.K;
  const Elem* sortedE = srt.E;
  const unsigned long long pmask = srt.pmask;

  // 2. walk: thread t owns the sorted positions [k0, k1) and visits them in order; the
  // predecessor stays in registers, runs of equal keys accumulate in the thread
  // The ranges, and with them every rounding of the journey's sums, depend on n alone: a journey
  // of up to 512 points is walked as 64 ranges by either kernel shape, a longer one as 256.
  const int nr = (NT == kJSmallBlock || n <= kJSmallMax) ? kJSmallBlock : NT;
  const int k0 = tid < nr ? (int)((long long)n * tid / nr) : n;
  const int k1 = tid < nr ? (int)((long long)n * (tid + 1) / nr) : n;
  typename Form::Acc dist;
  long long dwell_sum = 0, n_dup = 0, n_off = 0;
  RunPart pre{kKeyInvalid, 0u, 0u, 0.f, 0.f, 0.f, 0.f};
  RunPart run{kKeyInvalid, 0u, 0u, 0.f, 0.f, 0.f, 0.f};
  bool in_pre = false;  // the open run continues the previous thread's last run
  bool cont_all = false;
  if (k0 < k1) {
    int64_t p_ts = 0;
    double p_lat = 0.0, p_lon = 0.0;
    typename Form::Cos p_cos{};
    float p_spd = 0.0f;
    if (k0 > 0) {  // predecessor: the previous thread's last point
      const Rec q = R[keyed ? (uint32_t)(sortedK[k0 - 1] & pmask) : sortedE[k0 - 1].pos];
      p_ts = q.ts;
      p_lat = q.lat;
      p_lon = q.lon;
      p_spd = q.spd;
      p_cos = Form::cosine(q.lat, g);
      run.key = point_key(q.lat, q.lon, q.ts, g, bi);
      run.mn = __int_as_float(0x7F800000);   // +inf
      run.mx = __int_as_float((int)0xFF800000u);  // -inf
      in_pre = true;  // an empty fragment of the previous thread's run
    } else if (has_prev) {  // predecessor: the journey's last point of an earlier window
      p_ts = js.l_ts[slot];
      p_lat = js.l_lat[slot];
      p_lon = js.l_lon[slot];
      p_spd = js.l_spd[slot];
      p_cos = Form::cosine(p_lat, g);
      run.key = js.l_key[slot];
      run.mn = __int_as_float(0x7F800000);
      run.mx = __int_as_float((int)0xFF800000u);
      in_pre = true;
    }
    // the next record is loaded one point ahead and the position of the one after it two, so
    // that neither load waits on the other within an iteration
    uint32_t nxt_p = keyed ? (uint32_t)(sortedK[k0] & pmask) : sortedE[k0].pos;
    Rec nxt = R[nxt_p];
    if (k0 + 1 < k1) nxt_p = keyed ? (uint32_t)(sortedK[k0 + 1] & pmask) : sortedE[k0 + 1].pos;
    for (int k = k0; k < k1; ++k) {
      const Rec cur = nxt;
      if (k + 1 < k1) nxt = R[nxt_p];
      if (k + 2 < k1) nxt_p = keyed ? (uint32_t)(sortedK[k + 2] & pmask) : sortedE[k + 2].pos;
      const typename Form::Cos ccur = Form::cosine(cur.lat, g);
      const uint32_t key = point_key(cur.lat, cur.lon, cur.ts, g, bi);
      uint8_t fl = 0;
      typename Form::Dist d = 0;
      float vh = 0.0f, ac = 0.0f;
      int64_t dw = 0;
      if (k == 0) {
        s_first_ts = cur.ts;
        s_first_lat = cur.lat;
        s_first_lon = cur.lon;
      }
      if (k == 0 && !has_prev) {
        fl |= kFStart;
      } else {
        const int64_t dt = (int64_t)((unsigned long long)cur.ts - (unsigned long long)p_ts);
        if (dt == 0) fl |= kFDup;
        d = Form::distance(p_lat, p_lon, p_cos, cur.lat, cur.lon, ccur, g);
        if (dt > 0) {
          // stored as float32: computed in float32 from the binary64 distance
          const float fdt = (dt <= 0x7FFFFFFFll) ? (float)(int32_t)dt : i64_to_f32_rare(dt);
          vh = to_f32(d) * Form::div(3600.0f, fdt);
          ac = Form::div(cur.spd - p_spd, 0.0036f * fdt);
        }
        if (p_spd < g.v_stop && cur.spd < g.v_stop) {
          fl |= kFStop;
          dw = dt;
        }
      }
      if (key == kKeyInvalid) fl |= kFOffgrid;
      if (o.perm) {
        const uint32_t gp = off + (uint32_t)k;
        o.perm[gp] = cur.idx;
        o.d[gp] = (double)d;
        o.vhat[gp] = vh;
        o.accel[gp] = ac;
        o.dwell_pt[gp] = dw;
        o.key[gp] = key;
        o.flags[gp] = fl;
      }
      dist.add(d);
      dwell_sum += dw;
      n_dup += (fl & kFDup) ? 1 : 0;
      n_off += (key == kKeyInvalid) ? 1 : 0;
      // runs of equal keys (the first fragment may continue the previous thread's run)
      if (k > k0 || in_pre) {
        if (key == run.key) {
          run_add(run, cur.spd);
          p_ts = cur.ts; p_lat = cur.lat; p_lon = cur.lon; p_cos = ccur; p_spd = cur.spd;
          continue;
        }
        if (in_pre) {
          pre = run;
          in_pre = false;
        } else {
          run_put<NT>(rbuf, &s_nbuf, o, st, run);
        }
      }
      run = RunPart{key, 1u, off + (uint32_t)k, cur.spd, 0.f, cur.spd, cur.spd};
      p_ts = cur.ts; p_lat = cur.lat; p_lon = cur.lon; p_cos = ccur; p_spd = cur.spd;
    }
    if (k1 == n) {
      s_last_ts = p_ts;
      s_last_lat = p_lat;
      s_last_lon = p_lon;
      s_last_spd = p_spd;
      s_last_key = run.key;
    }
    if (in_pre) {  // no key change in the whole range
      pre = run;
      cont_all = true;
    }
  }
  // 3. journey sums in a fixed order; stitch run fragments across thread ranges in order
  // (the four block sums in one pass: each value takes the warp tree and then the warps in
  // order, as block_sum does; the totals are valid in thread 0)
  double sd = warp_sum(dist.value());
  long long sw = warp_sum(dwell_sum), sdup = warp_sum(n_dup), soff = warp_sum(n_off);
  if (lane == 0) {
    red_d[tid >> 5] = sd;
    red_i[0][tid >> 5] = sw;
    red_i[1][tid >> 5] = sdup;
    red_i[2][tid >> 5] = soff;
  }
  __syncthreads();
  if (tid == 0) {
    sd = 0.0;
    sw = sdup = soff = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
      sd += red_d[w];
      sw += red_i[0][w];
      sdup += red_i[1][w];
      soff += red_i[2][w];
    }
  }
  StitchSmem<NT>& ss = *reinterpret_cast<StitchSmem<NT>*>(smem_raw);  // the sort buffers are done
  ss.pre[tid] = pre;
  ss.suf[tid] = run;
  ss.has[tid] = k0 < k1;
  ss.cont[tid] = cont_all;
  __syncthreads();
  if (tid < 32) {
    // the run left open by the last window continues here, under this window's offset
    const RunPart init = has_prev ? RunPart{js.l_key[slot], js.r_cnt[slot], off, js.r_s[slot], js.r_c[slot],
                                            js.r_mn[slot], js.r_mx[slot]}
                                  : run_empty();
    const RunPart open = stitch_runs<NT>(ss, nr, init, rbuf, &s_nbuf, o, st);
    if (tid == 31) s_open = open;
  }
  __syncthreads();
  if (tid == 0) {
    const RunPart open = s_open;
    if (stream) {  // the open run and the journey's sums stay on the device
      if (!has_prev) {
        js.start_ts[slot] = s_first_ts;
        js.slat[slot] = s_first_lat;
        js.slon[slot] = s_first_lon;
      }
      js.n[slot] += n;
      js.end_ts[slot] = s_last_ts;
      js.dist[slot] += sd;
      js.dwell[slot] += sw;
      js.l_ts[slot] = s_last_ts;
      js.l_lat[slot] = s_last_lat;
      js.l_lon[slot] = s_last_lon;
      js.l_spd[slot] = s_last_spd;
      js.l_key[slot] = s_last_key;
      const bool keep = open.key != kKeyInvalid;
      js.r_cnt[slot] = keep ? open.cnt : 0u;
      js.r_s[slot] = open.s;
      js.r_c[slot] = open.c;
      js.r_mn[slot] = open.mn;
      js.r_mx[slot] = open.mx;
    } else {
      run_put<NT>(rbuf, &s_nbuf, o, st, open);
      o.n[j] = n;
      o.off[j] = off;
      o.start_ts[j] = s_first_ts;
      o.end_ts[j] = s_last_ts;
      o.duration[j] = (int64_t)((unsigned long long)s_last_ts - (unsigned long long)s_first_ts);
      o.dist[j] = sd;
      o.dwell[j] = sw;
      o.slat[j] = s_first_lat;
      o.slon[j] = s_first_lon;
      o.elat[j] = s_last_lat;
      o.elon[j] = s_last_lon;
    }
    if (sdup) atomicAdd(&st->n_dup, (unsigned long long)sdup);
    if (soff) atomicAdd(&st->n_offgrid, (unsigned long long)soff);
    const uint32_t nb = min(s_nbuf, (uint32_t)kRunBuf);
    s_base = nb ? atomicAdd(&st->n_runs, nb) : 0u;
  }
  __syncthreads();
  // the staged runs, written out together
  const uint32_t nb = min(s_nbuf, (uint32_t)kRunBuf), base = s_base;
  for (uint32_t i = tid; i < nb; i += NT) {
    const uint32_t g = base + i;
    if (g >= o.run_cap) {
      atomicOr(&st->err, kErrCapacity);
      break;
    }
    const RunSlot q = rbuf[i];
    o.run_sortkey[g] = ((unsigned long long)q.key << 32) | q.start;
    o.run_cnt[g] = q.cnt;
    o.run_sum[g] = (double)q.s + (double)q.c;
    o.run_min[g] = q.mn;
    o.run_max[g] = q.mx;
  }
}

// The journey kernel. Persistent: each CTA takes the next journey of the work list `order`
// (journey ranks, longest first, so that the long journeys of an uneven batch start early and
// the short ones fill the tail) through the work counter until the list is exhausted.
// With wend, the persistent kernel stops at the list's first *wend journeys. Otherwise CTA b takes
// journey order[b] (rank b without a list): the block scheduler's
// dispatch order then gives the same longest-first start without the loop.
// split > 0 shares the journeys between the two shapes: those of up to min(split, 512) points
// go to the 64-thread kernel (which takes the list from its short end), the rest to the
// 256-thread kernel; each skips the other's journeys. Both run over the same list.
template <int NT>
__device__ __forceinline__ bool journey_mine(uint32_t n, uint32_t split) {
  const uint32_t lim = min(split, (uint32_t)kJSmallMax);
  if constexpr (NT == kJBlock) return split == 0 || n > lim;
  else return n <= lim;
}

template <class Form, bool Persistent, int NT>
__global__ void __launch_bounds__(NT, JShape<NT>::kMinBlocks) k_journeys(
    const Rec* __restrict__ rec, const uint32_t* __restrict__ jn, const uint32_t* __restrict__ joff, uint32_t J,
    Elem* scrA, Elem* scrB, GridParams g, Batch bt, JourneyOut o, DevState* st,
    const uint32_t* __restrict__ jslot, JState js, const uint32_t* __restrict__ order, uint32_t* work,
    uint32_t split, const uint32_t* __restrict__ wend = nullptr) {
  if constexpr (!Persistent) {
    if (blockIdx.x >= J) return;
    const uint32_t w = (NT == kJBlock) ? blockIdx.x : J - 1 - blockIdx.x;
    const uint32_t j = order ? order[w] : blockIdx.x;
    if (journey_mine<NT>(jn[j], split)) journey_one<Form, NT>(j, rec, jn, joff, scrA, scrB, g, bt, o, st, jslot, js);
  } else {
    static_assert(!Persistent || NT == kJBlock, "persistent CTAs take the 256-thread shape");
    __shared__ uint32_t s_w;
    const uint32_t w1 = wend ? *wend : J;  // the list's first w1 journeys (all without wend)
    for (;;) {
      if (threadIdx.x == 0) s_w = atomicAdd(work, 1u);
      __syncthreads();
      const uint32_t w = s_w;
      __syncthreads();
      if (w >= w1) break;
      const uint32_t j = order ? order[w] : w;
      if (!journey_mine<NT>(jn[j], split)) {
        if (order) break;  // longest first: the rest of the list is the 64-thread kernel's
        continue;
      }
      journey_one<Form, NT>(j, rec, jn, joff, scrA, scrB, g, bt, o, st, jslot, js);
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- batch path: sort, then walk
// Journeys of up to 8192 points: the batch path orders each journey's bucket by (timestamp,
// row) (k_journey_sort_class, one persistent grid per size class) and writes only the order,
// the bucket positions as u16; one warp per journey then walks the bucketed records through
// those positions (k_journey_walk), at the occupancy that suits the walk rather than the sort.
// Writing the order instead of a second, ordered record array halves the sort's time; the walk
// pays with gathered reads (each lane its own 32-byte record) instead of coalesced ones.

__device__ __forceinline__ void ld_rec(const Rec* p, unsigned long long& a, unsigned long long& b,
                                       unsigned long long& c, unsigned long long& d) {
  asm("ld.global.v4.b64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}
// The same, for records read once (the walk): no L1 allocation, so the stream of records does
// not evict the grid tables and cosine entries every point looks up.
__device__ __forceinline__ void ld_rec_once(const Rec* p, unsigned long long& a, unsigned long long& b,
                                            unsigned long long& c, unsigned long long& d) {
  asm("ld.global.L1::no_allocate.v4.b64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}
__device__ __forceinline__ void st_rec(Rec* p, unsigned long long a, unsigned long long b, unsigned long long c,
                                       unsigned long long d) {
  asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d) : "memory");
}

// ---- staged sort: the journey's timestamps held in shared memory
// A journey of n <= CAP points (CAP <= 65536): one pass loads its timestamps (as order-preserving
// keys) into shared memory T; a counting sort by time bucket (about two points per bucket)
// places the u16 positions P; an insertion sort by (timestamp, row index) finishes each bucket;
// the records are then copied to `out` in that order. Shared memory: T (8 B), P (2 B) and the
// bucket counters (4 B per two points): 12 * CAP bytes. Returns false, having written nothing,
// when a bucket holds more than kMaxBucket points (the caller then takes the general sort).
template <int CAP>
__host__ __device__ constexpr int staged_smem() { return CAP * 12; }

__device__ __forceinline__ bool staged_less(const unsigned long long* T, const Rec* __restrict__ R, uint32_t a,
                                            uint32_t b) {
  const unsigned long long ta = T[a], tb = T[b];
  return ta < tb || (ta == tb && R[a].idx < R[b].idx);
}

// The points k = 0..m-1 with order-preserving timestamps T[k] in [tmin, tmax], ordered by
// (timestamp, row index) into the u16 array O: a counting sort by time bucket (max(1, m/2)
// buckets, about two points each), then an insertion sort inside each bucket; idx_of(k) gives a
// point's row index (read only for equal timestamps). cnt: max(1, m/2) u32 counters. Returns
// false, with O unset, when a bucket holds more than kMaxBucket points. Every thread of the CTA
// calls it; ends with a barrier.
template <int NT, class IdxOf>
__device__ bool staged_order(const unsigned long long* T, int m, unsigned long long tmin, unsigned long long tmax,
                             uint16_t* O, uint32_t* cnt, uint32_t* s_scan, int* s_flag, IdxOf idx_of) {
  const int tid = threadIdx.x;
  const int nb = max(1, m >> 1);
  const unsigned long long span = tmax - tmin;
  const bool narrow = span <= 0xFFFFFFFFull;
  const float scale = (float)nb / ((float)span + 1.0f);
  for (int b = tid; b < nb; b += NT) cnt[b] = 0;
  if (tid == 0) *s_flag = 0;
  __syncthreads();
  for (int i = tid; i < m; i += NT) atomicAdd(&cnt[time_bucket(T[i] - tmin, narrow, scale, nb)], 1u);
  __syncthreads();
  // bucket offsets (each thread a contiguous chunk of buckets); crowded buckets detected
  const int chunk = (nb + NT - 1) / NT;
  const int c0 = min(nb, tid * chunk), c1 = min(nb, c0 + chunk);
  uint32_t sum = 0, mx = 0;
  for (int b = c0; b < c1; ++b) {
    sum += cnt[b];
    mx = max(mx, cnt[b]);
  }
  uint32_t base = block_excl_scan<NT>(sum, s_scan, nullptr);
  if (mx > (uint32_t)kMaxBucket) *s_flag = 1;
  for (int b = c0; b < c1; ++b) {
    const uint32_t v = cnt[b];
    cnt[b] = base;
    base += v;
  }
  __syncthreads();
  if (*s_flag) return false;
  // positions by bucket (cnt[b] ends as the end of bucket b)
  for (int i = tid; i < m; i += NT) O[atomicAdd(&cnt[time_bucket(T[i] - tmin, narrow, scale, nb)], 1u)] = (uint16_t)i;
  __syncthreads();
  // each bucket by (timestamp, row index)
  for (int b = tid; b < nb; b += NT) {
    const int b0 = b ? (int)cnt[b - 1] : 0, b1 = (int)cnt[b];
    for (int i = b0 + 1; i < b1; ++i) {
      const uint16_t v = O[i];
      const unsigned long long tv = T[v];
      int q = i - 1;
      while (q >= b0) {
        const unsigned long long tq = T[O[q]];
        if (tq < tv || (tq == tv && idx_of(O[q]) < idx_of(v))) break;
        O[q + 1] = O[q];
        --q;
      }
      O[q + 1] = v;
    }
  }
  __syncthreads();
  return true;
}

// Block-wide range of the threads' [lo, hi] into *s_lo, *s_hi (set to ~0 and 0 by the caller
// before a barrier); ends with a barrier.
__device__ __forceinline__ void block_range(unsigned long long lo, unsigned long long hi, unsigned long long* s_lo,
                                            unsigned long long* s_hi) {
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o2));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o2));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(s_lo, lo);
    atomicMax(s_hi, hi);
  }
  __syncthreads();
}

// The staged order of the journey's bucket R[0..n) into the u16 positions P (at 8 * CAP bytes
// into the dynamic shared memory, valid until the CTA's next use of it); false when a time
// bucket is crowded. Once its timestamps are read, the nn records at Rn (the CTA's next
// journey, or none) are prefetched into L2, so that its own load finds them there. Every thread
// of the CTA calls it; ends with a barrier.
template <int NT, int CAP>
__device__ bool staged_journey_order(const Rec* __restrict__ R, int n, const Rec* Rn = nullptr, int nn = 0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* T = reinterpret_cast<unsigned long long*>(smem_raw);
  uint16_t* P = reinterpret_cast<uint16_t*>(smem_raw + 8 * CAP);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(smem_raw + 10 * CAP);
  __shared__ unsigned long long s_tmin, s_tmax;
  __shared__ uint32_t s_scan[NT / 32 + 1];
  __shared__ int s_flag;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_tmin = ~0ull;
    s_tmax = 0ull;
  }
  // the timestamps, once, into shared memory; their range
  unsigned long long lo = ~0ull, hi = 0ull;
#pragma unroll 4
  for (int i = tid; i < n; i += NT) {
    const unsigned long long t = (unsigned long long)R[i].ts ^ kSign64;
    T[i] = t;
    lo = min(lo, t);
    hi = max(hi, t);
  }
  // the next journey's records into L2 (one prefetch per 128-byte line) while this one sorts
  for (int i = tid; i < (nn + 3) / 4; i += NT)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(Rn + 4 * i));
  __syncthreads();
  block_range(lo, hi, &s_tmin, &s_tmax);
  return staged_order<NT>(T, n, s_tmin, s_tmax, P, cnt, s_scan, &s_flag, [R](int k) { return R[k].idx; });
}
template <int CAP>
__device__ __forceinline__ const uint16_t* staged_positions() {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return reinterpret_cast<const uint16_t*>(smem_raw + 8 * CAP);
}

// Journey size classes over the work list (sizes non-increasing along it): bounds[c] is the
// first list position of class c, bounds[4] = J; classes: above 8192 points, 4097-8192,
// 513-4096, up to 512. One warp per class boundary (96 threads): a 32-way search, each round
// probing 32 evenly spaced positions of the range that holds the boundary and keeping the part
// between the last probe below the class limit's side and the first at or under it (about
// four rounds of two dependent loads for 60,000 journeys, against 16 for a binary search).
__device__ __forceinline__ uint32_t sort_class_max(int c) { return c == 0 ? 8192u : (c == 1 ? 4096u : 512u); }
__global__ void k_size_classes(const uint32_t* __restrict__ jn, const uint32_t* __restrict__ order, uint32_t J,
                               uint32_t* __restrict__ bounds, uint32_t* __restrict__ work) {
  if (blockIdx.x != 0) return;
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    bounds[0] = 0;
    bounds[4] = J;
  }
  if (threadIdx.x < 4) work[threadIdx.x] = 0;
  if (c >= 3) return;
  const uint32_t lim = sort_class_max(c);
  // the first w with jn[order[w]] <= lim lies in [lo, hi] (hi = J: none)
  uint32_t lo = 0, hi = J;
  while (lo < hi) {
    const uint32_t step = (hi - lo + 31) / 32;
    // the last lane probes hi - 1
    const uint32_t q = (uint32_t)min((unsigned long long)lo + (unsigned long long)(lane + 1) * step - 1,
                                     (unsigned long long)hi - 1);
    const uint32_t under = __ballot_sync(0xffffffffu, jn[order[q]] <= lim);
    if (under == 0) {
      lo = hi;  // every position below hi is above the limit
    } else {
      const int f = __ffs(under) - 1;
      const uint32_t qf = __shfl_sync(0xffffffffu, q, f);
      const uint32_t qp = __shfl_sync(0xffffffffu, q, f > 0 ? f - 1 : 0);
      hi = qf;
      if (f > 0) lo = qp + 1;
    }
  }
  if (lane == 0) bounds[c + 1] = lo;
}

// One size class of the journey sort, persistent: CTAs take the class's journeys in list order
// through its work counter, each claim one journey ahead of the one sorted (whose records are
// prefetched into L2 meanwhile): the staged sort, falling back to the general sort when a time
// bucket is crowded. (Journeys above 8192 points take the fused journey kernel.)
template <int NT, int CAP>
__host__ __device__ constexpr int sort_class_min_blocks() { return NT == 64 ? 12 : (CAP > 4096 ? 2 : 3); }

template <int NT, int CAP>
__global__ void __launch_bounds__(NT, sort_class_min_blocks<NT, CAP>()) k_journey_sort_class(const Rec* __restrict__ rec, const uint32_t* __restrict__ jn,
                                                           const uint32_t* __restrict__ joff,
                                                           const uint32_t* __restrict__ order,
                                                           const uint32_t* __restrict__ bounds, int cls,
                                                           uint32_t* work, Elem* scrA, Elem* scrB,
                                                           uint16_t* __restrict__ spos, DevState* st) {
  __shared__ uint32_t s_w, s_wn;
  const uint32_t w0 = bounds[cls], w1 = bounds[cls + 1];
  uint32_t wc = 0;
  if (threadIdx.x == 0) wc = w0 + atomicAdd(work, 1u);
  for (;;) {
    // the next journey is claimed one ahead, so that its records can be fetched during this one
    if (threadIdx.x == 0) {
      s_w = wc;
      s_wn = wc < w1 ? w0 + atomicAdd(work, 1u) : w1;
      wc = s_wn;
    }
    __syncthreads();
    const uint32_t w = s_w, wn = s_wn;
    __syncthreads();
    if (w >= w1) break;
    const uint32_t j = order[w];
    const int n = (int)jn[j];
    const uint32_t off = joff[j];
    const Rec* R = rec + off;
    const Rec* Rn = nullptr;
    int nn = 0;
    if (wn < w1) {
      const uint32_t jn2 = order[wn];
      Rn = rec + joff[jn2];
      nn = (int)jn[jn2];
    }
    if (staged_journey_order<NT, CAP>(R, n, Rn, nn)) {
      const uint16_t* P = staged_positions<CAP>();
      for (int k = threadIdx.x; k < n; k += NT) spos[off + k] = P[k];
    } else {
      const JSorted srt = journey_sort<NT>(R, n, off, scrA, scrB, st);
      for (int k = threadIdx.x; k < n; k += NT) spos[off + k] = (uint16_t)srt.pos(k);
    }
    __syncthreads();
  }
}

// Runs of equal keys inside one warp's iteration: compensated speed sum, min, max (a run's
// count follows from its first and last positions).
struct RunAgg {
  float s, c, mn, mx;
};
__device__ __forceinline__ RunAgg agg_then(const RunAgg& a, const RunAgg& b) {  // a before b
  RunAgg r;
  r.s = a.s;
  r.c = a.c;
  fsum_add(r.s, r.c, b.s);
  r.c += b.c;
  r.mn = fminf(a.mn, b.mn);
  r.mx = fmaxf(a.mx, b.mx);
  return r;
}
// Shuffles of the per-point cosine of the two forms.
__device__ __forceinline__ Cos64 shfl_cos(const Cos64& c, int src) {
  Cos64 r;
  r.h = __shfl_sync(0xffffffffu, c.h, src);
  r.l = __shfl_sync(0xffffffffu, c.l, src);
  r.eps = __shfl_sync(0xffffffffu, c.eps, src);
  return r;
}
__device__ __forceinline__ float shfl_cos(float c, int src) { return __shfl_sync(0xffffffffu, c, src); }
__device__ __forceinline__ Cos64 shfl_up_cos(const Cos64& c, int d) {
  Cos64 r;
  r.h = __shfl_up_sync(0xffffffffu, c.h, d);
  r.l = __shfl_up_sync(0xffffffffu, c.l, d);
  r.eps = __shfl_up_sync(0xffffffffu, c.eps, d);
  return r;
}
__device__ __forceinline__ float shfl_up_cos(float c, int d) { return __shfl_up_sync(0xffffffffu, c, d); }

constexpr int kWalkBlock = 128;
constexpr int kWalkRunCap = 64;  // closed runs staged per warp before they are written out

// A warp's closed runs, staged in shared memory and written out kWalkRunCap at a time with one
// global allocation (an atomic on the run counter) per batch of runs.
__device__ __forceinline__ void walk_flush(RunSlot* buf, uint32_t& nbuf, const JourneyOut& o, DevState* st) {
  const int lane = threadIdx.x & 31;
  if (nbuf == 0) return;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(&st->n_runs, nbuf);
  base = __shfl_sync(0xffffffffu, base, 0);
  __syncwarp();
  for (uint32_t i = lane; i < nbuf; i += 32) {
    const uint32_t gi = base + i;
    if (gi >= o.run_cap) {
      atomicOr(&st->err, kErrCapacity);
      break;
    }
    const RunSlot q = buf[i];
    o.run_sortkey[gi] = ((unsigned long long)q.key << 32) | q.start;
    o.run_cnt[gi] = q.cnt;
    o.run_sum[gi] = (double)q.s + (double)q.c;
    o.run_min[gi] = q.mn;
    o.run_max[gi] = q.mx;
  }
  __syncwarp();
  nbuf = 0;
}

// Warp sum of a run aggregate in a fixed shuffle tree (lane 0 holds the result).
__device__ __forceinline__ RunAgg warp_agg(RunAgg a) {
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    RunAgg q;
    q.s = __shfl_down_sync(0xffffffffu, a.s, o2);
    q.c = __shfl_down_sync(0xffffffffu, a.c, o2);
    q.mn = __shfl_down_sync(0xffffffffu, a.mn, o2);
    q.mx = __shfl_down_sync(0xffffffffu, a.mx, o2);
    a = agg_then(a, q);
  }
  return a;
}

__device__ __forceinline__ RunAgg agg_empty() {
  return RunAgg{0.f, 0.f, __int_as_float(0x7F800000), __int_as_float((int)0xFF800000u)};
}
__device__ __forceinline__ void agg_add(RunAgg& a, float v) {
  fsum_add(a.s, a.c, v);
  a.mn = fminf(a.mn, v);
  a.mx = fmaxf(a.mx, v);
}

// Stages one closed run (lane 0 of the warp writes it) and flushes the warp's buffer when full.
__device__ __forceinline__ void walk_put(RunSlot* buf, uint32_t& nbuf, const JourneyOut& o, DevState* st,
                                         uint32_t key, uint32_t start, uint32_t cnt, const RunAgg& a) {
  if (nbuf == (uint32_t)kWalkRunCap) walk_flush(buf, nbuf, o, st);
  if ((threadIdx.x & 31) == 0) {
    RunSlot& q = buf[nbuf];
    q.s = a.s;
    q.c = a.c;
    q.key = key;
    q.cnt = cnt;
    q.start = start;
    q.mn = a.mn;
    q.mx = a.mx;
  }
  nbuf += 1;
  __syncwarp();
}

// The walk of journey j (n points at srec[off ..)) by one warp. Iteration t takes points
// 32t + lane; a point's predecessor is the previous lane's point (a shuffle), lane 0's the last
// point of the previous iteration (carried). Every per-journey sum and run aggregate is formed in
// an order fixed by the points' positions alone: each lane sums its own points in order, and the
// lanes' partial sums are added by a fixed shuffle tree (at the journey's end for the journey
// sums, when a run closes for the run aggregates: a run's points in one lane accumulate in that
// lane until the warp reduces the run).
template <class Form>
__device__ __forceinline__ void walk_journey(uint32_t j, const Rec* __restrict__ S, const uint16_t* __restrict__ P,
                                             int n, uint32_t off,
                                             const GridParams& g, const Batch& bt, const JourneyOut& o,
                                             DevState* st, RunSlot* rbuf, uint32_t& nbuf,
                                             unsigned long long& n_dup, unsigned long long& n_off,
                                             const unsigned long long* sthr) {
  const int lane = threadIdx.x & 31;
  const BatchInst* bi = bt.n_inst ? bt.inst + inst_of_row(bt, S[0].idx) : nullptr;
  typename Form::Acc dist;
  long long dwell = 0;
  uint32_t dup = 0, offg = 0;
  // the last point of the previous iteration (valid from the second iteration on)
  int64_t c_ts = 0;
  double c_lat = 0.0, c_lon = 0.0;
  float c_spd = 0.0f;
  typename Form::Cos c_cos{};
  uint32_t c_key = kKeyInvalid;
  int64_t first_ts = 0;
  // the run open after the previous iteration: key and first position (warp-uniform), and this
  // lane's share of its points
  uint32_t o_key = kKeyInvalid, o_start = 0;
  RunAgg la = agg_empty();
  // records one iteration ahead, their bucket positions two
  unsigned long long na = 0, nb = 0, nc = 0, nd = 0;
  if (lane < n) ld_rec_once(S + P[lane], na, nb, nc, nd);
  uint32_t pn = (32 + lane < n) ? P[32 + lane] : 0u;
  for (int base = 0; base < n; base += 32) {
    const int k = base + lane;
    const bool valid = k < n;
    const unsigned long long ra = na, rb = nb, rc = nc, rd = nd;
    if (k + 32 < n) ld_rec_once(S + pn, na, nb, nc, nd);
    if (k + 64 < n) pn = P[k + 64];
    const int64_t ts = (int64_t)ra;
    const double lat = dfrom(rb), lon = dfrom(rc);
    const float spd = __uint_as_float((uint32_t)rd);
    const uint32_t idx = (uint32_t)(rd >> 32);
    typename Form::Cos ccur{};
    uint32_t key = kKeyInvalid;
    if (valid) {
      ccur = Form::cosine(lat, g);
      key = sthr ? cell_key<true>(lat, lon, ts, g, sthr, sthr + g.n_rows + 1) : point_key(lat, lon, ts, g, bi);
    }
    // predecessor: the previous lane's point, or the carried one
    int64_t p_ts = (int64_t)__shfl_up_sync(0xffffffffu, (unsigned long long)ts, 1);
    double p_lat = __shfl_up_sync(0xffffffffu, lat, 1), p_lon = __shfl_up_sync(0xffffffffu, lon, 1);
    float p_spd = __shfl_up_sync(0xffffffffu, spd, 1);
    typename Form::Cos p_cos = shfl_up_cos(ccur, 1);
    uint32_t p_key = __shfl_up_sync(0xffffffffu, key, 1);
    if (lane == 0) {
      p_ts = c_ts;
      p_lat = c_lat;
      p_lon = c_lon;
      p_spd = c_spd;
      p_cos = c_cos;
      p_key = c_key;
    }
    if (base == 0) first_ts = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)ts, 0);
    if (valid) {
      uint8_t fl = 0;
      typename Form::Dist d = 0;
      float vh = 0.0f, ac = 0.0f;
      int64_t dw = 0;
      if (k == 0) {
        fl |= kFStart;
      } else {
        const int64_t dt = (int64_t)((unsigned long long)ts - (unsigned long long)p_ts);
        if (dt == 0) fl |= kFDup;
        d = Form::distance(p_lat, p_lon, p_cos, lat, lon, ccur, g);
        if (dt > 0) {
          const float fdt = (dt <= 0x7FFFFFFFll) ? (float)(int32_t)dt : i64_to_f32_rare(dt);
          vh = to_f32(d) * Form::div(3600.0f, fdt);
          ac = Form::div(spd - p_spd, 0.0036f * fdt);
        }
        if (p_spd < g.v_stop && spd < g.v_stop) {
          fl |= kFStop;
          dw = dt;
        }
      }
      if (key == kKeyInvalid) fl |= kFOffgrid;
      dist.add(d);
      dwell += dw;
      dup += (fl & kFDup) ? 1u : 0u;
      offg += (key == kKeyInvalid) ? 1u : 0u;
      const uint32_t gp = off + (uint32_t)k;
      if (o.perm) {
        o.perm[gp] = idx;
        o.d[gp] = (double)d;
        o.vhat[gp] = vh;
        o.accel[gp] = ac;
        o.dwell_pt[gp] = dw;
        o.key[gp] = key;
        o.flags[gp] = fl;
      }
      if (k == 0) {
        o.start_ts[j] = ts;
        o.slat[j] = lat;
        o.slon[j] = lon;
      }
      if (k == n - 1) {
        o.end_ts[j] = ts;
        o.duration[j] = (int64_t)((unsigned long long)ts - (unsigned long long)first_ts);
        o.elat[j] = lat;
        o.elon[j] = lon;
      }
    }
    // runs of equal keys: heads where the key changes (or the journey starts)
    const bool head = valid && (k == 0 || key != p_key);
    uint32_t hmask = __ballot_sync(0xffffffffu, head);
    if (hmask == 0) {
      if (valid) agg_add(la, spd);  // the open run goes on through the whole iteration
    } else {
      // lanes before the first head close the open run
      int h = __ffs(hmask) - 1;
      if (valid && lane < h) agg_add(la, spd);
      const RunAgg r = warp_agg(la);
      const uint32_t r_cnt = off + (uint32_t)(base + h) - o_start;
      if (o_key != kKeyInvalid && r_cnt > 0) walk_put(rbuf, nbuf, o, st, o_key, o_start, r_cnt, r);
      // runs that start and end inside this iteration, one warp reduction each
      hmask &= hmask - 1;
      while (hmask) {
        const int h2 = __ffs(hmask) - 1;
        const uint32_t kh = __shfl_sync(0xffffffffu, key, h);
        RunAgg a = agg_empty();
        if (lane >= h && lane < h2) agg_add(a, spd);
        const RunAgg r2 = warp_agg(a);
        if (kh != kKeyInvalid) walk_put(rbuf, nbuf, o, st, kh, off + (uint32_t)(base + h), (uint32_t)(h2 - h), r2);
        h = h2;
        hmask &= hmask - 1;
      }
      // the last run of the iteration stays open: its lanes start their shares
      la = agg_empty();
      if (valid && lane >= h) agg_add(la, spd);
      o_key = __shfl_sync(0xffffffffu, key, h);
      o_start = off + (uint32_t)(base + h);
    }
    // carry the last point to the next iteration
    c_ts = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)ts, 31);
    c_lat = __shfl_sync(0xffffffffu, lat, 31);
    c_lon = __shfl_sync(0xffffffffu, lon, 31);
    c_spd = __shfl_sync(0xffffffffu, spd, 31);
    c_cos = shfl_cos(ccur, 31);
    c_key = __shfl_sync(0xffffffffu, key, 31);
  }
  // the run open at the journey's end
  {
    const RunAgg r = warp_agg(la);
    const uint32_t r_cnt = off + (uint32_t)n - o_start;
    if (o_key != kKeyInvalid && r_cnt > 0) walk_put(rbuf, nbuf, o, st, o_key, o_start, r_cnt, r);
  }
  // journey sums: each lane's own sum, then a fixed shuffle tree
  const double sd = dist.warp_total();
  const long long sw = warp_sum(dwell);
  const uint32_t sdup = warp_sum(dup), soff = warp_sum(offg);
  if (lane == 0) {
    o.n[j] = n;
    o.off[j] = off;
    o.dist[j] = sd;
    o.dwell[j] = sw;
    n_dup += sdup;
    n_off += soff;
  }
}

// Grid threshold tables of up to this many entries (both axes) are copied into the walk's
// shared memory (16 KB), single-instance runs only.
constexpr int kWalkThrMax = 2048;
// resident walk blocks per SM (the register budget per thread follows)
template <class Form> struct WalkMinBlocks { static constexpr int value = 8; };
template <> struct WalkMinBlocks<Fp64Form> { static constexpr int value = 7; };
__host__ __device__ constexpr bool walk_thr_shared(int n_rows, int n_cols, int n_inst) {
  return n_inst == 0 && n_rows + n_cols + 2 <= kWalkThrMax;
}

// One warp per journey, journeys taken longest first from the work list (from position *wbeg
// on, or all of it) through the work counter; a persistent grid. The dynamic shared memory
// holds the grid's threshold tables when walk_thr_shared (8 bytes per entry), else nothing.
template <class Form>
__global__ void __launch_bounds__(kWalkBlock, WalkMinBlocks<Form>::value) k_journey_walk(const Rec* __restrict__ rec,
                                                            const uint16_t* __restrict__ spos,
                                                            const uint32_t* __restrict__ jn,
                                                            const uint32_t* __restrict__ joff, uint32_t J,
                                                            GridParams g, Batch bt, JourneyOut o, DevState* st,
                                                            const uint32_t* __restrict__ order, uint32_t* work,
                                                            const uint32_t* __restrict__ wbeg) {
  __shared__ RunSlot s_runs[kWalkBlock / 32][kWalkRunCap];
  extern __shared__ unsigned long long s_thr[];
  const unsigned long long* sthr = nullptr;
  if (walk_thr_shared(g.n_rows, g.n_cols, bt.n_inst)) {
    for (int i = threadIdx.x; i <= g.n_rows; i += kWalkBlock) s_thr[i] = g.row_thr[i];
    for (int i = threadIdx.x; i <= g.n_cols; i += kWalkBlock) s_thr[g.n_rows + 1 + i] = g.col_thr[i];
    __syncthreads();
    sthr = s_thr;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RunSlot* rbuf = s_runs[warp];
  uint32_t nbuf = 0;
  unsigned long long n_dup = 0, n_off = 0;
  const uint32_t w0 = wbeg ? *wbeg : 0u;  // the list from position *wbeg on (all without wbeg)
  for (;;) {
    uint32_t w = 0;
    if (lane == 0) w = w0 + atomicAdd(work, 1u);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= J) break;
    const uint32_t j = order ? order[w] : w;
    const uint32_t off = joff[j];
    walk_journey<Form>(j, rec + off, spos + off, (int)jn[j], off, g, bt, o, st, rbuf, nbuf, n_dup, n_off, sthr);
  }
  walk_flush(rbuf, nbuf, o, st);
  if (lane == 0) {
    if (n_dup) atomicAdd(&st->n_dup, n_dup);
    if (n_off) atomicAdd(&st->n_offgrid, n_off);
  }
}

// Work list keys: the journeys by size, longest first (ties by rank).
__global__ void k_size_keys(const uint32_t* __restrict__ jn, uint32_t J, unsigned long long* __restrict__ keys) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < J) keys[r] = 0xFFFFFFFFull - jn[r];
}

// Per-point features that need a journey's earlier points (materialised points only): the time
// since the current stop began (dwell summed over consecutive stop steps: a segmented scan,
// reset at every step that is not a stop, which includes the journey's first point) and the
// acceleration from the implied speeds of this and the previous step (both with dt > 0),
// evaluated in binary64 from the step distances and stored as float32. One warp per journey,
// 32 points at a time, the scan carried from chunk to chunk.
__global__ void __launch_bounds__(256) k_point_extras(const uint32_t* __restrict__ jn,
                                                      const uint32_t* __restrict__ joff, uint32_t J,
                                                      const int64_t* __restrict__ ts, Batch bt,
                                                      const uint32_t* __restrict__ perm,
                                                      const double* __restrict__ d,
                                                      const int64_t* __restrict__ dwell,
                                                      const uint8_t* __restrict__ flags,
                                                      int64_t* __restrict__ stop_ms,
                                                      float* __restrict__ accel_v) {
  const int lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < J; j += nwarps) {
    const uint32_t off = joff[j], n = jn[j];
    long long carry = 0;
    for (uint32_t b = 0; b < n; b += 32) {
      const uint32_t k = b + lane, g = off + k;
      long long v = 0;
      uint32_t reset = 1;
      float av = 0.0f;
      if (k < n) {
        if (flags[g] & kFStop) {
          v = dwell[g];
          reset = 0;
        }
        if (k >= 2) {
          const int64_t t0 = row_ts(ts, bt, perm[g - 2]), t1 = row_ts(ts, bt, perm[g - 1]), t2 = row_ts(ts, bt, perm[g]);
          const int64_t dt1 = (int64_t)((unsigned long long)t1 - (unsigned long long)t0);
          const int64_t dt2 = (int64_t)((unsigned long long)t2 - (unsigned long long)t1);
          if (dt1 > 0 && dt2 > 0) {
            const double s1 = (double)dt1 / 1000.0, s2 = (double)dt2 / 1000.0;
            av = (float)((d[g] / s2 - d[g - 1] / s1) / s2);
          }
        }
      }
      // inclusive segmented scan: the sum since the last reset at or before this lane
#pragma unroll
      for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const long long pv = __shfl_up_sync(0xffffffffu, v, o2);
        const uint32_t pr = __shfl_up_sync(0xffffffffu, reset, o2);
        if (lane >= o2 && !reset) {
          v += pv;
          reset = pr;
        }
      }
      const long long out = reset ? v : v + carry;  // no reset in this chunk up to here: continue the run
      if (k < n) {
        stop_ms[g] = out;
        accel_v[g] = av;
      }
      carry = __shfl_sync(0xffffffffu, out, 31);
    }
  }
}

}  // namespace cvetl
