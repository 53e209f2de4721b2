// csv.cuh — extract from CSV text: split lines, parse and validate each row, and write the
// kept rows to columns in file order (Methods, "Connected Vehicle Dataset": per-vehicle CSV
// text; Table 1 shows the columns). The paper gives no grammar; the one used here:
//   row      = 6 fields separated by ','; one trailing '\r' is stripped; empty lines are rows
//   integer  = -?[0-9]{1,18}                (journey id, timestamp in ms)
//   decimal  = -?[0-9]+(\.[0-9]+)?  with at most 15 digits in total
//   value    = the binary64 value nearest to M / 10^k (M the digits as an integer, k the number
//              of fraction digits), i.e. one round-to-nearest division of two exact binary64s
//   range    = |lat| <= 90 and |lon| <= 180; speed and heading are rounded to float32
// Every line is a row, in file order, and its extracted-row index is its line number; a line
// breaking any rule becomes the row (0, 0, NaN, NaN, NaN, NaN), which the extract drops and
// counts as malformed. Row i's place in the columns is then known from the line starts alone:
// tile t's first row is the number of line starts before it (a prefix sum of per-tile counts),
// so tiles are parsed independently, with no ordering between them.
//
// Decimal conversion uses no floating-point division: M / 10^k = (M / 5^k) * 2^-k, and
// M / 5^k is computed exactly as an integer quotient of M * 2^t (128-bit) by 5^k through a
// 128-bit reciprocal ceil(2^128 / 5^k) with one correction step; the 55-57-bit quotient and its
// remainder then give the round-to-nearest-even binary64 result directly.
#pragma once
#include "common.cuh"

namespace cvetl {

constexpr int kCsvTile = 12288;  // bytes per tile (multiple of 16)
constexpr int kCsvHalo = 1024;   // bytes past the tile kept in shared memory (lines crossing its end)
constexpr int kCsvBlock = 256;

__constant__ unsigned long long kPow5[16] = {1ull, 5ull, 25ull, 125ull, 625ull, 3125ull, 15625ull,
                                             78125ull, 390625ull, 1953125ull, 9765625ull,
                                             48828125ull, 244140625ull, 1220703125ull,
                                             6103515625ull, 30517578125ull};
// ceil(2^128 / 5^k) as {high 64 bits, low 64 bits}
__constant__ unsigned long long kRecip5[16][2] = {
    {0ull, 0ull},  // k = 0: no division
    {0x3333333333333333ull, 0x3333333333333334ull},
    {0x0a3d70a3d70a3d70ull, 0xa3d70a3d70a3d70bull},
    {0x020c49ba5e353f7cull, 0xed916872b020c49cull},
    {0x0068db8bac710cb2ull, 0x95e9e1b089a02753ull},
    {0x0014f8b588e368f0ull, 0x8461f9f01b866e44ull},
    {0x000431bde82d7b63ull, 0x4dad31fcd24e160eull},
    {0x0000d6bf94d5e57aull, 0x42bc3d329076046aull},
    {0x00002af31dc46118ull, 0x73bf3f70834acdafull},
    {0x0000089705f4136bull, 0x4a59731680a88f8aull},
    {0x000001b7cdfd9d7bull, 0xdbab7d6ae6881cb6ull},
    {0x00000057f5ff85e5ull, 0x92557f7bc7b4d28bull},
    {0x000000119799812dull, 0xea11197f27f0f6e9ull},
    {0x0000000384b84d09ull, 0x2ed0384ca19697c9ull},
    {0x00000000b424dc35ull, 0x095cd80f538484c2ull},
    {0x0000000024075f3dull, 0xceac2b3643e74dc1ull},
};

typedef unsigned __int128 u128;

// floor(a * b / 2^128) from 64-bit limbs
__device__ __forceinline__ u128 mulhi128(u128 a, u128 b) {
  const unsigned long long a0 = (unsigned long long)a, a1 = (unsigned long long)(a >> 64);
  const unsigned long long b0 = (unsigned long long)b, b1 = (unsigned long long)(b >> 64);
  const u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
  const u128 mid = (p00 >> 64) + (unsigned long long)p01 + (unsigned long long)p10;
  return p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
}

// The binary64 value nearest to M / 10^k (ties to even), M < 10^15, 0 <= k <= 15.
__device__ __forceinline__ double dec_to_f64(unsigned long long M, int k) {
  if (M == 0) return 0.0;
  if (k == 0) return __ull2double_rn(M);  // exact: M < 2^53
  const unsigned long long d = kPow5[k];
  const int L = 64 - __clzll((long long)M), Ld = 64 - __clzll((long long)d);
  const int t = 56 + Ld - L;  // x / d lies in [2^55, 2^57)
  const u128 x = (u128)M << t;
  const u128 R = ((u128)kRecip5[k][0] << 64) | kRecip5[k][1];
  unsigned long long q = (unsigned long long)mulhi128(x, R);  // q or q + 1
  __int128 r = (__int128)x - (__int128)((u128)q * d);
  if (r < 0) {
    q -= 1;
    r += d;
  }
  const int b = 64 - __clzll((long long)q);
  int s = b - 53;  // 3 or 4 bits below the binary64 significand
  unsigned long long mant = q >> s;
  const unsigned long long low = q & ((1ull << s) - 1), half = 1ull << (s - 1);
  if (low > half || (low == half && (r != 0 || (mant & 1)))) mant += 1;
  if (mant >> 53) {
    mant >>= 1;
    s += 1;
  }
  const int e = 52 + s - t - k;
  return __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) | (mant & ((1ull << 52) - 1))));
}

__device__ __forceinline__ bool is_digit(unsigned c) { return c - '0' <= 9u; }

// Parses one line (without its '\n'); p may point to shared or global memory.
__device__ bool parse_row(const unsigned char* p, int len, int64_t& jid, int64_t& ts, double& lat,
                          double& lon, float& spd, float& hd) {
  if (len > 0 && p[len - 1] == '\r') --len;
  if (len == 0) return false;
  int i = 0;
  long long iv[2];
  for (int f = 0; f < 2; ++f) {
    bool neg = false;
    if (i < len && p[i] == '-') {
      neg = true;
      ++i;
    }
    int nd = 0;
    unsigned long long v = 0;
    while (i < len && p[i] != ',') {
      const unsigned c = p[i];
      if (!is_digit(c) || ++nd > 18) return false;
      v = v * 10 + (c - '0');
      ++i;
    }
    if (nd == 0 || i >= len) return false;
    ++i;  // ','
    iv[f] = neg ? -(long long)v : (long long)v;
  }
  double dv[4];
  for (int f = 0; f < 4; ++f) {
    bool neg = false;
    if (i < len && p[i] == '-') {
      neg = true;
      ++i;
    }
    int ni = 0, nf = 0;
    unsigned long long M = 0;
    while (i < len && is_digit(p[i])) {
      if (++ni > 15) return false;
      M = M * 10 + (p[i] - '0');
      ++i;
    }
    if (ni == 0) return false;
    if (i < len && p[i] == '.') {
      ++i;
      while (i < len && is_digit(p[i])) {
        if (ni + ++nf > 15) return false;
        M = M * 10 + (p[i] - '0');
        ++i;
      }
      if (nf == 0) return false;
    }
    if (f < 3) {
      if (i >= len || p[i] != ',') return false;
      ++i;
    } else if (i != len) {
      return false;
    }
    const double v = dec_to_f64(M, nf);
    dv[f] = neg ? -v : v;
  }
  // |lat| <= 90, |lon| <= 180 (on the bit patterns)
  const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
  if (((unsigned long long)__double_as_longlong(dv[0]) & kAbs) > 0x4056800000000000ull) return false;
  if (((unsigned long long)__double_as_longlong(dv[1]) & kAbs) > 0x4066800000000000ull) return false;
  jid = iv[0];
  ts = iv[1];
  lat = dv[0];
  lon = dv[1];
  spd = __double2float_rn(dv[2]);
  hd = __double2float_rn(dv[3]);
  return true;
}

// ---- byte-parallel helpers (SWAR: several bytes per 32- or 64-bit word)
// Bit i of the result is set when byte i of w equals c (exact per byte: no borrow between bytes).
__device__ __forceinline__ uint32_t byte_eq_mask4(uint32_t w, uint32_t c4) {
  const uint32_t x = w ^ c4;
  const uint32_t z = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;  // 0x80 where x's byte is 0
  return ((z >> 7) & 1u) | ((z >> 14) & 2u) | ((z >> 21) & 4u) | ((z >> 28) & 8u);
}

// 8 bytes at byte offset pos of a 16-byte aligned shared buffer (two aligned loads + shift).
__device__ __forceinline__ unsigned long long load8(const unsigned char* s, int pos) {
  const unsigned long long* w = reinterpret_cast<const unsigned long long*>(s + (pos & ~7));
  const int sh = (pos & 7) * 8;
  const unsigned long long lo = w[0];
  if (sh == 0) return lo;
  return (lo >> sh) | (w[1] << (64 - sh));
}

// The value of n (1..8) ASCII decimal digits held in the low n bytes of x (first digit in the
// lowest byte), or false if one of them is not a digit. The digits are moved to the top bytes
// and the bottom bytes filled with '0', then pairs, quads and the octet are combined by
// multiply-and-shift inside the word.
__device__ __forceinline__ bool digits8(unsigned long long x, int n, unsigned long long& v) {
  const int sh = 8 * (8 - n);
  x = sh ? ((x << sh) | (0x3030303030303030ull >> (64 - sh))) : x;
  const unsigned long long t = x - 0x3030303030303030ull;  // digit values (a byte below '0' sets its top bit)
  if (((x + 0x4646464646464646ull) | t) & 0x8080808080808080ull) return false;  // some byte outside '0'..'9'
  unsigned long long y = (t * 10 + (t >> 8)) & 0x00FF00FF00FF00FFull;      // 2-digit lanes
  y = (y * 100 + (y >> 16)) & 0x0000FFFF0000FFFFull;                      // 4-digit lanes
  v = (y * 10000 + (y >> 32)) & 0xFFFFFFFFull;                            // 8 digits
  return true;
}

// The value of the n (1..18) digits at s[pos, pos + n): a leading chunk of 1..8 digits, then
// chunks of 8.
__device__ __forceinline__ bool digits_at(const unsigned char* s, int pos, int n, unsigned long long& v) {
  const int m = n - ((n - 1) >> 3) * 8;
  unsigned long long acc, d;
  if (!digits8(load8(s, pos), m, acc)) return false;
  for (pos += m, n -= m; n > 0; pos += 8, n -= 8) {
    if (!digits8(load8(s, pos), 8, d)) return false;
    acc = acc * 100000000ull + d;
  }
  v = acc;
  return true;
}

// Fields of one line of the staged window by the separator masks: an integer field.
__device__ __forceinline__ bool int_field(const unsigned char* s, int a, int b, long long& out) {
  bool neg = false;
  if (a < b && s[a] == '-') {
    neg = true;
    ++a;
  }
  const int n = b - a;
  if (n < 1 || n > 18) return false;
  unsigned long long v;
  if (!digits_at(s, a, n, v)) return false;
  out = neg ? -(long long)v : (long long)v;
  return true;
}

// A decimal field -?[0-9]+(\.[0-9]+)? with at most 15 digits.
__device__ __forceinline__ bool dec_field(const unsigned char* s, int a, int b, double& out) {
  bool neg = false;
  if (a < b && s[a] == '-') {
    neg = true;
    ++a;
  }
  const int len = b - a;
  if (len < 1 || len > 16) return false;  // 15 digits and one '.'
  // position of the first '.' (if any) in the field
  int dot = -1;
  {
    const unsigned long long w0 = load8(s, a), w1 = load8(s, a + 8);
    const uint32_t m = byte_eq_mask4((uint32_t)w0, 0x2E2E2E2Eu) | (byte_eq_mask4((uint32_t)(w0 >> 32), 0x2E2E2E2Eu) << 4) |
                       (byte_eq_mask4((uint32_t)w1, 0x2E2E2E2Eu) << 8) | (byte_eq_mask4((uint32_t)(w1 >> 32), 0x2E2E2E2Eu) << 12);
    const uint32_t in = m & ((1u << len) - 1u);
    if (in) dot = __ffs(in) - 1;
  }
  const int ni = dot < 0 ? len : dot, nf = dot < 0 ? 0 : len - dot - 1;
  if (ni < 1 || (dot >= 0 && nf < 1) || ni + nf > 15) return false;
  unsigned long long hi, lo = 0;
  if (!digits_at(s, a, ni, hi)) return false;
  if (nf && !digits_at(s, a + ni + 1, nf, lo)) return false;  // a second '.' is not a digit
  const unsigned long long M = hi * (kPow5[nf] << nf) + lo;  // hi * 10^nf + lo < 10^15
  const double v = dec_to_f64(M, nf);
  out = neg ? -v : v;
  return true;
}

// One line [a, e) of the staged window, fields located with the comma mask.
__device__ __forceinline__ bool parse_line_masked(const unsigned char* s, const uint32_t* cm, int a, int e,
                                                  int64_t& jid, int64_t& ts, double& lat, double& lon,
                                                  float& spd, float& hd) {
  if (e > a && s[e - 1] == '\r') --e;
  if (e == a) return false;
  int sep[6];
  int nsep = 0;
  for (int w = a >> 5; w <= ((e - 1) >> 5) && nsep < 6; ++w) {
    uint32_t m = cm[w];
    const int lo = w << 5;
    if (lo < a) m &= ~0u << (a - lo);
    if (lo + 32 > e) m &= (e - lo >= 32) ? ~0u : ((1u << (e - lo)) - 1u);
    while (m && nsep < 6) {
      sep[nsep++] = lo + __ffs(m) - 1;
      m &= m - 1;
    }
  }
  if (nsep != 5) return false;
  long long iv0, iv1;
  double d0, d1, d2, d3;
  if (!int_field(s, a, sep[0], iv0) || !int_field(s, sep[0] + 1, sep[1], iv1)) return false;
  if (!dec_field(s, sep[1] + 1, sep[2], d0) || !dec_field(s, sep[2] + 1, sep[3], d1) ||
      !dec_field(s, sep[3] + 1, sep[4], d2) || !dec_field(s, sep[4] + 1, e, d3))
    return false;
  const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
  if (((unsigned long long)__double_as_longlong(d0) & kAbs) > 0x4056800000000000ull) return false;
  if (((unsigned long long)__double_as_longlong(d1) & kAbs) > 0x4066800000000000ull) return false;
  jid = iv0;
  ts = iv1;
  lat = d0;
  lon = d1;
  spd = __double2float_rn(d2);
  hd = __double2float_rn(d3);
  return true;
}

struct CsvOut {
  int64_t *jid, *ts;
  double *lat, *lon;
  float *speed, *heading;
};

// Pass 1: line starts per tile. Byte b starts a line when b = 0 or byte b - 1 is '\n', so a
// tile's count is its newlines, less one for a newline in its last byte, plus one for a newline
// just before it (or for the first tile).
__global__ void __launch_bounds__(kCsvBlock) k_csv_tile_lines(const unsigned char* __restrict__ buf,
                                                              unsigned long long len, uint32_t n_tiles,
                                                              uint32_t* __restrict__ lines,
                                                              unsigned long long* __restrict__ total) {
  __shared__ uint32_t scratch[kCsvBlock / 32];
  for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const unsigned long long base = (unsigned long long)t * kCsvTile;
    const unsigned long long end = min(base + (unsigned long long)kCsvTile, len);
    uint32_t c = 0;
    for (unsigned long long b0 = base + threadIdx.x * 16ull; b0 < end; b0 += kCsvBlock * 16ull) {
      if (b0 + 16 <= end) {
        const uint4 v = *reinterpret_cast<const uint4*>(buf + b0);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t x = w[q] ^ 0x0A0A0A0Au;  // bytes equal to '\n' become 0
          c += __popc((x - 0x01010101u) & ~x & 0x80808080u);
        }
      } else {
        for (unsigned long long p = b0; p < end; ++p) c += buf[p] == '\n';
      }
    }
    c = block_sum<kCsvBlock, uint32_t>(c, scratch);  // ends with a barrier: scratch is free again
    if (threadIdx.x == 0) {
      const uint32_t before = (base == 0) ? 1u : (buf[base - 1] == '\n' ? 1u : 0u);
      const uint32_t l = c - (buf[end - 1] == '\n' ? 1u : 0u) + before;
      lines[t] = l;
      atomicAdd(total, (unsigned long long)l);  // 64-bit: the caller checks the 32-bit prefix sums
    }
  }
}

// Pass 2: parse tile blockIdx.x, whose first row is tile_row[blockIdx.x]. One pass turns the
// staged bytes into newline and comma bit masks; line starts, line ends and field separators
// then come from the masks, and the digits are read eight at a time. Line i of the tile is row
// tile_row + i: consecutive threads write consecutive rows.
__global__ void __launch_bounds__(kCsvBlock) k_csv_parse(const unsigned char* __restrict__ buf,
                                                         unsigned long long len,
                                                         const uint32_t* __restrict__ tile_row, CsvOut out,
                                                         uint32_t cap, DevState* st) {
  __shared__ __align__(16) unsigned char s_buf[kCsvTile + kCsvHalo + 32];
  __shared__ uint32_t s_nl[(kCsvTile + kCsvHalo) / 32 + 1], s_cm[(kCsvTile + kCsvHalo) / 32 + 1];
  __shared__ uint16_t s_start[kCsvTile];
  __shared__ uint32_t s_scan[kCsvBlock / 32 + 1];
  __shared__ unsigned char s_prev;
  const int tid = threadIdx.x;
  const uint32_t tile = blockIdx.x;
  const unsigned long long base = (unsigned long long)tile * kCsvTile;
  const int tlen = (int)min((unsigned long long)kCsvTile, len - base);
  const int wlen = (int)min((unsigned long long)(kCsvTile + kCsvHalo), len - base);
  // stage the tile (+ halo) in shared memory: 16-byte loads (base is 16-byte aligned); zero the
  // 32 bytes after the window (the word loads of the parser may read into them)
  for (int o = tid * 16; o < wlen; o += kCsvBlock * 16) {
    if (o + 16 <= wlen) *reinterpret_cast<uint4*>(s_buf + o) = *reinterpret_cast<const uint4*>(buf + base + o);
    else
      for (int q = o; q < wlen; ++q) s_buf[q] = buf[base + q];
  }
  if (tid < 32) s_buf[wlen + tid] = 0;
  if (tid == 0) s_prev = (base == 0) ? (unsigned char)'\n' : buf[base - 1];
  __syncthreads();
  // newline and comma bit masks of the window, one bit per byte: each thread classifies one
  // 4-byte word, eight lanes' nibbles combine into a 32-bit mask word
  const int nmask = (wlen + 31) / 32;
  for (int q0 = tid & ~31; q0 < nmask * 8; q0 += kCsvBlock) {  // warp-uniform trip count
    const int q = q0 + (tid & 31);
    const bool have = q < nmask * 8;  // groups of 8 lanes are all in or all out
    const uint32_t w = have ? reinterpret_cast<const uint32_t*>(s_buf)[q] : 0u;
    uint32_t nl = byte_eq_mask4(w, 0x0A0A0A0Au) << ((q & 7) * 4);
    uint32_t cm = byte_eq_mask4(w, 0x2C2C2C2Cu) << ((q & 7) * 4);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      nl |= __shfl_xor_sync(0xffffffffu, nl, o);
      cm |= __shfl_xor_sync(0xffffffffu, cm, o);
    }
    if (have && (q & 7) == 0) {
      s_nl[q >> 3] = nl;
      s_cm[q >> 3] = cm;
    }
  }
  __syncthreads();
  // line starts inside the tile (a byte after a newline): 2 mask words per thread
  const int tw = (tlen + 31) / 32;
  uint32_t smask[2];
  uint32_t cnt = 0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int w = tid * 2 + u;
    uint32_t m = 0;
    if (w < tw) {
      m = (s_nl[w] << 1) | (w ? (s_nl[w - 1] >> 31) : (s_prev == '\n' ? 1u : 0u));
      if ((w + 1) * 32 > tlen) m &= (tlen - w * 32 >= 32) ? ~0u : ((1u << (tlen - w * 32)) - 1u);
    }
    smask[u] = m;
    cnt += __popc(m);
  }
  uint32_t total;
  uint32_t r = block_excl_scan<kCsvBlock>(cnt, s_scan, &total);
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    uint32_t m = smask[u];
    while (m) {
      s_start[r++] = (uint16_t)((tid * 2 + u) * 32 + __ffs(m) - 1);
      m &= m - 1;
    }
  }
  __syncthreads();
  const int nstart = (int)total;
  const uint32_t row0 = tile_row[tile];
  for (int i = tid; i < nstart; i += kCsvBlock) {
    const int sl = s_start[i];
    // the line's end: the next newline bit at or after its start
    int w = sl >> 5;
    uint32_t m = s_nl[w] & (~0u << (sl & 31));
    while (!m && ++w < nmask) m = s_nl[w];
    int64_t a, b;
    double c, d;
    float e, f;
    bool ok;
    if (m) {
      ok = parse_line_masked(s_buf, s_cm, sl, w * 32 + __ffs(m) - 1, a, b, c, d, e, f);
    } else if (base + wlen == len) {
      ok = parse_line_masked(s_buf, s_cm, sl, wlen, a, b, c, d, e, f);
    } else {  // the line runs past the staged window: read it from global memory
      unsigned long long g = base + wlen;
      while (g < len && buf[g] != '\n') ++g;
      ok = parse_row(buf + base + sl, (int)(g - (base + sl)), a, b, c, d, e, f);
    }
    if (!ok) {  // a row without a position
      a = b = 0;
      c = d = __longlong_as_double(0x7FF8000000000000ll);
      e = f = __int_as_float(0x7FC00000);
    }
    const uint32_t o = row0 + (uint32_t)i;
    if (o < cap) {
      out.jid[o] = a;
      out.ts[o] = b;
      out.lat[o] = c;
      out.lon[o] = d;
      out.speed[o] = e;
      out.heading[o] = f;
    } else {
      atomicOr(&st->err, kErrCapacity);
    }
  }
}

}  // namespace cvetl
