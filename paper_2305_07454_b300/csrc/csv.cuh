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
// Decimal conversion uses no floating-point division and no binary64 arithmetic:
// M / 10^k = (M / 5^k) * 2^-k, and q = floor(M * 2^t / 5^k) (55-57 bits) comes from one 64 x 64
// multiply-high of the left-justified M by a 64-bit reciprocal of 5^k, corrected once with the
// exact remainder; q and the remainder then give the round-to-nearest-even binary64 result.
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
// bit length of 5^k
__constant__ int kLen5[16] = {1, 3, 5, 7, 10, 12, 14, 17, 19, 21, 24, 26, 28, 31, 33, 35};
// floor(2^(63 + Ld) / 5^k), Ld the bit length of 5^k: a reciprocal in [2^63, 2^64)
__constant__ unsigned long long kRecip5[16] = {
    0ull,  // k = 0: no division
    0xccccccccccccccccull, 0xa3d70a3d70a3d70aull, 0x83126e978d4fdf3bull, 0xd1b71758e219652bull,
    0xa7c5ac471b478423ull, 0x8637bd05af6c69b5ull, 0xd6bf94d5e57a42bcull, 0xabcc77118461cefcull,
    0x89705f4136b4a597ull, 0xdbe6fecebdedd5beull, 0xafebff0bcb24aafeull, 0x8cbccc096f5088cbull,
    0xe12e13424bb40e13ull, 0xb424dc35095cd80full, 0x901d7cf73ab0acd9ull,
};

// The binary64 value of an integer M < 2^53 (exact), by its bit layout.
__device__ __forceinline__ double u53_to_f64(unsigned long long M) {
  if (M == 0) return 0.0;
  const int L = 64 - __clzll((long long)M);
  const unsigned long long mant = M << (53 - L);  // leading bit at position 52
  return __longlong_as_double((long long)(((unsigned long long)(1022 + L) << 52) | (mant & ((1ull << 52) - 1))));
}

// The binary64 value nearest to M / 10^k (ties to even), M < 10^15, 0 <= k <= 15.
// With L, Ld the bit lengths of M and d = 5^k and t = 56 + Ld - L, q = floor(M 2^t / d) lies in
// [2^55, 2^57). Mn = M 2^(64 - L) and R = floor(2^(63 + Ld) / d) give hi = floor(Mn R / 2^64) in
// (M 2^(t+7) / d - 2, M 2^(t+7) / d], so hi >> 7 is q or q - 1; the remainder
// M 2^t - q d lies in [0, 2d) (below 2^36), so 64-bit wrapping arithmetic computes it exactly.
__device__ __forceinline__ double dec_to_f64(unsigned long long M, int k) {
  if (M == 0) return 0.0;
  if (k == 0) return u53_to_f64(M);
  const unsigned long long d = kPow5[k];
  const int L = 64 - __clzll((long long)M), Ld = kLen5[k];
  const int t = 56 + Ld - L;
  unsigned long long q = __umul64hi(M << (64 - L), kRecip5[k]) >> 7;
  unsigned long long r = (t >= 64 ? 0ull : (M << t)) - q * d;
  if (r >= d) {
    q += 1;
    r -= d;
  }
  int s = 3 + (int)(q >> 56);  // q has 56 or 57 bits: 3 or 4 below the binary64 significand
  unsigned long long mant = q >> s;
  const uint32_t low = (uint32_t)q & ((1u << s) - 1u), half = 1u << (s - 1);
  if (low > half || (low == half && (r != 0 || (mant & 1)))) mant += 1;
  if (mant >> 53) {
    mant >>= 1;
    s += 1;
  }
  const int e = 52 + s - t - k;
  return __longlong_as_double((long long)(((unsigned long long)(e + 1023) << 52) | (mant & ((1ull << 52) - 1))));
}

__device__ __forceinline__ double negate_if(double v, bool neg) {
  return neg ? dfrom(dbits(v) ^ 0x8000000000000000ull) : v;
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
    dv[f] = negate_if(dec_to_f64(M, nf), neg);
  }
  // |lat| <= 90, |lon| <= 180 (on the bit patterns)
  const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
  if ((dbits(dv[0]) & kAbs) > 0x4056800000000000ull) return false;
  if ((dbits(dv[1]) & kAbs) > 0x4066800000000000ull) return false;
  jid = iv[0];
  ts = iv[1];
  lat = dv[0];
  lon = dv[1];
  spd = f64_to_f32_rn_z(dv[2]);
  hd = f64_to_f32_rn_z(dv[3]);
  return true;
}

// ---- byte-parallel helpers (SWAR: several bytes per 32- or 64-bit word)
// Bit j (0..3) set when byte j of w equals the byte repeated in c4. The zero-byte test leaves
// bit 7 of each matching byte, and one multiply by 1 + 2^7 + 2^14 + 2^21 moves bits 7, 15, 23
// and 31 to bits 28..31 (the partial products land on distinct bits, so nothing carries).
__device__ __forceinline__ uint32_t byte_eq_nibble(uint32_t w, uint32_t c4) {
  const uint32_t x = w ^ c4;
  const uint32_t z = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
  return (z * 0x00204081u) >> 28;
}

// 8 bytes at byte offset pos of a 16-byte aligned shared buffer: three aligned 32-bit words and
// two byte permutes (no shift of a 64-bit value, no branch on the offset).
__device__ __forceinline__ unsigned long long load8(const unsigned char* s, int pos) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(s + (pos & ~3));
  const uint32_t sel = 0x3210u + 0x1111u * (uint32_t)(pos & 3);  // bytes off .. off + 3 of the pair
  const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
  return (unsigned long long)__byte_perm(w0, w1, sel) | ((unsigned long long)__byte_perm(w1, w2, sel) << 32);
}

// The value of n (1..8) ASCII decimal digits held in the low n bytes of x (first digit in the
// lowest byte), or false if one of them is not a digit. The digits are moved to the top bytes
// and the bottom bytes filled with '0'; each 32-bit half (four digits) is then combined by
// multiply-and-shift inside the word (pairs, then the quad), and the halves by one multiply-add.
// 32-bit words keep every step a single integer instruction.
__device__ __forceinline__ bool digits8(unsigned long long x, int n, unsigned long long& v) {
  const int sh = 8 * (8 - n);
  x = sh ? ((x << sh) | (0x3030303030303030ull >> (64 - sh))) : x;
  const uint32_t a = (uint32_t)x, b = (uint32_t)(x >> 32);  // digits 1-4, digits 5-8
  uint32_t ta = a - 0x30303030u, tb = b - 0x30303030u;     // a byte below '0' sets its top bit
  if (((a + 0x46464646u) | ta | (b + 0x46464646u) | tb) & 0x80808080u) return false;  // outside '0'..'9'
  ta = (ta * 10u + (ta >> 8)) & 0x00FF00FFu;  // 2-digit lanes
  tb = (tb * 10u + (tb >> 8)) & 0x00FF00FFu;
  ta = (ta * 100u + (ta >> 16)) & 0xFFFFu;    // 4 digits
  tb = (tb * 100u + (tb >> 16)) & 0xFFFFu;
  v = (unsigned long long)(ta * 10000u + tb);
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

// The value of the n (1..16) digits at s[pos, pos + n) as two groups, the last min(n, 8)
// digits and the k = n - 8 before them (none when n <= 8, read as one '0'): the same work for
// every length, so the lanes of a warp whose fields differ in length do not diverge.
__device__ __forceinline__ bool digits16_at(const unsigned char* s, int pos, int n, unsigned long long& v) {
  const int k = n > 8 ? n - 8 : 0;
  const unsigned long long lead = load8(s, pos), last = load8(s, pos + k);
  unsigned long long hv, lv;
  bool ok = digits8(last, n - k, lv);
  ok &= digits8(k ? lead : 0x30ull, k ? k : 1, hv);
  v = hv * 100000000ull + lv;
  return ok;
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
  if (!(n <= 16 ? digits16_at(s, a, n, v) : digits_at(s, a, n, v))) return false;
  out = neg ? -(long long)v : (long long)v;
  return true;
}

// A decimal field -?[0-9]+(\.[0-9]+)? with at most 15 digits. Its (at most 16) bytes are
// loaded as two words once: the '.' is found by a byte compare, removed by shifting the bytes
// above it down, and the remaining digit string is converted eight digits at a time.
__device__ __forceinline__ bool dec_field(const unsigned char* s, int a, int b, double& out) {
  const bool neg = a < b && s[a] == '-';
  if (neg) ++a;
  const int len = b - a;
  if (len < 1 || len > 16) return false;  // 15 digits and one '.'
  unsigned long long lo = load8(s, a), hi = load8(s, a + 8);  // bytes [a, a + 16)
  const uint32_t dm = (byte_eq_nibble((uint32_t)lo, 0x2E2E2E2Eu) | (byte_eq_nibble((uint32_t)(lo >> 32), 0x2E2E2E2Eu) << 4) |
                       (byte_eq_nibble((uint32_t)hi, 0x2E2E2E2Eu) << 8) |
                       (byte_eq_nibble((uint32_t)(hi >> 32), 0x2E2E2E2Eu) << 12)) &
                      ((1u << len) - 1u);
  int n = len, nf = 0;
  if (dm) {
    const int dot = __ffs(dm) - 1;
    nf = len - dot - 1;
    if (dot == 0 || nf == 0) return false;  // digits on both sides of the '.'
    n = len - 1;
    const unsigned long long slo = (lo >> 8) | (hi << 56), shi = hi >> 8;  // all bytes one down
    if (dot < 8) {
      const unsigned long long keep = (1ull << (8 * dot)) - 1;
      lo = (lo & keep) | (slo & ~keep);
      hi = shi;
    } else {
      const unsigned long long keep = (1ull << (8 * (dot - 8))) - 1;
      hi = (hi & keep) | (shi & ~keep);
    }
  }
  if (n > 15) return false;
  // the n digits, bytes [0, n) of (lo, hi) (a second '.' is not a digit), as two groups: the
  // last min(n, 8) and the k = n - 8 before them (none when n <= 8, read as one '0'), the same
  // work for every length
  const int k = n > 8 ? n - 8 : 0;
  const unsigned long long last = k ? ((lo >> (8 * k)) | (hi << ((64 - 8 * k) & 63))) : lo;
  unsigned long long M, hv;
  bool ok = digits8(last, n - k, M);
  ok &= digits8(k ? lo : 0x30ull, k ? k : 1, hv);
  if (!ok) return false;
  M += hv * 100000000ull;
  out = negate_if(dec_to_f64(M, nf), neg);
  return true;
}

// The five ',' of a line longer than 64 bytes, from the comma mask (a rare path: kept out of
// line so that the common path below holds its positions in registers).
__device__ __noinline__ bool long_line_seps(const uint32_t* cm, int a, int e, int* sep) {
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
  return nsep == 5;
}

// One line [a, e) of the staged window, fields located with the comma mask.
__device__ __forceinline__ bool parse_line_masked(const unsigned char* s, const uint32_t* cm, int a, int e,
                                                  int64_t& jid, int64_t& ts, double& lat, double& lon,
                                                  float& spd, float& hd) {
  if (e > a && s[e - 1] == '\r') --e;
  if (e == a) return false;
  int sep[5];
  if (e - a <= 64) {  // the comma bits of bytes [a, a + 64) from three mask words
    const int w = a >> 5, sh = a & 31;
    unsigned long long m = (((unsigned long long)cm[w + 1] << 32) | cm[w]) >> sh;
    if (sh) m |= (unsigned long long)cm[w + 2] << (64 - sh);
    if (e - a < 64) m &= (1ull << (e - a)) - 1;
    if (__popcll(m) != 5) return false;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      sep[k] = a + __ffsll((long long)m) - 1;
      m &= m - 1;
    }
  } else {
    int s6[6];
    if (!long_line_seps(cm, a, e, s6)) return false;
#pragma unroll
    for (int k = 0; k < 5; ++k) sep[k] = s6[k];
  }
  long long iv0, iv1;
  double d0, d1, d2, d3;
  if (!int_field(s, a, sep[0], iv0) || !int_field(s, sep[0] + 1, sep[1], iv1)) return false;
  if (!dec_field(s, sep[1] + 1, sep[2], d0) || !dec_field(s, sep[2] + 1, sep[3], d1) ||
      !dec_field(s, sep[3] + 1, sep[4], d2) || !dec_field(s, sep[4] + 1, e, d3))
    return false;
  const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
  if ((dbits(d0) & kAbs) > 0x4056800000000000ull) return false;
  if ((dbits(d1) & kAbs) > 0x4066800000000000ull) return false;
  jid = iv0;
  ts = iv1;
  lat = d0;
  lon = d1;
  spd = f64_to_f32_rn_z(d2);
  hd = f64_to_f32_rn_z(d3);
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
  unsigned long long block_lines = 0;  // (thread 0) added to *total once
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
      block_lines += l;
    }
  }
  if (threadIdx.x == 0 && block_lines) atomicAdd(total, block_lines);  // 64-bit: the caller checks the 32-bit prefix sums
}

// Pass 2: parse tile blockIdx.x, whose first row is tile_row[blockIdx.x]. One pass turns the
// staged bytes into newline and comma bit masks; line starts, line ends and field separators
// then come from the masks, and the digits are read eight at a time. Line i of the tile is row
// tile_row + i: consecutive threads write consecutive rows.
// 5 CTAs per SM (48 registers a thread): measured faster than 3 without the cap (78 registers)
// although the cap spills a few values
__global__ void __launch_bounds__(kCsvBlock, 5) k_csv_parse(const unsigned char* __restrict__ buf,
                                                         unsigned long long len,
                                                         const uint32_t* __restrict__ tile_row, CsvOut out,
                                                         uint32_t cap, DevState* st) {
  __shared__ __align__(16) unsigned char s_buf[kCsvTile + kCsvHalo + 32];
  __shared__ uint32_t s_nl[(kCsvTile + kCsvHalo) / 32 + 2], s_cm[(kCsvTile + kCsvHalo) / 32 + 2];
  __shared__ uint16_t s_start[kCsvTile];
  __shared__ uint32_t s_scan[kCsvBlock / 32 + 1];
  __shared__ unsigned char s_prev;
  const int tid = threadIdx.x;
  const uint32_t tile = blockIdx.x;
  const unsigned long long base = (unsigned long long)tile * kCsvTile;
  const int tlen = (int)min((unsigned long long)kCsvTile, len - base);
  const int wlen = (int)min((unsigned long long)(kCsvTile + kCsvHalo), len - base);
  // stage the window (tile + halo) and build its newline and comma masks, one bit per byte:
  // thread t takes the 32-byte chunks t, t + kCsvBlock, ... (16-byte loads: base is 16-byte
  // aligned), stores the bytes to shared memory and derives the two mask words from its
  // registers. The bytes after the window are zero (the word loads of the parser may read 32
  // bytes past a field), and so are the two mask words after the last.
  const int nmask = (wlen + 31) / 32;
  for (int ch = tid; ch < nmask; ch += kCsvBlock) {
    const int o = ch * 32;
    uint32_t w[8];
    if (o + 32 <= wlen) {
      const uint4 v0 = *reinterpret_cast<const uint4*>(buf + base + o);
      const uint4 v1 = *reinterpret_cast<const uint4*>(buf + base + o + 16);
      w[0] = v0.x; w[1] = v0.y; w[2] = v0.z; w[3] = v0.w;
      w[4] = v1.x; w[5] = v1.y; w[6] = v1.z; w[7] = v1.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint32_t x = 0;
        for (int bb = 0; bb < 4; ++bb) {
          const int p = o + 4 * q + bb;
          if (p < wlen) x |= (uint32_t)buf[base + p] << (8 * bb);
        }
        w[q] = x;
      }
    }
    *reinterpret_cast<uint4*>(s_buf + o) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(s_buf + o + 16) = make_uint4(w[4], w[5], w[6], w[7]);
    uint32_t nl = 0, cm = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      nl |= byte_eq_nibble(w[q], 0x0A0A0A0Au) << (4 * q);
      cm |= byte_eq_nibble(w[q], 0x2C2C2C2Cu) << (4 * q);
    }
    s_nl[ch] = nl;
    s_cm[ch] = cm;
  }
  if (tid < 32) s_buf[nmask * 32 + tid] = 0;
  if (tid < 2) {
    s_nl[nmask + tid] = 0;
    s_cm[nmask + tid] = 0;
  }
  if (tid == 0) s_prev = (base == 0) ? (unsigned char)'\n' : buf[base - 1];
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
    // the line's end: the newline before the next line's start, or for the tile's last line
    // the next newline bit at or after its start
    int w = sl >> 5;
    uint32_t m;
    if (i + 1 < nstart) {
      const int e = s_start[i + 1] - 1;
      w = e >> 5;
      m = 1u << (e & 31);
    } else {
      m = s_nl[w] & (~0u << (sl & 31));
      while (!m && ++w < nmask) m = s_nl[w];
    }
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
