// common.cuh — device utilities shared by the cvetl kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace cvetl {

constexpr uint32_t kKeyInvalid = 0xFFFFFFFFu;
constexpr uint64_t kSign64 = 0x8000000000000000ull;

// per-point flags (same values as CVETL_F_* in cvetl.h)
constexpr uint8_t kFStart = 0x01, kFDup = 0x02, kFOffgrid = 0x04, kFStop = 0x08;

// Error bits written by kernels into DevState::err (never a trap).
constexpr uint32_t kErrLookbackTimeout = 1u;
constexpr uint32_t kErrHashOverflow = 2u;
constexpr uint32_t kErrHashMissing = 4u;
constexpr uint32_t kErrCapacity = 8u;
constexpr uint32_t kErrIdRange = 16u;  // a batch row's journey id is outside [-2^57, 2^57)

// Device-side counters and status of one batch.
struct DevState {
  uint32_t err;
  uint32_t n_distinct;  // distinct journey ids seen by the hash table
  uint32_t n_runs;      // cell runs emitted by the journey kernel
  uint32_t n_cells;
  uint32_t n_big;       // journeys taking the chunked-sort path
  uint32_t n_touched;   // stream mode: journeys with points finalised by this window
  uint32_t n_long;      // stream mode: of those, the ones above the 64-thread journey kernel's limit
  unsigned long long n_malformed;
  unsigned long long n_dup;
  unsigned long long n_offgrid;
  unsigned long long n_too_late;  // stream mode: records older than the previous watermark
  uint32_t n_final, n_pending;    // stream mode: finalised / still pending after a window's split
  uint32_t n_appended;            // stream mode: rows the window's extract appended
  // largest key and largest complemented key among the collected journey ids: the ids' sort
  // covers only the bits below the highest bit where the smallest and largest key differ
  unsigned long long key_max, key_nmin;
};

// Folds every lane's largest and smallest key into DevState's key_max / key_nmin (one atomic
// pair per warp). All lanes of the warp call it; has = false lanes contribute nothing.
__device__ __forceinline__ void warp_key_span(bool has, unsigned long long kmax, unsigned long long kmin,
                                              DevState* st) {
  unsigned long long mx = has ? kmax : 0ull, nmn = has ? ~kmin : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nmn = max(nmn, __shfl_xor_sync(0xffffffffu, nmn, o));
  }
  if ((threadIdx.x & 31) == 0 && (mx | nmn)) {
    atomicMax(&st->key_max, mx);
    atomicMax(&st->key_nmin, nmn);
  }
}

// One extracted record, bucketed by journey: 32 bytes, one DRAM sector, written by one store
// (a separate 4-byte array would take a partial-sector write per record at a random address).
struct __align__(32) Rec {
  int64_t ts;
  double lat;
  double lon;
  float spd;     // canonical speed (+0.0 for -0.0)
  uint32_t idx;  // extracted-row index: the tie-break of equal timestamps, the materialised permutation
};
static_assert(sizeof(Rec) == 32, "Rec must be one 32-byte sector");

// The bit pattern of a double, moved through PTX so that integer operations on it stay integer
// operations: the compiler otherwise recognises sign-bit masks of a reinterpreted double as
// binary64 negations and absolute values, which run on the binary64 pipe.
__device__ __forceinline__ unsigned long long dbits(double x) {
  unsigned long long b;
  asm("mov.b64 %0, %1;" : "=l"(b) : "d"(x));
  return b;
}
__device__ __forceinline__ double dfrom(unsigned long long b) {
  double x;
  asm("mov.b64 %0, %1;" : "=d"(x) : "l"(b));
  return x;
}

// float -> double by the bit layout, exact for every float (denormals included), without a
// conversion instruction on the binary64 pipe.
__device__ __forceinline__ double f32_to_f64_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t ex = (b >> 23) & 0xFFu, man = b & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  if (ex == 0xFFu) return dfrom(sign | 0x7FF0000000000000ull | ((unsigned long long)man << 29));
  if (ex == 0) {
    if (man == 0) return dfrom(sign);
    const int L = 32 - __clz((int)man);  // man = 1.x * 2^(L-1): the value is 2^(L-150) * 1.x
    return dfrom(sign | ((unsigned long long)(873 + L) << 52) | (((unsigned long long)man << (53 - L)) & 0xFFFFFFFFFFFFFull));
  }
  return dfrom(sign | ((unsigned long long)(ex + 896) << 52) | ((unsigned long long)man << 29));
}

// Order-preserving map of a double onto uint64 (for finite values and +-inf).
__host__ __device__ __forceinline__ uint64_t ord_f64(double x) {
#ifdef __CUDA_ARCH__
  uint64_t b = dbits(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
#endif
  return (b & kSign64) ? ~b : (b | kSign64);
}

// The conversion instruction (it runs on the binary64 pipe), out of line so that the compiler
// cannot turn the rare branch that needs it into a conversion on every call.
__device__ __noinline__ float f64_to_f32_rare(double x) { return (float)x; }

// 64-bit integer -> float conversions run on the binary64 pipe too: the rare wide cases call
// these, out of line for the same reason.
__device__ __noinline__ float u64_to_f32_rz_rare(unsigned long long x) { return __ull2float_rz(x); }
__device__ __noinline__ float i64_to_f32_rare(long long x) { return (float)x; }

// double -> float rounded to nearest even by the bit layout when the result is a normal float
// (other values take the conversion instruction).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = dbits(x);
  const uint32_t hi = (uint32_t)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7FF);
  if (e < 1023 - 126 || e > 1023 + 127) return f64_to_f32_rare(x);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  uint32_t keep = (uint32_t)(m >> 29);
  const unsigned long long rest = m & ((1ull << 29) - 1), half = 1ull << 28;
  keep += (rest > half || (rest == half && (keep & 1u))) ? 1u : 0u;
  // a mantissa carry moves into the exponent (and to infinity past the largest float)
  return __uint_as_float((hi & 0x80000000u) | (((uint32_t)(e - 1023 + 127) << 23) + keep));
}
// The same, with zeros (frequent among parsed speeds) also kept off the binary64 pipe.
__device__ __forceinline__ float f64_to_f32_rn_z(double x) {
  const unsigned long long b = dbits(x);
  if ((b << 1) == 0) return __uint_as_float((uint32_t)(b >> 32));  // +-0
  return f64_to_f32_rn(x);
}

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// The lanes of the warp whose label equals this lane's (labels below 2^BITS), by one ballot
// per label bit: a label's peers agree with it on every bit. A few full-rate vote instructions
// in place of one match.any, which is far slower per instruction.
template <int BITS>
__device__ __forceinline__ uint32_t match_label(uint32_t label) {
  uint32_t m = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < BITS; ++b) {
    const bool bit = (label >> b) & 1u;
    const uint32_t v = __ballot_sync(0xffffffffu, bit);
    m &= bit ? v : ~v;
  }
  return m;
}

// atomicAdd(ctr, 1) for each lane that calls it, as one atomic per warp (the lanes of a warp
// that reach it together): returns the lane's own slot, in lane order.
__device__ __forceinline__ uint32_t warp_inc(uint32_t* ctr) {
  const uint32_t active = __activemask();
  const int leader = __ffs(active) - 1;
  uint32_t base = 0;
  if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(ctr, (uint32_t)__popc(active));
  base = __shfl_sync(active, base, leader);
  return base + (uint32_t)__popc(active & lanemask_lt());
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Inclusive warp scan (Hillis-Steele with shuffles).
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan over a block of NT threads (one value each). scratch: NT/32 + 1 words.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* scratch, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = warp_incl_scan(v);
  if (lane == 31) scratch[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < NT / 32) ? scratch[lane] : 0u;
    uint32_t wi = warp_incl_scan(w);
    if (lane < NT / 32) scratch[lane] = wi - w;
    if (lane == NT / 32 - 1) scratch[NT / 32] = wi;
  }
  __syncthreads();
  uint32_t r = scratch[warp] + inc - v;
  if (total) *total = scratch[NT / 32];
  __syncthreads();
  return r;
}

// Deterministic block sum (fixed shuffle tree, then warp partials in order).
template <int NT, typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  T r = T(0);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) r += scratch[w];
  }
  __syncthreads();
  return r;  // valid in thread 0
}

}  // namespace cvetl
