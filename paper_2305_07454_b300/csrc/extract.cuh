// extract.cuh — validation of binary columns, journey counting in an open-addressing hash
// table, ranking of distinct journey ids, and the scatter of every kept record into its
// journey's bucket as one 32-byte record.
#pragma once
#include "common.cuh"
#include "keying.cuh"

namespace cvetl {

constexpr uint64_t kHashEmpty = ~0ull;  // bit pattern of id -1 (the table is filled with 0xFF); that id uses slot `cap`
constexpr int kMaxProbe = 4096;

struct Hash {
  unsigned long long* keys;  // cap entries (+1 unused)
  uint32_t* cnt;             // cap + 1 counts
  uint32_t* aux;             // cap + 1 scatter cursors
  uint32_t mask;             // cap - 1
  uint32_t cap;
};

// A kept row has finite lat, lon and speed with |lat| <= 90 and |lon| <= 180. Tested on the bit
// patterns: |x| <= c for c >= 0 is (bits(x) & ~sign) <= bits(c), which also rejects NaN/inf.
__device__ __forceinline__ bool row_valid(double lat, double lon, float spd) {
  const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long b90 = 0x4056800000000000ull;   // 90.0
  const unsigned long long b180 = 0x4066800000000000ull;  // 180.0
  unsigned long long la = dbits(lat) & kAbs;
  unsigned long long lo = dbits(lon) & kAbs;
  uint32_t sp = (uint32_t)__float_as_int(spd) & 0x7FFFFFFFu;
  return la <= b90 && lo <= b180 && sp < 0x7F800000u;
}

__device__ __forceinline__ float canon_speed(float s) {
  return ((__float_as_int(s) & 0x7FFFFFFF) == 0) ? 0.0f : s;
}

// A slot's key read through L1. A slot only ever changes from empty to a key (by the CAS below),
// so a stale copy can only read empty: the CAS then returns the slot's key and the probe goes on
// from the right value. Cached reads save the L2 round trip of the slots L1 still holds.
__device__ __forceinline__ uint64_t ld_slot_key(const unsigned long long* p) {
  uint64_t v;
  asm volatile("ld.global.ca.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ int64_t hash_insert(const Hash& h, uint64_t key, uint32_t* n_distinct) {
  if (key == kHashEmpty) return (int64_t)h.cap;
  uint32_t s = (uint32_t)fmix64(key) & h.mask;
  for (int p = 0; p < kMaxProbe; ++p) {
    uint64_t k = ld_slot_key(&h.keys[s]);
    if (k == key) return s;
    if (k == kHashEmpty) {
      unsigned long long prev = atomicCAS(&h.keys[s], (unsigned long long)kHashEmpty,
                                          (unsigned long long)key);
      if (prev == kHashEmpty) {
        atomicAdd(n_distinct, 1u);
        return s;
      }
      if (prev == key) return s;
    }
    s = (s + 1) & h.mask;
  }
  return -1;
}

__device__ __forceinline__ int64_t hash_find(const Hash& h, uint64_t key) {
  if (key == kHashEmpty) return (int64_t)h.cap;
  uint32_t s = (uint32_t)fmix64(key) & h.mask;
  for (int p = 0; p < kMaxProbe; ++p) {
    uint64_t k = h.keys[s];
    if (k == key) return s;
    if (k == kHashEmpty) return -1;
    s = (s + 1) & h.mask;
  }
  return -1;
}

// U rows per thread per iteration keep U independent probe / atomic chains in flight (2, 4 or 8)
// in blocks of NT threads (128, 256 or 512), both chosen by the tuner.

template <int U, int NT>
__global__ void __launch_bounds__(NT) k_hash_count(const int64_t* __restrict__ jid,
                                                    const double* __restrict__ lat,
                                                    const double* __restrict__ lon,
                                                    const float* __restrict__ spd, uint32_t n,
                                                    Hash h, Batch bt, uint32_t* __restrict__ row_slot,
                                                    DevState* st) {
  __shared__ unsigned long long scratch[NT / 32];
  unsigned long long bad = 0;
  const uint32_t step = gridDim.x * blockDim.x * U;
  for (uint32_t i0 = blockIdx.x * blockDim.x * U + threadIdx.x; i0 < n; i0 += step) {
    uint64_t id[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = i0 + u * blockDim.x;
      // a batch row's instance; its columns (the concatenated ones, or the instance's own)
      const int k = (bt.n_inst && i < n) ? inst_of_row(bt, i) : 0;
      RowCols c;
      const uint32_t r = row_cols(bt, RowCols{jid, nullptr, lat, lon, spd}, i, k, c);
      ok[u] = i < n && row_valid(c.lat[r], c.lon[r], c.spd[r]);
      id[u] = (i < n) ? (uint64_t)c.jid[r] : 0;
      if (i < n && !ok[u]) ++bad;
      if (ok[u] && bt.n_inst && !composite_id(k, (int64_t)id[u], &id[u])) {
        atomicOr(&st->err, kErrIdRange);
        ok[u] = false;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = i0 + u * blockDim.x;
      uint32_t slot = kKeyInvalid;  // dropped row
      if (ok[u]) {
        int64_t s = hash_insert(h, id[u], &st->n_distinct);
        if (s < 0) atomicOr(&st->err, kErrHashOverflow);
        else {
          atomicAdd(&h.cnt[s], 1u);
          slot = (uint32_t)s;
        }
      }
      if (i < n) row_slot[i] = slot;
    }
  }
  unsigned long long b = block_sum<NT, unsigned long long>(bad, scratch);
  if (threadIdx.x == 0 && b) atomicAdd(&st->n_malformed, b);
}

// Distinct ids (as order-preserving keys) and their slots, in arbitrary order.
__global__ void k_collect_slots(Hash h, unsigned long long* __restrict__ ukey,
                                uint32_t* __restrict__ uslot, uint32_t* counter, DevState* st) {
  unsigned long long kmax = 0, knmin = 0;  // this thread's span of keys
  bool any = false;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= h.cap; s += gridDim.x * blockDim.x) {
    bool occ;
    uint64_t id;
    if (s < h.cap) {
      id = h.keys[s];
      occ = id != kHashEmpty;
    } else {
      id = kHashEmpty;
      occ = h.cnt[s] > 0;
    }
    if (occ) {
      uint32_t i = atomicAdd(counter, 1u);
      const unsigned long long k = id ^ kSign64;  // signed order as unsigned order
      ukey[i] = k;
      uslot[i] = s;
      kmax = max(kmax, k);
      knmin = max(knmin, ~k);
      any = true;
    }
  }
  warp_key_span(any, kmax, ~knmin, st);
}

// Journey rank r (ascending id): size, id (a batch's (instance, id) is unpacked).
// slot_rank (may be null) receives each hash slot's journey rank.
__global__ void k_journey_sizes(const unsigned long long* __restrict__ skey,
                                const uint32_t* __restrict__ sslot, uint32_t J, Hash h,
                                uint32_t* __restrict__ jn, int64_t* __restrict__ jid_out, int batched,
                                uint32_t* __restrict__ slot_rank) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < J) {
    jn[r] = h.cnt[sslot[r]];
    if (slot_rank) slot_rank[sslot[r]] = r;
    const uint64_t id = skey[r] ^ kSign64;
    jid_out[r] = batched ? composite_jid(id) : (int64_t)id;
  }
}

// One block for J <= kOffsetsMax journeys (a stream window's): each journey's size, its offset
// (exclusive prefix of the sizes), its bucket cursor and the total, in one launch instead of the
// three of the general path. Thread t takes journeys 4t .. 4t + 3.
constexpr int kOffsetsBlock = 1024;
constexpr uint32_t kOffsetsMax = 4u * kOffsetsBlock;
__global__ void __launch_bounds__(kOffsetsBlock) k_journey_offsets(const uint32_t* __restrict__ sslot, uint32_t J,
                                                                   Hash h, uint32_t* __restrict__ jn,
                                                                   uint32_t* __restrict__ joff,
                                                                   uint32_t* __restrict__ total) {
  __shared__ uint32_t scratch[kOffsetsBlock / 32 + 1];
  const uint32_t r0 = 4u * threadIdx.x;
  uint32_t c[4], sum = 0, tot = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    c[u] = (r0 + u < J) ? h.cnt[sslot[r0 + u]] : 0u;
    sum += c[u];
  }
  uint32_t base = block_excl_scan<kOffsetsBlock>(sum, scratch, &tot);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const uint32_t r = r0 + u;
    if (r < J) {
      jn[r] = c[u];
      joff[r] = base;
      h.aux[sslot[r]] = base;
    }
    base += c[u];
  }
  if (threadIdx.x == 0) *total = tot;
}

__global__ void k_journey_cursors(const uint32_t* __restrict__ sslot, uint32_t J,
                                  const uint32_t* __restrict__ joff, Hash h) {
  uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < J) h.aux[sslot[r]] = joff[r];
}

// Every kept row goes to its journey's bucket (the order inside a bucket is arbitrary; the
// journey kernel sorts it by (timestamp, row index)). The counting pass left each row's hash
// slot (or kKeyInvalid for a dropped row), so no probe is needed here. U rows per thread per
// iteration keep U atomic -> store chains in flight. Each record, with its row index, is one
// 32-byte store at the bucket cursor: consecutive cursor positions of a journey are written in
// the order the atomics hand them out, so L2 assembles whole lines before writing them back.
template <int U, int NT>
__global__ void __launch_bounds__(NT) k_scatter(const int64_t* __restrict__ ts,
                                                 const double* __restrict__ lat,
                                                 const double* __restrict__ lon,
                                                 const float* __restrict__ spd,
                                                 const uint32_t* __restrict__ row_slot, uint32_t n,
                                                 Hash h, Batch bt, Rec* __restrict__ rec) {
  const uint32_t step = gridDim.x * blockDim.x * U;
  for (uint32_t i0 = blockIdx.x * blockDim.x * U + threadIdx.x; i0 < n; i0 += step) {
    uint32_t slot[U], pos[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = i0 + u * blockDim.x;
      slot[u] = (i < n) ? row_slot[i] : kKeyInvalid;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      pos[u] = (slot[u] != kKeyInvalid) ? atomicAdd(&h.aux[slot[u]], 1u) : 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (slot[u] == kKeyInvalid) continue;
      const uint32_t i = i0 + u * blockDim.x;
      RowCols q;
      const uint32_t r = row_cols(bt, RowCols{nullptr, ts, lat, lon, spd}, i, bt.cols ? inst_of_row(bt, i) : 0, q);
      const unsigned long long a = (unsigned long long)q.ts[r];
      const unsigned long long b = (unsigned long long)__double_as_longlong(q.lat[r]);
      const unsigned long long c = (unsigned long long)__double_as_longlong(q.lon[r]);
      const unsigned long long d = (unsigned long long)(uint32_t)__float_as_int(canon_speed(q.spd[r])) |
                                   ((unsigned long long)i << 32);
      asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(rec + pos[u]), "l"(a), "l"(b),
                   "l"(c), "l"(d)
                   : "memory");
    }
  }
}

// The same scatter with each thread on R (a multiple of 4) consecutive rows per iteration, the
// columns read with 32-byte (timestamp, latitude, longitude) and 16-byte (speed, slot) vector
// loads: a sixteenth of the load instructions with R = 16, for a kernel whose warps wait on the
// load-store queue. Needs the five columns and the slots 32- / 16-byte aligned and the rows in
// one set of columns (not a batch read in place); rows past the last full group go one per
// thread.
__device__ __forceinline__ void ld_v4_b64(const void* p, unsigned long long& a, unsigned long long& b,
                                          unsigned long long& c, unsigned long long& d) {
  asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}

constexpr int kScatterRows = 16;  // R of the launched kernel

template <int NT, int R>
__global__ void __launch_bounds__(NT) k_scatter_rows(const int64_t* __restrict__ ts, const double* __restrict__ lat,
                                                     const double* __restrict__ lon, const float* __restrict__ spd,
                                                     const uint32_t* __restrict__ row_slot, uint32_t n, Hash h,
                                                     Rec* __restrict__ rec) {
  static_assert(R % 4 == 0, "rows per thread: a multiple of 4");
  const uint32_t ng = n / R;
  const uint32_t step = gridDim.x * NT;
  for (uint32_t q = blockIdx.x * NT + threadIdx.x; q < ng; q += step) {
    const uint32_t i = q * R;
    uint32_t slot[R], pos[R];
#pragma unroll
    for (int v = 0; v < R / 4; ++v) {
      const uint4 sl = __ldg(reinterpret_cast<const uint4*>(row_slot + i) + v);
      slot[4 * v] = sl.x;
      slot[4 * v + 1] = sl.y;
      slot[4 * v + 2] = sl.z;
      slot[4 * v + 3] = sl.w;
    }
#pragma unroll
    for (int u = 0; u < R; ++u) pos[u] = (slot[u] != kKeyInvalid) ? atomicAdd(&h.aux[slot[u]], 1u) : 0u;
    unsigned long long t[R], la[R], lo[R];
    float sp[R];
#pragma unroll
    for (int v = 0; v < R / 4; ++v) {
      ld_v4_b64(ts + i + 4 * v, t[4 * v], t[4 * v + 1], t[4 * v + 2], t[4 * v + 3]);
      ld_v4_b64(lat + i + 4 * v, la[4 * v], la[4 * v + 1], la[4 * v + 2], la[4 * v + 3]);
      ld_v4_b64(lon + i + 4 * v, lo[4 * v], lo[4 * v + 1], lo[4 * v + 2], lo[4 * v + 3]);
      const float4 s4 = __ldg(reinterpret_cast<const float4*>(spd + i) + v);
      sp[4 * v] = s4.x;
      sp[4 * v + 1] = s4.y;
      sp[4 * v + 2] = s4.z;
      sp[4 * v + 3] = s4.w;
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
      if (slot[u] == kKeyInvalid) continue;
      const unsigned long long d = (unsigned long long)(uint32_t)__float_as_int(canon_speed(sp[u])) |
                                   ((unsigned long long)(i + u) << 32);
      asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(rec + pos[u]), "l"(t[u]), "l"(la[u]),
                   "l"(lo[u]), "l"(d)
                   : "memory");
    }
  }
  // the last n mod R rows
  const uint32_t g = blockIdx.x * NT + threadIdx.x, i = ng * R + g;
  if (g < n % R && row_slot[i] != kKeyInvalid) {
    const uint32_t p = atomicAdd(&h.aux[row_slot[i]], 1u);
    const unsigned long long d = (unsigned long long)(uint32_t)__float_as_int(canon_speed(spd[i])) |
                                 ((unsigned long long)i << 32);
    asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(rec + p), "l"((unsigned long long)ts[i]),
                 "l"((unsigned long long)__double_as_longlong(lat[i])),
                 "l"((unsigned long long)__double_as_longlong(lon[i])), "l"(d)
                 : "memory");
  }
}

// The 16-row scatter for a batch read in place: row groups numbered per instance (an
// instance's last group may be partial), each thread's group found by binary search over the
// instances' first groups, the instance's column pointers read from the batch table (all of
// them aligned: checked when the batch was extracted). Slots are read one by one unless the
// group's first row is a multiple of 4.
template <int NT, int R>
__global__ void __launch_bounds__(NT) k_scatter_groups(const uint32_t* __restrict__ row_slot, uint32_t n,
                                                       uint32_t n_groups, Batch bt, Hash h, Rec* __restrict__ rec) {
  static_assert(R % 4 == 0, "rows per thread: a multiple of 4");
  const uint32_t step = gridDim.x * NT;
  for (uint32_t g = blockIdx.x * NT + threadIdx.x; g < n_groups; g += step) {
    const int k = inst_of_group(bt, g);
    const uint32_t row0 = __ldg(&bt.inst[k].row_begin);
    const uint32_t row1 = (k + 1 < bt.n_inst) ? __ldg(&bt.inst[k + 1].row_begin) : n;
    const uint32_t r = (g - __ldg(&bt.inst[k].group_begin)) * R;  // the group's first row in the instance
    const uint32_t i = row0 + r;                                    // and in the batch
    RowCols c;
    row_cols(bt, RowCols{}, i, k, c);
    if (r + R <= row1 - row0) {
      uint32_t slot[R], pos[R];
      if ((i & 3u) == 0) {
#pragma unroll
        for (int v = 0; v < R / 4; ++v) {
          const uint4 sl = __ldg(reinterpret_cast<const uint4*>(row_slot + i) + v);
          slot[4 * v] = sl.x;
          slot[4 * v + 1] = sl.y;
          slot[4 * v + 2] = sl.z;
          slot[4 * v + 3] = sl.w;
        }
      } else {
#pragma unroll
        for (int u = 0; u < R; ++u) slot[u] = __ldg(row_slot + i + u);
      }
#pragma unroll
      for (int u = 0; u < R; ++u) pos[u] = (slot[u] != kKeyInvalid) ? atomicAdd(&h.aux[slot[u]], 1u) : 0u;
      unsigned long long t[R], la[R], lo[R];
      float sp[R];
#pragma unroll
      for (int v = 0; v < R / 4; ++v) {
        ld_v4_b64(c.ts + r + 4 * v, t[4 * v], t[4 * v + 1], t[4 * v + 2], t[4 * v + 3]);
        ld_v4_b64(c.lat + r + 4 * v, la[4 * v], la[4 * v + 1], la[4 * v + 2], la[4 * v + 3]);
        ld_v4_b64(c.lon + r + 4 * v, lo[4 * v], lo[4 * v + 1], lo[4 * v + 2], lo[4 * v + 3]);
        const float4 s4 = __ldg(reinterpret_cast<const float4*>(c.spd + r) + v);
        sp[4 * v] = s4.x;
        sp[4 * v + 1] = s4.y;
        sp[4 * v + 2] = s4.z;
        sp[4 * v + 3] = s4.w;
      }
#pragma unroll
      for (int u = 0; u < R; ++u) {
        if (slot[u] == kKeyInvalid) continue;
        const unsigned long long d = (unsigned long long)(uint32_t)__float_as_int(canon_speed(sp[u])) |
                                     ((unsigned long long)(i + u) << 32);
        asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(rec + pos[u]), "l"(t[u]), "l"(la[u]),
                     "l"(lo[u]), "l"(d)
                     : "memory");
      }
    } else {  // the instance's partial last group
      for (uint32_t u = 0; r + u < row1 - row0; ++u) {
        const uint32_t s = row_slot[i + u];
        if (s == kKeyInvalid) continue;
        const uint32_t p = atomicAdd(&h.aux[s], 1u);
        const unsigned long long d = (unsigned long long)(uint32_t)__float_as_int(canon_speed(c.spd[r + u])) |
                                     ((unsigned long long)(i + u) << 32);
        asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(rec + p),
                     "l"((unsigned long long)c.ts[r + u]),
                     "l"((unsigned long long)__double_as_longlong(c.lat[r + u])),
                     "l"((unsigned long long)__double_as_longlong(c.lon[r + u])), "l"(d)
                     : "memory");
      }
    }
  }
}

}  // namespace cvetl
