// stream.cuh — stream mode: windows of records are appended to a device-resident pending
// store; each window finalises the pending points whose timestamp is at or below the watermark
// (window end - lateness), continuing every journey from its device-resident tail (last point,
// open run, running sums), and folds the window's closed runs into a device-resident cell table.
// A point at or below the watermark has arrived when its window closes (records are at most
// `lateness` late), so each journey is finalised in timestamp order and the tables after the
// last window equal those of one batch over the same records. Records older than the previous
// watermark when they arrive are dropped and counted as too late.
#pragma once
#include "common.cuh"
#include "extract.cuh"
#include "journey.cuh"
#include "cells.cuh"

namespace cvetl {

// Appends the window's kept rows to the pending store after its first p_base entries (the
// record carries its arrival index arrival_base + row; st->n_appended counts the appended rows);
// rows whose timestamp is below the previous watermark are dropped as too late.
__global__ void __launch_bounds__(256) k_stream_append(const int64_t* __restrict__ jid,
                                                       const int64_t* __restrict__ ts,
                                                       const double* __restrict__ lat,
                                                       const double* __restrict__ lon,
                                                       const float* __restrict__ spd, uint32_t n,
                                                       uint32_t arrival_base, int64_t w_prev,
                                                       int has_w_prev, int64_t* __restrict__ p_jid,
                                                       Rec* __restrict__ p_rec, uint32_t p_base,
                                                       uint32_t p_cap, DevState* st) {
  __shared__ unsigned long long scratch[8];
  unsigned long long bad = 0, late = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double la = lat[i], lo = lon[i];
    const float sp = spd[i];
    if (!row_valid(la, lo, sp)) {
      ++bad;
      continue;
    }
    const int64_t t = ts[i];
    if (has_w_prev && t < w_prev) {
      ++late;
      continue;
    }
    const uint32_t o = p_base + warp_inc(&st->n_appended);
    if (o >= p_cap) {
      atomicOr(&st->err, kErrCapacity);
      continue;
    }
    p_jid[o] = jid[i];
    Rec r;
    r.ts = t;
    r.lat = la;
    r.lon = lo;
    r.spd = canon_speed(sp);
    r.idx = arrival_base + i;
    p_rec[o] = r;
  }
  const unsigned long long b = block_sum<256, unsigned long long>(bad, scratch);
  const unsigned long long l = block_sum<256, unsigned long long>(late, scratch);
  if (threadIdx.x == 0) {
    if (b) atomicAdd(&st->n_malformed, b);
    if (l) atomicAdd(&st->n_too_late, l);
  }
}

// Splits the pending store: timestamps <= watermark go to the finalised list (with their hash
// slot and the count per journey; st->n_final), the rest to the next pending store
// (st->n_pending). The store holds n entries, or, with appended != nullptr, base + *appended of
// at most n (the count the window's extract left on the device).
__global__ void __launch_bounds__(256) k_stream_split(const int64_t* __restrict__ p_jid,
                                                      const Rec* __restrict__ p_rec, uint32_t n,
                                                      uint32_t base, const uint32_t* __restrict__ appended,
                                                      int64_t wm, int finalize_all, Hash h,
                                                      int64_t* __restrict__ q_jid, Rec* __restrict__ q_rec,
                                                      Rec* __restrict__ f_rec,
                                                      uint32_t* __restrict__ f_slot, DevState* st) {
  if (appended) n = min(n, base + *appended);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const Rec r = p_rec[i];
    const int64_t id = p_jid[i];
    if (finalize_all || r.ts <= wm) {
      const int64_t s = hash_insert(h, (uint64_t)id, &st->n_distinct);
      if (s < 0) {
        atomicOr(&st->err, kErrHashOverflow);
        continue;
      }
      atomicAdd(&h.cnt[s], 1u);
      const uint32_t o = warp_inc(&st->n_final);
      f_rec[o] = r;
      f_slot[o] = (uint32_t)s;
    } else {
      const uint32_t o = warp_inc(&st->n_pending);
      q_jid[o] = id;
      q_rec[o] = r;
    }
  }
}

// Journeys touched by this window (count > 0; st->n_touched), with their ids as order-preserving
// keys.
// lim > 0: also counts the journeys with more than lim points in this window (n_long), which
// tells the host whether the 256-thread journey kernel has work.
__global__ void k_stream_touched(Hash h, unsigned long long* __restrict__ ukey,
                                 uint32_t* __restrict__ uslot, DevState* st, uint32_t lim) {
  unsigned long long kmax = 0, knmin = 0;  // this thread's span of keys
  bool any = false;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= h.cap; s += gridDim.x * blockDim.x) {
    const uint32_t cnt = h.cnt[s];
    if (cnt == 0) continue;
    if (lim && cnt > lim) warp_inc(&st->n_long);
    const uint64_t id = (s < h.cap) ? h.keys[s] : kHashEmpty;
    const uint32_t i = atomicAdd(&st->n_touched, 1u);
    const unsigned long long k = id ^ kSign64;
    ukey[i] = k;
    uslot[i] = s;
    kmax = max(kmax, k);
    knmin = max(knmin, ~k);
    any = true;
  }
  warp_key_span(any, kmax, ~knmin, st);
}

__global__ void __launch_bounds__(256) k_stream_scatter(const Rec* __restrict__ f_rec,
                                                        const uint32_t* __restrict__ f_slot,
                                                        uint32_t n, Hash h, Rec* __restrict__ rec) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t pos = atomicAdd(&h.aux[f_slot[i]], 1u);
    rec[pos] = f_rec[i];
  }
}

// Every journey's open run is closed (end of the stream): emitted with a start marker that
// cannot collide with a window position.
__global__ void k_stream_close_runs(Hash h, JState js, unsigned long long* __restrict__ run_sortkey,
                                    uint32_t* __restrict__ run_cnt, double* __restrict__ run_sum,
                                    float* __restrict__ run_min, float* __restrict__ run_max,
                                    uint32_t run_cap, DevState* st) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= h.cap; s += gridDim.x * blockDim.x) {
    const bool occ = (s < h.cap) ? (h.keys[s] != kHashEmpty) : (js.n[s] > 0);
    if (!occ || js.n[s] == 0) continue;
    const uint32_t key = js.l_key[s], cnt = js.r_cnt[s];
    if (key == kKeyInvalid || cnt == 0) continue;
    const uint32_t i = atomicAdd(&st->n_runs, 1u);
    if (i >= run_cap) {
      atomicOr(&st->err, kErrCapacity);
      continue;
    }
    run_sortkey[i] = ((unsigned long long)key << 32) | (0x80000000u | s);
    run_cnt[i] = cnt;
    run_sum[i] = (double)js.r_s[s] + (double)js.r_c[s];
    run_min[i] = js.r_mn[s];
    run_max[i] = js.r_mx[s];
    js.r_cnt[s] = 0;
  }
}

// Cell table kept across windows: open addressing keyed by the cell key.
struct CellHash {
  uint32_t* keys;  // kKeyInvalid = empty
  uint32_t* count;
  double* sum;
  float *mn, *mx;
  uint32_t mask, cap;
};

__device__ __forceinline__ int64_t cell_slot(const CellHash& c, uint32_t key, uint32_t* n_cells) {
  uint32_t s = (uint32_t)fmix64(key) & c.mask;
  for (int p = 0; p < kMaxProbe; ++p) {
    const uint32_t k = ld_relaxed_u32(&c.keys[s]);
    if (k == key) return s;
    if (k == kKeyInvalid) {
      const uint32_t prev = atomicCAS(&c.keys[s], kKeyInvalid, key);
      if (prev == kKeyInvalid) {
        atomicAdd(n_cells, 1u);
        return s;
      }
      if (prev == key) return s;
    }
    s = (s + 1) & c.mask;
  }
  return -1;
}

// One thread per distinct key of the window's sorted runs: the window's aggregate of that key
// (runs in sorted order) is added to the table. Keys are distinct, so no two threads update one
// slot, and windows are folded in order: the result does not depend on thread timing.
__global__ void k_cell_fold(const unsigned long long* __restrict__ skey, const uint32_t* __restrict__ sidx,
                            uint32_t R, const uint32_t* __restrict__ head,
                            const uint32_t* __restrict__ run_cnt, const double* __restrict__ run_sum,
                            const float* __restrict__ run_min, const float* __restrict__ run_max,
                            CellHash c, uint32_t* n_cells, DevState* st) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R) return;
  // head == nullptr: a cell's first run is found here (its key differs from the previous run's)
  if (head ? !head[i] : (i > 0 && (skey[i] >> 32) == (skey[i - 1] >> 32))) return;
  const uint32_t key = (uint32_t)(skey[i] >> 32);
  uint32_t cnt = 0;
  double sum = 0.0;
  float mn = run_min[sidx[i]], mx = run_max[sidx[i]];
  for (uint32_t m = i; m < R && (uint32_t)(skey[m] >> 32) == key; ++m) {
    const uint32_t r = sidx[m];
    cnt += run_cnt[r];
    sum += run_sum[r];
    mn = fminf(mn, run_min[r]);
    mx = fmaxf(mx, run_max[r]);
  }
  const int64_t s = cell_slot(c, key, n_cells);
  if (s < 0) {
    atomicOr(&st->err, kErrHashOverflow);
    return;
  }
  if (c.count[s] == 0) {
    c.sum[s] = sum;
    c.mn[s] = mn;
    c.mx[s] = mx;
  } else {
    c.sum[s] += sum;
    c.mn[s] = fminf(c.mn[s], mn);
    c.mx[s] = fmaxf(c.mx[s], mx);
  }
  c.count[s] += cnt;
}

// Moves every entry of a cell table into a larger one.
__global__ void k_cell_rehash(CellHash from, CellHash to, uint32_t* n_cells, DevState* st) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < from.cap; s += gridDim.x * blockDim.x) {
    const uint32_t key = from.keys[s];
    if (key == kKeyInvalid) continue;
    const int64_t d = cell_slot(to, key, n_cells);
    if (d < 0) {
      atomicOr(&st->err, kErrHashOverflow);
      continue;
    }
    to.count[d] = from.count[s];
    to.sum[d] = from.sum[s];
    to.mn[d] = from.mn[s];
    to.mx[d] = from.mx[s];
  }
}

// Occupied cells (key, slot), in arbitrary order.
__global__ void k_cell_collect(CellHash c, unsigned long long* __restrict__ ukey,
                               uint32_t* __restrict__ uslot, uint32_t* counter) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < c.cap; s += gridDim.x * blockDim.x) {
    const uint32_t key = c.keys[s];
    if (key == kKeyInvalid) continue;
    const uint32_t i = atomicAdd(counter, 1u);
    ukey[i] = key;
    uslot[i] = s;
  }
}

// Moves every journey of a journey hash (and its state) into a larger table.
__global__ void k_journey_rehash(Hash from, JState a, Hash to, JState b, uint32_t* n_distinct,
                                 DevState* st) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= from.cap; s += gridDim.x * blockDim.x) {
    const bool occ = (s < from.cap) ? (from.keys[s] != kHashEmpty) : (a.n[s] > 0);
    if (!occ) continue;
    const uint64_t id = (s < from.cap) ? from.keys[s] : kHashEmpty;
    const int64_t d = hash_insert(to, id, n_distinct);
    if (d < 0) {
      atomicOr(&st->err, kErrHashOverflow);
      continue;
    }
    b.n[d] = a.n[s];
    b.start_ts[d] = a.start_ts[s];
    b.end_ts[d] = a.end_ts[s];
    b.dwell[d] = a.dwell[s];
    b.dist[d] = a.dist[s];
    b.slat[d] = a.slat[s];
    b.slon[d] = a.slon[s];
    b.l_ts[d] = a.l_ts[s];
    b.l_lat[d] = a.l_lat[s];
    b.l_lon[d] = a.l_lon[s];
    b.l_spd[d] = a.l_spd[s];
    b.l_key[d] = a.l_key[s];
    b.r_cnt[d] = a.r_cnt[s];
    b.r_s[d] = a.r_s[s];
    b.r_c[d] = a.r_c[s];
    b.r_mn[d] = a.r_mn[s];
    b.r_mx[d] = a.r_mx[s];
  }
}

// Journeys seen so far (id as order-preserving key, slot), in arbitrary order.
__global__ void k_journey_collect(Hash h, JState js, unsigned long long* __restrict__ ukey,
                                  uint32_t* __restrict__ uslot, uint32_t* counter) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= h.cap; s += gridDim.x * blockDim.x) {
    const bool occ = (s < h.cap) ? (h.keys[s] != kHashEmpty) : (js.n[s] > 0);
    if (!occ || js.n[s] == 0) continue;
    const uint64_t id = (s < h.cap) ? h.keys[s] : kHashEmpty;
    const uint32_t i = atomicAdd(counter, 1u);
    ukey[i] = id ^ kSign64;
    uslot[i] = s;
  }
}

// Result tables from the device-resident tables (cells by ascending key, journeys by id).
__global__ void k_cell_table_from_hash(const unsigned long long* __restrict__ skey,
                                       const uint32_t* __restrict__ sslot, uint32_t K, CellHash ch,
                                       int32_t n_rows, int32_t n_cols, CellOut o) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  const uint32_t key = (uint32_t)skey[i], s = sslot[i];
  const uint32_t cells = (uint32_t)n_rows * (uint32_t)n_cols;
  o.key[i] = key;
  o.bin[i] = (int32_t)(key / cells);
  o.row[i] = (int32_t)((key % cells) / (uint32_t)n_cols);
  o.col[i] = (int32_t)(key % (uint32_t)n_cols);
  o.count[i] = ch.count[s];
  o.sum[i] = ch.sum[s];
  o.mean[i] = ch.sum[s] / (double)ch.count[s];
  o.min[i] = ch.mn[s];
  o.max[i] = ch.mx[s];
}

__global__ void k_journey_n32(const uint32_t* __restrict__ sslot, uint32_t J, JState js,
                              uint32_t* __restrict__ n32) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < J) n32[r] = (uint32_t)js.n[sslot[r]];
}

__global__ void k_journey_table_from_state(const unsigned long long* __restrict__ skey,
                                           const uint32_t* __restrict__ sslot, uint32_t J, JState js,
                                           const uint32_t* __restrict__ off32, int64_t* __restrict__ jid,
                                           JourneyOut o) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= J) return;
  const uint32_t s = sslot[r];
  jid[r] = (int64_t)(skey[r] ^ kSign64);
  o.n[r] = js.n[s];
  o.off[r] = off32[r];
  o.start_ts[r] = js.start_ts[s];
  o.end_ts[r] = js.end_ts[s];
  o.duration[r] = (int64_t)((unsigned long long)js.end_ts[s] - (unsigned long long)js.start_ts[s]);
  o.dist[r] = js.dist[s];
  o.dwell[r] = js.dwell[s];
  o.slat[r] = js.slat[s];
  o.slon[r] = js.slon[s];
  o.elat[r] = js.l_lat[s];
  o.elon[r] = js.l_lon[s];
}

}  // namespace cvetl
