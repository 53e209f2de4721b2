// cvetl.cu — the C ABI (include/cvetl.h): context, device buffers and the launch sequence of
// the extract / transform / load kernels.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "cvetl.h"

#include "common.cuh"
#include "radix_sort.cuh"
#include "cta_sort.cuh"
#include "scan.cuh"
#include "extract.cuh"
#include "journey.cuh"
#include "cells.cuh"
#include "csv.cuh"
#include "stream.cuh"
#include "lattice.cuh"
#include "probe.cuh"

using namespace cvetl;

namespace {

enum Stage {
  ST_HASH, ST_COLLECT, ST_SORT_HIST, ST_SORT_PASS, ST_SIZES, ST_SCAN, ST_CURSORS, ST_SCATTER,
  ST_JOURNEYS, ST_CELL_HEADS, ST_CELL_WRITE, ST_CSV_COUNT, ST_CSV_PARSE, ST_STREAM_APPEND,
  ST_STREAM_SPLIT, ST_STREAM_TABLES, ST_CTA_SORT, ST_LATTICE, ST_POINT_EXTRAS, ST_LATTICE_KEYS,
  ST_LATTICE_FOLD, ST_JOURNEY_SORT, ST_JOURNEY_WALK, ST_COUNT
};
const char* kStageNames[ST_COUNT] = {"hash_count", "collect_slots", "radix_histogram",
                                     "radix_onesweep", "journey_sizes", "scan", "journey_cursors",
                                     "scatter", "journeys", "cell_heads", "cell_write",
                                     "csv_count", "csv_parse", "stream_append", "stream_split",
                                     "stream_tables", "cta_sort", "lattice", "point_extras", "lattice_keys",
                                     "lattice_fold", "journey_sort", "journey_walk"};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

std::string g_create_error;

}  // namespace

struct cvetl_ctx {
  cvetl_config cfg{};
  cudaStream_t st = nullptr;
  std::string err;
  int state = 0;  // 0 empty, 1 extracted, 2 transformed, 3 loaded
  size_t held = 0;
  std::map<std::string, DevBuf> bufs;
  // extracted columns (n_rows of them) from n_in input rows or lines
  int64_t n_in = 0, n_rows = 0, csv_malformed = 0;
  const float* heading = nullptr;
  const int64_t* jid = nullptr;
  const int64_t* ts = nullptr;
  const double* lat = nullptr;
  const double* lon = nullptr;
  const float* spd = nullptr;
  // keying tables
  unsigned long long* row_thr = nullptr;
  unsigned long long* col_thr = nullptr;
  GridParams gp{};
  // device status and its pinned host mirror
  DevState* dstate = nullptr;
  DevState* hstate = nullptr;
  uint32_t J = 0, R = 0, K = 0, n_valid = 0;
  // outputs
  JourneyOut jo{};
  CellOut co{};
  LatticeOut lattice{};
  int64_t* jid_sorted = nullptr;
  // batch of instances (cvetl_extract_batch); bt.n_inst = 0 for one instance
  Batch bt{};
  std::vector<int64_t> inst_rows, inst_keys;  // first row / key of each instance, + the totals
  std::vector<int64_t> inst_cells, inst_journeys;  // first cell / journey row (after cvetl_load)
  uint32_t* inst_counts = nullptr;  // device: journeys [kMaxInst], then cells [kMaxInst]
  uint32_t* cell_total = nullptr;   // device: the cell count of the last batch
  uint32_t hint_distinct = 0;       // journeys of the last batch (sizes the next hash table)
  uint32_t* slot_rank = nullptr;    // journey rank of each hash slot (last batch)
  uint32_t* row_slot = nullptr;     // hash slot of each extracted row (last batch)
  int id_bits = 64;                 // bits the journey-id sort covers (from the ids' key span)
  std::vector<double> batch_key;    // the last batch's instance grids and sizes
  size_t batch_groups = 0;          // row groups of the batch (kScatterRows rows per instance-local group)
  bool batch_aligned = false;       // a batch read in place whose columns all suit the vector loads
  // stream mode
  struct {
    bool flushed = false, has_w_prev = false;
    bool unread_append = false;  // the last extract's counters are still on the device
    int64_t w_prev = 0, window_end = 0;
    uint32_t arrival = 0, n_pending = 0, n_window = 0;
    int side = 0, jgen = 0, cgen = 0;
    Hash jh{};
    JState js{};
    CellHash ch{};
    uint32_t n_journeys = 0, n_cells = 0;
    int64_t tot_malformed = 0, tot_late = 0, tot_dup = 0, tot_off = 0, tot_final = 0, tot_runs = 0;
  } ss;
  // launch shapes (cvetl_tuning); results do not depend on them
  struct {
    int journey_ctas = 0;      // persistent journey CTAs per SM (1..3); 0: one CTA per journey
    int row_unroll = 4;        // rows per thread per iteration of the counting pass and the scatter
    int row_block = 256;       // threads per block of the counting pass (and the unaligned scatter)
    int small_sort_max = 4096;  // pairs up to which one block sorts (0..kCtaSortMax)
    int small_journey_max = 512;  // journeys of up to this many points take 64-thread CTAs (0: none)
    int scatter_block = 128;   // threads per block of the 16-row scatter (aligned columns)
  } tune;
  // CUDA graphs of the batch path after sizing (config.graph), one per shape
  struct GraphKey {
    uint64_t n, J, nv, cap, gen;
    const void* cols[5];
    const void* inst;
    int n_inst, precision, materialize, t0, t1, t2, id_bits, aligned;
    bool operator==(const GraphKey& o) const { return memcmp(this, &o, sizeof o) == 0; }
  };
  struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
    int64_t launches[ST_COUNT];
  };
  std::vector<GraphEntry> graphs;
  bool capturing = false;       // a graph capture is in progress on the stream
  cudaStream_t cap_stream = nullptr;  // captures run here (the legacy default stream cannot be captured)
  int64_t cap_launches[ST_COUNT] = {};
  uint64_t buf_gen = 0;         // bumped whenever a device buffer moves
  int64_t graph_replays = 0;
  // statistics
  int64_t launches[ST_COUNT] = {};
  double ms[ST_COUNT] = {};
  int64_t total_launches = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> event_pool;
  cudaEvent_t copy_ev = nullptr;  // stream mode: a window's host columns copied
};

namespace {

cvetl_status fail(cvetl_ctx* c, cvetl_status s, const char* fmt, ...) {
  char b[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b, sizeof b, fmt, ap);
  va_end(ap);
  if (c) c->err = b;
  else g_create_error = b;
  return s;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(c, CVETL_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

cudaEvent_t take_event(cvetl_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct LaunchScope {
  cvetl_ctx* c;
  int stage;
  cudaEvent_t a = nullptr, b = nullptr;
  LaunchScope(cvetl_ctx* c_, int s) : c(c_), stage(s) {
    if (c->capturing) {  // counted when the graph is launched; no per-kernel events in a graph
      c->cap_launches[s] += 1;
      return;
    }
    c->launches[s] += 1;
    c->total_launches += 1;
    if (c->cfg.profile) {
      a = take_event(c);
      b = take_event(c);
      cudaEventRecord(a, c->st);
    }
  }
  ~LaunchScope() {
    if (a) {
      cudaEventRecord(b, c->st);
      c->pending.push_back({stage, {a, b}});
    }
  }
};

#define LAUNCH(stage, ...)                          \
  do {                                              \
    LaunchScope ls_(c, stage);                      \
    __VA_ARGS__;                                    \
  } while (0)

#define LAUNCH_CHECK()                                                                        \
  do {                                                                                        \
    cudaError_t e_ = cudaGetLastError();                                                      \
    if (e_ != cudaSuccess) return fail(c, CVETL_ECUDA, "kernel launch: %s", cudaGetErrorString(e_)); \
  } while (0)

// Grow-only named device buffer. On success *out holds at least `bytes`.
// Size of a buffer that must hold `bytes`: bytes + bytes / frac at its first allocation and
// above 256 MB (a batch's buffers, sized once per workload); twice `bytes` when a smaller buffer
// grows again, so that the buffers of a stream of windows growing through the day move a few
// times instead of at every larger window (each move frees and allocates, which synchronises
// the device and stalls every other context on it).
inline size_t grow_to(size_t bytes, size_t frac, bool again) {
  return (again && bytes < ((size_t)256 << 20)) ? 2 * bytes : bytes + bytes / frac;
}

template <typename T>
cvetl_status ensure(cvetl_ctx* c, const char* name, size_t count, T** out) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 256;
  DevBuf& b = c->bufs[name];
  if (b.bytes < bytes) {
    if (c->capturing) return fail(c, CVETL_ECUDA, "internal: buffer %s would move during a graph capture", name);
    c->buf_gen += 1;
    size_t grow = grow_to(bytes, 8, b.bytes > 0);
    size_t after = c->held - b.bytes + grow;
    if (c->cfg.mem_budget_bytes && after > c->cfg.mem_budget_bytes) {
      return fail(c, CVETL_EFULL, "buffer %s needs %zu bytes; the context holds %zu of a %zu budget",
                  name, grow, c->held, c->cfg.mem_budget_bytes);
    }
    if (b.p) {
      cudaStreamSynchronize(c->st);
      cudaFree(b.p);
      c->held -= b.bytes;
      b.p = nullptr;
      b.bytes = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, grow) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CVETL_ENOMEM, "cudaMalloc(%zu) for %s failed", grow, name);
    }
    b.p = p;
    b.bytes = grow;
    c->held += grow;
  }
  *out = reinterpret_cast<T*>(b.p);
  return CVETL_OK;
}

#define ENSURE(name, count, ptr)                          \
  do {                                                    \
    cvetl_status s_ = ensure(c, name, (count), (ptr));    \
    if (s_ != CVETL_OK) return s_;                        \
  } while (0)

// Resident blocks per SM of a kernel (at least 1).
template <typename F>
int occupancy(F kernel, int block, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess) per_sm = 1;
  return per_sm > 0 ? per_sm : 1;
}

constexpr int kSortBlockB = 512;  // threads of the 4097-8192 class
constexpr int kSortSmemB = cmax(staged_smem<8192>(), 4096 * 16);  // its fallback's pair sort chunk
constexpr int kSortBlockC = 512;  // threads of the 513-4096 class
constexpr int kSortSmemC = cmax(cmax(staged_smem<4096>(), kJSmem), 4096 * 16);
constexpr int kSortSmemD = cmax(staged_smem<512>(), kJSmallSmem);

int grid_for(size_t n, int block, int max_blocks_per_sm = 8) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t want = (n + block - 1) / block;
  size_t cap = (size_t)sms * max_blocks_per_sm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

// ---- host keying tables ---------------------------------------------------------------
double from_ord(unsigned long long u) {
  unsigned long long b = (u & kSign64) ? (u ^ kSign64) : ~u;
  double x;
  memcpy(&x, &b, 8);
  return x;
}

// floor(RN(RN(x - xmin) / step)) in binary64; the host build has FMA contraction off.
double bin_f64(double x, double xmin, double step) {
  volatile double d = x - xmin;
  volatile double q = d / step;
  return std::floor(q);
}

// Smallest binary64 x (as an order-preserving key) with bin_f64(x) >= k.
unsigned long long threshold(double xmin, double step, int k) {
  unsigned long long lo = ord_f64(-DBL_MAX), hi = ord_f64(INFINITY);
  while (lo < hi) {
    unsigned long long mid = lo + (hi - lo) / 2;
    if (bin_f64(from_ord(mid), xmin, step) >= (double)k) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// ---- radix sort driver ----------------------------------------------------------------
// Sorts n (key, value) pairs by bits [begin_bit, end_bit) of the key. keys is overwritten.
// vals == nullptr means value = position. The sorted pairs are returned in *ko / *vo.
// n_dev != nullptr: the pair count is in device memory and n is its upper bound (no host read,
// so the sequence can be captured in a CUDA graph).
template <typename K>
cvetl_status sort_pairs(cvetl_ctx* c, const char* tag, K* keys, uint32_t* vals, uint32_t n,
                        int begin_bit, int end_bit, K** ko, uint32_t** vo, const uint32_t* n_dev = nullptr) {
  if (n == 0) {
    *ko = keys;
    *vo = vals;
    return CVETL_OK;
  }
  const int passes = (end_bit - begin_bit + rs::kBits - 1) / rs::kBits;
  std::string t(tag);
  K* k2;
  uint32_t *va, *vb, *hist, *status, *tiles;
  ENSURE((t + ".k2").c_str(), n, &k2);
  ENSURE((t + ".vb").c_str(), n, &vb);
  if (!n_dev && n <= (uint32_t)c->tune.small_sort_max) {  // small: one block, shared memory
    if (n <= kCtaSortSmallMax)
      LAUNCH(ST_CTA_SORT, (k_cta_sort<K, kCtaSortBlockSmall><<<1, kCtaSortBlockSmall,
                                                              cta_sort_smem<K, kCtaSortBlockSmall>(), c->st>>>(
                              keys, vals, n, begin_bit, end_bit, k2, vb)));
    else
      LAUNCH(ST_CTA_SORT, (k_cta_sort<K, kCtaSortBlock><<<1, kCtaSortBlock, cta_sort_smem<K>(), c->st>>>(
                              keys, vals, n, begin_bit, end_bit, k2, vb)));
    LAUNCH_CHECK();
    *ko = k2;
    *vo = vb;
    return CVETL_OK;
  }
  if (vals) va = vals;
  else ENSURE((t + ".va").c_str(), n, &va);
  const uint32_t ntiles = (n + rs::kTile - 1) / rs::kTile;
  ENSURE("sort.hist", rs::kMaxPasses * rs::kRadix, &hist);
  ENSURE("sort.status", (size_t)ntiles * rs::kRadix, &status);
  ENSURE("sort.tiles", rs::kMaxPasses, &tiles);
  CK(cudaMemsetAsync(hist, 0, rs::kMaxPasses * rs::kRadix * 4, c->st));
  CK(cudaMemsetAsync(tiles, 0, rs::kMaxPasses * 4, c->st));
  LAUNCH(ST_SORT_HIST, (rs::k_histogram<K><<<grid_for(n, rs::kBlock, 4), rs::kBlock, 0, c->st>>>(
                           keys, n, begin_bit, passes, end_bit, hist, n_dev)));
  LAUNCH_CHECK();
  LAUNCH(ST_SORT_HIST, (rs::k_hist_scan<<<passes, rs::kBlock, 0, c->st>>>(hist)));
  LAUNCH_CHECK();
  K* kin = keys;
  K* kout = k2;
  const uint32_t* vin = vals;
  uint32_t* vout = vb;
  const size_t smem = (size_t)rs::kTile * (sizeof(K) + 4);
  for (int p = 0; p < passes; ++p) {
    CK(cudaMemsetAsync(status, 0, (size_t)ntiles * rs::kRadix * 4, c->st));
    LAUNCH(ST_SORT_PASS, (rs::k_onesweep<K><<<ntiles, rs::kBlock, smem, c->st>>>(
                             kin, vin, kout, vout, n, begin_bit + rs::kBits * p,
                             rs::digit_mask(begin_bit + rs::kBits * p, end_bit), hist + p * rs::kRadix, status, tiles + p, &c->dstate->err, n_dev)));
    LAUNCH_CHECK();
    // next pass reads what this one wrote
    K* tk = kin;
    kin = kout;
    kout = tk;
    uint32_t* nv = (vout == vb) ? va : vb;
    vin = vout;
    vout = nv;
  }
  *ko = kin;
  *vo = const_cast<uint32_t*>(vin);
  return CVETL_OK;
}

// Exclusive prefix sum of n counts (n_dev != nullptr: the count is in device memory, n its upper
// bound); *total_dev receives the sum.
cvetl_status scan_u32(cvetl_ctx* c, const uint32_t* in, uint32_t n, uint32_t* out, uint32_t* total_dev,
                      const uint32_t* n_dev = nullptr) {
  const uint32_t nb = (n + scan::kTile - 1) / scan::kTile;
  uint32_t* sums;
  ENSURE("scan.sums", nb + 1, &sums);
  if (n == 0) {
    CK(cudaMemsetAsync(total_dev, 0, 4, c->st));
    return CVETL_OK;
  }
  if (nb == 1 && !n_dev) {
    LAUNCH(ST_SCAN, (scan::k_scan_small<<<1, scan::kBlock, 0, c->st>>>(in, n, out, total_dev)));
    LAUNCH_CHECK();
    return CVETL_OK;
  }
  LAUNCH(ST_SCAN, (scan::k_tile_sums<<<nb, scan::kBlock, 0, c->st>>>(in, n, sums, n_dev)));
  LAUNCH_CHECK();
  LAUNCH(ST_SCAN, (scan::k_scan_sums<<<1, scan::kBlock, 0, c->st>>>(sums, nb, total_dev)));
  LAUNCH_CHECK();
  LAUNCH(ST_SCAN, (scan::k_apply<<<nb, scan::kBlock, 0, c->st>>>(in, n, sums, out, n_dev)));
  LAUNCH_CHECK();
  return CVETL_OK;
}

// Bits the journey-id sort must cover: up to the highest bit where the smallest and largest
// collected key differ (the keys agree above it). Reads DevState's key span.
int key_span_bits(cvetl_ctx* c) {
  unsigned long long span[2] = {0, 0};
  if (cudaMemcpy(span, &c->dstate->key_max, sizeof span, cudaMemcpyDeviceToHost) != cudaSuccess) return 64;
  const unsigned long long diff = span[0] ^ ~span[1];
  return diff ? 64 - __builtin_clzll(diff) : 1;
}

cvetl_status read_state(cvetl_ctx* c) {
  CK(cudaMemcpyAsync(c->hstate, c->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->hstate->err & kErrLookbackTimeout)
    return fail(c, CVETL_ETIMEOUT, "a radix-sort look-back wait gave up");
  if (c->hstate->err & kErrHashMissing)
    return fail(c, CVETL_ECUDA, "internal: a journey id was missing from the hash table");
  if (c->hstate->err & kErrCapacity)
    return fail(c, CVETL_ECUDA, "internal: run buffer capacity exceeded");
  return CVETL_OK;
}

uint32_t next_pow2(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return (uint32_t)(p > 0x80000000ull ? 0x80000000ull : p);
}

}  // namespace

// CSV text -> parsed columns on the device: line starts per tile, their prefix sum (each
// tile's first row; the total sizes the columns), then the tiles are parsed independently.
cvetl_status extract_csv(cvetl_ctx* c, const cvetl_input* in) {
  const size_t len = in->csv_len;
  if (len && !in->csv) return fail(c, CVETL_EINVAL, "cvetl_extract: NULL csv");
  if (len > (size_t)CVETL_MAX_RECORDS * 128) return fail(c, CVETL_EINVAL, "csv_len %zu is too large", len);
  cudaSetDevice(c->cfg.device);
  c->state = 0;
  const unsigned char* buf = (const unsigned char*)in->csv;
  if (len && (!in->on_device || ((uintptr_t)buf & 15))) {
    unsigned char* d;
    ENSURE("in.csv", len, &d);
    CK(cudaMemcpyAsync(d, in->csv, len, in->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
    buf = d;
  }
  const uint32_t n_tiles = (uint32_t)((len + kCsvTile - 1) / kCsvTile);
  uint32_t *tile_lines, *tile_row, *total;
  unsigned long long* total64;
  ENSURE("csv.tile_lines", (size_t)n_tiles, &tile_lines);
  ENSURE("csv.tile_row", (size_t)n_tiles, &tile_row);
  ENSURE("csv.lines", 1, &total);
  ENSURE("csv.lines64", 1, &total64);
  CK(cudaMemsetAsync(total64, 0, 8, c->st));
  if (n_tiles) {
    LAUNCH(ST_CSV_COUNT, (k_csv_tile_lines<<<grid_for((size_t)n_tiles * kCsvBlock, kCsvBlock), kCsvBlock, 0, c->st>>>(
                             buf, len, n_tiles, tile_lines, total64)));
    LAUNCH_CHECK();
  }
  {
    cvetl_status s = scan_u32(c, tile_lines, n_tiles, tile_row, total);
    if (s != CVETL_OK) return s;
  }
  unsigned long long lines64 = 0;
  CK(cudaMemcpyAsync(&lines64, total64, 8, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (lines64 > (unsigned long long)CVETL_MAX_RECORDS)  // (also keeps the 32-bit row offsets exact)
    return fail(c, CVETL_EINVAL, "the text holds more than %lld lines", (long long)CVETL_MAX_RECORDS);
  const uint32_t n_lines = (uint32_t)lines64;
  int64_t *jid, *ts;
  double *lat, *lon;
  float *spd, *hd;
  ENSURE("csv.jid", n_lines, &jid);
  ENSURE("csv.ts", n_lines, &ts);
  ENSURE("csv.lat", n_lines, &lat);
  ENSURE("csv.lon", n_lines, &lon);
  ENSURE("csv.spd", n_lines, &spd);
  ENSURE("csv.hd", n_lines, &hd);
  CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));
  if (n_tiles) {
    CsvOut o{jid, ts, lat, lon, spd, hd};
    LAUNCH(ST_CSV_PARSE, (k_csv_parse<<<n_tiles, kCsvBlock, 0, c->st>>>(buf, len, tile_row, o, n_lines, c->dstate)));
    LAUNCH_CHECK();
  }
  cvetl_status s = read_state(c);
  if (s != CVETL_OK) return s;
  // malformed lines are rows without a position: the extract counts them with the other
  // dropped rows
  c->n_in = (int64_t)n_lines;
  c->csv_malformed = 0;
  c->n_rows = n_lines;
  c->jid = jid;
  c->ts = ts;
  c->lat = lat;
  c->lon = lon;
  c->spd = spd;
  c->heading = hd;
  c->J = c->R = c->K = c->n_valid = 0;
  c->bt = Batch{};
  c->state = 1;
  return CVETL_OK;
}

// ---- stream mode ------------------------------------------------------------------------
// A persistent buffer that grows by copying its first `keep` elements (the per-batch scratch of
// ensure() is reallocated without copying).
template <typename T>
cvetl_status grow_keep(cvetl_ctx* c, const char* name, size_t count, size_t keep, T** out) {
  size_t bytes = count * sizeof(T);
  if (bytes < 256) bytes = 256;
  DevBuf& b = c->bufs[name];
  if (b.bytes >= bytes) {
    *out = reinterpret_cast<T*>(b.p);
    return CVETL_OK;
  }
  if (c->capturing) return fail(c, CVETL_ECUDA, "internal: buffer %s would move during a graph capture", name);
  c->buf_gen += 1;
  const size_t grow = grow_to(bytes, 4, b.bytes > 0);
  if (c->cfg.mem_budget_bytes && c->held + grow > c->cfg.mem_budget_bytes)
    return fail(c, CVETL_EFULL, "buffer %s needs %zu more bytes; the context holds %zu of a %zu budget",
                name, grow, c->held, c->cfg.mem_budget_bytes);
  void* p = nullptr;
  if (cudaMalloc(&p, grow) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CVETL_ENOMEM, "cudaMalloc(%zu) for %s failed", grow, name);
  }
  if (b.p) {
    if (keep) CK(cudaMemcpyAsync(p, b.p, keep * sizeof(T), cudaMemcpyDeviceToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    cudaFree(b.p);
    c->held -= b.bytes;
  }
  b.p = p;
  b.bytes = grow;
  c->held += grow;
  *out = reinterpret_cast<T*>(p);
  return CVETL_OK;
}

#define GROW(name, count, keep, ptr)                           \
  do {                                                         \
    cvetl_status s_ = grow_keep(c, name, (count), (keep), (ptr)); \
    if (s_ != CVETL_OK) return s_;                             \
  } while (0)

// A journey table of `cap` slots (+ the spare slot) and its state arrays, zeroed.
cvetl_status alloc_journey_table(cvetl_ctx* c, uint32_t cap, int gen, Hash* h, JState* js) {
  const size_t m = (size_t)cap + 1;
  char nm[64];
#define JBUF(field, type, ptr)                                        \
  snprintf(nm, sizeof nm, "sj%d." field, gen);                       \
  ENSURE(nm, m, ptr);                                                 \
  CK(cudaMemsetAsync(*(ptr), 0, m * sizeof(type), c->st));
  JBUF("keys", unsigned long long, &h->keys);
  CK(cudaMemsetAsync(h->keys, 0xFF, m * 8, c->st));
  JBUF("cnt", uint32_t, &h->cnt);
  JBUF("aux", uint32_t, &h->aux);
  JBUF("n", int64_t, &js->n);
  JBUF("start", int64_t, &js->start_ts);
  JBUF("end", int64_t, &js->end_ts);
  JBUF("dwell", int64_t, &js->dwell);
  JBUF("dist", double, &js->dist);
  JBUF("slat", double, &js->slat);
  JBUF("slon", double, &js->slon);
  JBUF("lts", int64_t, &js->l_ts);
  JBUF("llat", double, &js->l_lat);
  JBUF("llon", double, &js->l_lon);
  JBUF("lspd", float, &js->l_spd);
  JBUF("lkey", uint32_t, &js->l_key);
  JBUF("rcnt", uint32_t, &js->r_cnt);
  JBUF("rs", float, &js->r_s);
  JBUF("rc", float, &js->r_c);
  JBUF("rmn", float, &js->r_mn);
  JBUF("rmx", float, &js->r_mx);
#undef JBUF
  h->cap = cap;
  h->mask = cap - 1;
  return CVETL_OK;
}

cvetl_status alloc_cell_table(cvetl_ctx* c, uint32_t cap, int gen, CellHash* ch) {
  char nm[64];
  const size_t m = cap;
#define CBUF(field, type, ptr)                                        \
  snprintf(nm, sizeof nm, "sc%d." field, gen);                       \
  ENSURE(nm, m, ptr);                                                 \
  CK(cudaMemsetAsync(*(ptr), 0, m * sizeof(type), c->st));
  CBUF("keys", uint32_t, &ch->keys);
  CK(cudaMemsetAsync(ch->keys, 0xFF, m * 4, c->st));
  CBUF("count", uint32_t, &ch->count);
  CBUF("sum", double, &ch->sum);
  CBUF("mn", float, &ch->mn);
  CBUF("mx", float, &ch->mx);
#undef CBUF
  ch->cap = cap;
  ch->mask = cap - 1;
  return CVETL_OK;
}

void free_gen(cvetl_ctx* c, const char* prefix) {
  c->buf_gen += 1;
  cudaStreamSynchronize(c->st);
  for (auto it = c->bufs.begin(); it != c->bufs.end();) {
    if (it->first.rfind(prefix, 0) == 0) {
      if (it->second.p) cudaFree(it->second.p);
      c->held -= it->second.bytes;
      it = c->bufs.erase(it);
    } else {
      ++it;
    }
  }
}

uint32_t* stream_counter(cvetl_ctx* c, const char* name) {
  uint32_t* p = nullptr;
  ensure(c, name, 1, &p);
  return p;
}

// Grows the journey table (rehashing the journeys seen so far) so that it keeps a load <= 1/2
// with the journeys of up to `pending` more rows. Uses the context's device state.
cvetl_status ensure_journey_table(cvetl_ctx* c, uint64_t pending) {
  auto& ss = c->ss;
  if (ss.jh.cap == 0 || (uint64_t)(ss.n_journeys + pending) * 2 > ss.jh.cap) {
    uint32_t cap = next_pow2(2ull * ((uint64_t)ss.n_journeys + pending + 1024));
    Hash nh{};
    JState nj{};
    const int gen = ss.jgen ^ 1;
    cvetl_status s = alloc_journey_table(c, cap, gen, &nh, &nj);
    if (s != CVETL_OK) return s;
    uint32_t* nd = stream_counter(c, "sj.distinct");
    CK(cudaMemsetAsync(nd, 0, 4, c->st));
    if (ss.jh.cap) {
      CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));
      LAUNCH(ST_STREAM_TABLES, (k_journey_rehash<<<grid_for((size_t)ss.jh.cap + 1, 256), 256, 0, c->st>>>(
                                   ss.jh, ss.js, nh, nj, nd, c->dstate)));
      LAUNCH_CHECK();
      if ((s = read_state(c)) != CVETL_OK) return s;
      char pre[16];
      snprintf(pre, sizeof pre, "sj%d.", ss.jgen);
      free_gen(c, pre);
    }
    ss.jh = nh;
    ss.js = nj;
    ss.jgen = gen;
  }
  return CVETL_OK;
}

cvetl_status stream_extract(cvetl_ctx* c, const cvetl_input* in) {
  auto& ss = c->ss;
  if (ss.flushed) return fail(c, CVETL_ESTATE, "the stream was flushed; create a new context for a new stream");
  if (in->kind != CVETL_IN_COLUMNS) return fail(c, CVETL_EINVAL, "stream mode takes binary columns");
  if (c->state == 1 || c->state == 2)
    return fail(c, CVETL_ESTATE, "the previous window has not been transformed and loaded");
  if (ss.has_w_prev && in->window_end_ms < ss.window_end)
    return fail(c, CVETL_EINVAL, "windows must come in order of window_end_ms");
  const size_t n = (size_t)in->n;
  if ((uint64_t)ss.arrival + n > 0xFFFFFFFFull) return fail(c, CVETL_EINVAL, "the stream exceeds 2^32 rows");
  {  // the journey table sized for this window's rows before the device state counts them
    cvetl_status s = ensure_journey_table(c, (uint64_t)ss.n_pending + n);
    if (s != CVETL_OK) return s;
  }
  // admission: the pending store must hold what is pending plus this window
  const size_t need = (size_t)ss.n_pending + n;
  int64_t* pj;
  Rec* pr;
  char nj[32], nr[32];
  snprintf(nj, sizeof nj, "sp.jid%d", ss.side);
  snprintf(nr, sizeof nr, "sp.rec%d", ss.side);
  GROW(nj, need, ss.n_pending, &pj);
  GROW(nr, need, ss.n_pending, &pr);
  const int64_t* jid = in->jid;
  const int64_t* ts = in->ts;
  const double* lat = in->lat;
  const double* lon = in->lon;
  const float* spd = in->speed;
  if (!in->on_device && n) {
    int64_t *a, *b;
    double *x, *y;
    float* z;
    ENSURE("in.jid", n, &a);
    ENSURE("in.ts", n, &b);
    ENSURE("in.lat", n, &x);
    ENSURE("in.lon", n, &y);
    ENSURE("in.spd", n, &z);
    CK(cudaMemcpyAsync(a, in->jid, n * 8, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(b, in->ts, n * 8, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(x, in->lat, n * 8, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(y, in->lon, n * 8, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(z, in->speed, n * 4, cudaMemcpyHostToDevice, c->st));
    jid = a; ts = b; lat = x; lon = y; spd = z;
  }
  if (!in->on_device && n) {  // the host columns are copied when the call returns
    if (!c->copy_ev && cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming) != cudaSuccess)
      return fail(c, CVETL_ECUDA, "cudaEventCreate failed");
    CK(cudaEventRecord(c->copy_ev, c->st));
  }
  CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));
  if (n) {
    LAUNCH(ST_STREAM_APPEND, (k_stream_append<<<grid_for(n, 256), 256, 0, c->st>>>(
                                 jid, ts, lat, lon, spd, (uint32_t)n, ss.arrival, ss.w_prev,
                                 ss.has_w_prev ? 1 : 0, pj, pr, ss.n_pending, (uint32_t)need, c->dstate)));
    LAUNCH_CHECK();
  }
  if (!in->on_device && n) CK(cudaEventSynchronize(c->copy_ev));
  // the appended count and the drop counters stay on the device until the transform reads its
  // state: no host round trip between the window's extract and its transform
  ss.unread_append = true;
  ss.arrival += (uint32_t)n;
  ss.n_window = (uint32_t)n;
  ss.window_end = in->window_end_ms;
  c->n_in += (int64_t)n;
  c->state = 1;
  return CVETL_OK;
}

// Finalises the pending points at or below the watermark (all of them when `all`), continuing
// each journey from its state; the window's closed runs are left for stream_fold.
cvetl_status stream_finalize(cvetl_ctx* c, bool all) {
  auto& ss = c->ss;
  const int64_t wm = ss.window_end - c->cfg.lateness_ms;
  if (!ss.unread_append) {  // a flush: no extract before; the table is sized here
    cvetl_status s = ensure_journey_table(c, ss.n_pending);
    if (s != CVETL_OK) return s;
  }
  Hash& h = ss.jh;
  CK(cudaMemsetAsync(h.cnt, 0, ((size_t)h.cap + 1) * 4, c->st));
  // split the pending store: after an extract its size is on the device (np bounds it)
  const bool app = ss.unread_append;
  const uint32_t np = ss.n_pending + (app ? ss.n_window : 0u);
  int64_t *pj, *qj;
  Rec *pr, *qr, *fr;
  uint32_t* fs;
  char n1[32], n2[32];
  snprintf(n1, sizeof n1, "sp.jid%d", ss.side);
  snprintf(n2, sizeof n2, "sp.rec%d", ss.side);
  GROW(n1, np, np, &pj);
  GROW(n2, np, np, &pr);
  snprintf(n1, sizeof n1, "sp.jid%d", ss.side ^ 1);
  snprintf(n2, sizeof n2, "sp.rec%d", ss.side ^ 1);
  GROW(n1, np, 0, &qj);
  GROW(n2, np, 0, &qr);
  ENSURE("sf.rec", np, &fr);
  ENSURE("sf.slot", np, &fs);
  // journeys touched by the window, ascending id: bucket offsets
  unsigned long long* ukey;
  uint32_t* uslot;
  ENSURE("j.ukey", (size_t)np + 1, &ukey);
  ENSURE("j.uslot", (size_t)np + 1, &uslot);
  if (!app) CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));
  if (np) {
    LAUNCH(ST_STREAM_SPLIT, (k_stream_split<<<grid_for(np, 256), 256, 0, c->st>>>(
                                pj, pr, np, ss.n_pending, app ? &c->dstate->n_appended : nullptr, wm,
                                all ? 1 : 0, h, qj, qr, fr, fs, c->dstate)));
    LAUNCH_CHECK();
    const uint32_t lim = (uint32_t)std::min(c->tune.small_journey_max, kJSmallMax);
    LAUNCH(ST_COLLECT, (k_stream_touched<<<grid_for((size_t)h.cap + 1, 256), 256, 0, c->st>>>(h, ukey, uslot, c->dstate,
                                                                                              lim)));
    LAUNCH_CHECK();
  }
  cvetl_status s = read_state(c);
  if (s != CVETL_OK) return s;
  if (c->hstate->err & kErrHashOverflow) return fail(c, CVETL_ECUDA, "internal: journey table overflow");
  const uint32_t nf = c->hstate->n_final, nq = c->hstate->n_pending;
  if (app) {
    ss.tot_malformed += (int64_t)c->hstate->n_malformed;
    ss.tot_late += (int64_t)c->hstate->n_too_late;
    ss.unread_append = false;
  }
  ss.n_journeys += c->hstate->n_distinct;
  ss.side ^= 1;
  ss.n_pending = nq;
  const uint32_t J = c->hstate->n_touched, n_long = c->hstate->n_long;
  unsigned long long* skey;
  uint32_t* sslot;
  if ((s = sort_pairs<unsigned long long>(c, "jsort", ukey, uslot, J, 0, key_span_bits(c), &skey, &sslot)) != CVETL_OK)
    return s;
  uint32_t *jn, *joff, *total;
  int64_t* jid_tmp;
  ENSURE("j.n32", (size_t)J, &jn);
  ENSURE("j.off32", (size_t)J, &joff);
  ENSURE("j.total", 1, &total);
  ENSURE("j.idtmp", (size_t)J, &jid_tmp);
  if (J && J <= kOffsetsMax) {  // sizes, offsets and cursors in one block
    LAUNCH(ST_SIZES, (k_journey_offsets<<<1, kOffsetsBlock, 0, c->st>>>(sslot, J, h, jn, joff, total)));
    LAUNCH_CHECK();
  } else {
    if (J) {
      LAUNCH(ST_SIZES, (k_journey_sizes<<<(J + 255) / 256, 256, 0, c->st>>>(skey, sslot, J, h, jn, jid_tmp, 0, nullptr)));
      LAUNCH_CHECK();
    }
    if ((s = scan_u32(c, jn, J, joff, total)) != CVETL_OK) return s;
    if (J) {
      LAUNCH(ST_CURSORS, (k_journey_cursors<<<(J + 255) / 256, 256, 0, c->st>>>(sslot, J, joff, h)));
      LAUNCH_CHECK();
    }
  }
  Rec* rec;
  ENSURE("rec", nf, &rec);
  if (nf) {
    LAUNCH(ST_SCATTER, (k_stream_scatter<<<grid_for(nf, 256), 256, 0, c->st>>>(fr, fs, nf, h, rec)));
    LAUNCH_CHECK();
  }
  Elem *scrA, *scrB;
  ENSURE("scr.a", nf, &scrA);
  ENSURE("scr.b", nf, &scrB);
  JourneyOut o{};
  ENSURE("run.sortkey", (size_t)nf + ss.n_journeys, &o.run_sortkey);
  ENSURE("run.cnt", (size_t)nf + ss.n_journeys, &o.run_cnt);
  ENSURE("run.sum", (size_t)nf + ss.n_journeys, &o.run_sum);
  ENSURE("run.min", (size_t)nf + ss.n_journeys, &o.run_min);
  ENSURE("run.max", (size_t)nf + ss.n_journeys, &o.run_max);
  o.run_cap = (uint32_t)(nf + ss.n_journeys);
  c->jo = o;
  CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));
  if (J) {
    // a window's journey fragments are mostly short: each kernel shape launches only when the
    // window holds journeys of its range (n_long of the J above the 64-thread limit)
    const uint32_t split = (uint32_t)c->tune.small_journey_max;
    const bool big = !split || n_long > 0, small = split && n_long < J;
#define JRN(F, NT, SM) k_journeys<F, false, NT><<<J, NT, SM, c->st>>>(rec, jn, joff, J, scrA, scrB, c->gp, Batch{}, o, \
                                                                       c->dstate, sslot, ss.js, nullptr, nullptr, split)
    if (c->cfg.precision == CVETL_FP32) {
      if (big) LAUNCH(ST_JOURNEYS, (JRN(Fp32Form, kJBlock, kJSmem)));
      if (small) LAUNCH(ST_JOURNEYS, (JRN(Fp32Form, kJSmallBlock, kJSmallSmem)));
    } else {
      if (big) LAUNCH(ST_JOURNEYS, (JRN(Fp64Form, kJBlock, kJSmem)));
      if (small) LAUNCH(ST_JOURNEYS, (JRN(Fp64Form, kJSmallBlock, kJSmallSmem)));
    }
#undef JRN
    LAUNCH_CHECK();
  }
  if (all) {  // end of the stream: close every open run
    LAUNCH(ST_STREAM_TABLES, (k_stream_close_runs<<<grid_for((size_t)h.cap + 1, 256), 256, 0, c->st>>>(
                                 h, ss.js, o.run_sortkey, o.run_cnt, o.run_sum, o.run_min, o.run_max,
                                 o.run_cap, c->dstate)));
    LAUNCH_CHECK();
  }
  if ((s = read_state(c)) != CVETL_OK) return s;
  c->R = c->hstate->n_runs;
  ss.tot_dup += (int64_t)c->hstate->n_dup;
  ss.tot_off += (int64_t)c->hstate->n_offgrid;
  ss.tot_final += nf;
  ss.tot_runs += c->R;
  ss.w_prev = wm;
  ss.has_w_prev = true;
  return CVETL_OK;
}

// Folds the window's closed runs into the device-resident cell table.
cvetl_status stream_fold(cvetl_ctx* c) {
  auto& ss = c->ss;
  const uint32_t R = c->R;
  if ((uint64_t)(ss.n_cells + R) * 2 > ss.ch.cap) {
    const uint32_t cap = next_pow2(2ull * ((uint64_t)ss.n_cells + R + 4096));
    CellHash nc{};
    const int gen = ss.cgen ^ 1;
    cvetl_status s = alloc_cell_table(c, cap, gen, &nc);
    if (s != CVETL_OK) return s;
    uint32_t* ncount = stream_counter(c, "sc.count");
    CK(cudaMemsetAsync(ncount, 0, 4, c->st));
    if (ss.ch.cap) {
      CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));
      LAUNCH(ST_STREAM_TABLES, (k_cell_rehash<<<grid_for(ss.ch.cap, 256), 256, 0, c->st>>>(ss.ch, nc, ncount, c->dstate)));
      LAUNCH_CHECK();
      if ((s = read_state(c)) != CVETL_OK) return s;
      char pre[16];
      snprintf(pre, sizeof pre, "sc%d.", ss.cgen);
      free_gen(c, pre);
    }
    ss.ch = nc;
    ss.cgen = gen;
  }
  unsigned long long* skey;
  uint32_t* sidx;
  cvetl_status s = sort_pairs<unsigned long long>(c, "rsort", c->jo.run_sortkey, nullptr, R, 0, 64, &skey, &sidx);
  if (s != CVETL_OK) return s;
  CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));
  if (R) {  // each cell's first run found in the fold itself
    LAUNCH(ST_CELL_WRITE, (k_cell_fold<<<(R + 255) / 256, 256, 0, c->st>>>(
                              skey, sidx, R, nullptr, c->jo.run_cnt, c->jo.run_sum, c->jo.run_min,
                              c->jo.run_max, ss.ch, &c->dstate->n_cells, c->dstate)));
    LAUNCH_CHECK();
  }
  if ((s = read_state(c)) != CVETL_OK) return s;
  if (c->hstate->err & kErrHashOverflow) return fail(c, CVETL_ECUDA, "internal: cell table overflow");
  ss.n_cells += c->hstate->n_cells;
  return CVETL_OK;
}

// Builds the result tables from the device-resident journey and cell tables.
cvetl_status stream_tables(cvetl_ctx* c) {
  auto& ss = c->ss;
  // cells, ascending key
  const uint32_t K = ss.n_cells;
  unsigned long long* ck;
  uint32_t *cs, *counter;
  ENSURE("t.ckey", (size_t)K + 1, &ck);
  ENSURE("t.cslot", (size_t)K + 1, &cs);
  ENSURE("j.counter", 1, &counter);
  CK(cudaMemsetAsync(counter, 0, 4, c->st));
  if (ss.ch.cap) {
    LAUNCH(ST_STREAM_TABLES, (k_cell_collect<<<grid_for(ss.ch.cap, 256), 256, 0, c->st>>>(ss.ch, ck, cs, counter)));
    LAUNCH_CHECK();
  }
  unsigned long long* sk;
  uint32_t* sslot;
  cvetl_status s = sort_pairs<unsigned long long>(c, "csort", ck, cs, K, 0, 32, &sk, &sslot);
  if (s != CVETL_OK) return s;
  CellOut& co = c->co;
  ENSURE("out.c_key", (size_t)K, &co.key);
  ENSURE("out.c_row", (size_t)K, &co.row);
  ENSURE("out.c_col", (size_t)K, &co.col);
  ENSURE("out.c_bin", (size_t)K, &co.bin);
  ENSURE("out.c_count", (size_t)K, &co.count);
  ENSURE("out.c_sum", (size_t)K, &co.sum);
  ENSURE("out.c_mean", (size_t)K, &co.mean);
  ENSURE("out.c_min", (size_t)K, &co.min);
  ENSURE("out.c_max", (size_t)K, &co.max);
  if (K) {
    LAUNCH(ST_STREAM_TABLES, (k_cell_table_from_hash<<<(K + 255) / 256, 256, 0, c->st>>>(
                                 sk, sslot, K, ss.ch, c->cfg.n_rows, c->cfg.n_cols, co)));
    LAUNCH_CHECK();
  }
  c->K = K;
  // journeys, ascending id
  const uint32_t J = ss.n_journeys;
  unsigned long long* jk;
  uint32_t* jsl;
  ENSURE("t.jkey", (size_t)J + 1, &jk);
  ENSURE("t.jslot", (size_t)J + 1, &jsl);
  CK(cudaMemsetAsync(counter, 0, 4, c->st));
  if (ss.jh.cap) {
    LAUNCH(ST_STREAM_TABLES, (k_journey_collect<<<grid_for((size_t)ss.jh.cap + 1, 256), 256, 0, c->st>>>(
                                 ss.jh, ss.js, jk, jsl, counter)));
    LAUNCH_CHECK();
  }
  uint32_t Jn = 0;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(&Jn, counter, 4, cudaMemcpyDeviceToHost));
  unsigned long long* jsk;
  uint32_t* jss;
  if ((s = sort_pairs<unsigned long long>(c, "jtsort", jk, jsl, Jn, 0, 64, &jsk, &jss)) != CVETL_OK) return s;
  JourneyOut& o = c->jo;
  uint32_t *n32, *off32, *total;
  ENSURE("t.n32", (size_t)Jn, &n32);
  ENSURE("t.off32", (size_t)Jn, &off32);
  ENSURE("j.total", 1, &total);
  ENSURE("out.j_id", (size_t)Jn, &c->jid_sorted);
  ENSURE("out.j_n", (size_t)Jn, &o.n);
  ENSURE("out.j_off", (size_t)Jn, &o.off);
  ENSURE("out.j_start_ts", (size_t)Jn, &o.start_ts);
  ENSURE("out.j_end_ts", (size_t)Jn, &o.end_ts);
  ENSURE("out.j_duration", (size_t)Jn, &o.duration);
  ENSURE("out.j_dwell", (size_t)Jn, &o.dwell);
  ENSURE("out.j_dist", (size_t)Jn, &o.dist);
  ENSURE("out.j_slat", (size_t)Jn, &o.slat);
  ENSURE("out.j_slon", (size_t)Jn, &o.slon);
  ENSURE("out.j_elat", (size_t)Jn, &o.elat);
  ENSURE("out.j_elon", (size_t)Jn, &o.elon);
  if (Jn) {
    LAUNCH(ST_STREAM_TABLES, (k_journey_n32<<<(Jn + 255) / 256, 256, 0, c->st>>>(jss, Jn, ss.js, n32)));
    LAUNCH_CHECK();
  }
  if ((s = scan_u32(c, n32, Jn, off32, total)) != CVETL_OK) return s;
  if (Jn) {
    LAUNCH(ST_STREAM_TABLES, (k_journey_table_from_state<<<(Jn + 255) / 256, 256, 0, c->st>>>(
                                 jsk, jss, Jn, ss.js, off32, c->jid_sorted, o)));
    LAUNCH_CHECK();
  }
  c->J = Jn;
  CK(cudaStreamSynchronize(c->st));
  return CVETL_OK;
}

// The batch path after sizing (journey ids collected, J known): ids in order, bucket offsets,
// the scatter, the journey kernel, then the load stage's run sort and cell table. With exact,
// the run count is read back once and the load stage is sized by it; otherwise the load stage
// reads the run count from device memory and is sized for the worst case (one run per kept
// point), so that the whole sequence has no host read and can be captured in a CUDA graph.
cvetl_status post_sizing(cvetl_ctx* c, const Hash& h, uint32_t* row_slot, unsigned long long* ukey,
                         uint32_t* uslot, uint32_t J, bool exact) {
  const uint32_t n = (uint32_t)c->n_rows;
  ENSURE("hash.rank", (size_t)h.cap + 1, &c->slot_rank);
  c->row_slot = row_slot;
  unsigned long long* skey;
  uint32_t* sslot;
  {
    cvetl_status s = sort_pairs<unsigned long long>(c, "jsort", ukey, uslot, J, 0, c->id_bits, &skey, &sslot);
    if (s != CVETL_OK) return s;
  }
  uint32_t *jn, *joff, *total;
  ENSURE("j.n32", (size_t)J, &jn);
  ENSURE("j.off32", (size_t)J, &joff);
  ENSURE("j.total", 1, &total);
  ENSURE("out.j_id", (size_t)J, &c->jid_sorted);
  if (J) {
    LAUNCH(ST_SIZES, (k_journey_sizes<<<(J + 255) / 256, 256, 0, c->st>>>(skey, sslot, J, h, jn, c->jid_sorted,
                                                                       c->bt.n_inst ? 1 : 0, c->slot_rank)));
    LAUNCH_CHECK();
  }
  {
    cvetl_status s = scan_u32(c, jn, J, joff, total);
    if (s != CVETL_OK) return s;
  }
  if (J) {
    LAUNCH(ST_CURSORS, (k_journey_cursors<<<(J + 255) / 256, 256, 0, c->st>>>(sslot, J, joff, h)));
    LAUNCH_CHECK();
  }

  // 3. scatter kept rows into journey buckets
  const size_t nv = c->n_valid;
  Rec* rec;
  ENSURE("rec", nv, &rec);
  // columns aligned for the vector loads and in one set of columns: kScatterRows rows per thread
  const auto al = [](const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; };
  const bool groups = !c->bt.cols && al(c->ts, 32) && al(c->lat, 32) && al(c->lon, 32) && al(c->spd, 16) &&
                      al(row_slot, 16);
  if (n && groups) {
    const int NT = c->tune.scatter_block;
    const size_t ng = (size_t)n / kScatterRows > 0 ? (size_t)n / kScatterRows : 1;
#define SCATR(NT_) k_scatter_rows<NT_, kScatterRows><<<grid_for(ng, NT_, 2048 / NT_), NT_, 0, c->st>>>( \
    c->ts, c->lat, c->lon, c->spd, row_slot, n, h, rec)
    if (NT == 128) LAUNCH(ST_SCATTER, (SCATR(128)));
    else if (NT == 512) LAUNCH(ST_SCATTER, (SCATR(512)));
    else LAUNCH(ST_SCATTER, (SCATR(256)));
#undef SCATR
    LAUNCH_CHECK();
  } else if (n && c->bt.cols && c->batch_aligned && c->batch_groups) {  // a batch read in place, aligned
    const int NT = c->tune.scatter_block;
    const uint32_t G = (uint32_t)c->batch_groups;
#define SCATG(NT_) k_scatter_groups<NT_, kScatterRows><<<grid_for(G, NT_, 2048 / NT_), NT_, 0, c->st>>>( \
    row_slot, n, G, c->bt, h, rec)
    if (NT == 128) LAUNCH(ST_SCATTER, (SCATG(128)));
    else if (NT == 512) LAUNCH(ST_SCATTER, (SCATG(512)));
    else LAUNCH(ST_SCATTER, (SCATG(256)));
#undef SCATG
    LAUNCH_CHECK();
  } else if (n) {
    const int U = c->tune.row_unroll, NT = c->tune.row_block;
#define SCAT(U_, NT_) k_scatter<U_, NT_><<<grid_for((n + U_ - 1) / U_, NT_, 2048 / NT_), NT_, 0, c->st>>>( \
    c->ts, c->lat, c->lon, c->spd, row_slot, n, h, c->bt, rec)
#define SCAT_NT(U_)                                                    \
    if (NT == 128) LAUNCH(ST_SCATTER, (SCAT(U_, 128)));                \
    else if (NT == 512) LAUNCH(ST_SCATTER, (SCAT(U_, 512)));           \
    else LAUNCH(ST_SCATTER, (SCAT(U_, 256)));
    if (U == 2) { SCAT_NT(2) }
    else if (U == 8) { SCAT_NT(8) }
    else { SCAT_NT(4) }
#undef SCAT_NT
#undef SCAT
    LAUNCH_CHECK();
  }

  // 4. per-journey order (bucket positions by (timestamp, row)), then the walk: kinematics,
  // keys, journey table, cell runs
  Elem *scrA, *scrB;
  ENSURE("scr.a", nv, &scrA);
  ENSURE("scr.b", nv, &scrB);
  uint16_t* spos;  // each journey's bucket positions in (timestamp, row) order (journeys up to 8192 points)
  ENSURE("rec.order", nv, &spos);
  JourneyOut& o = c->jo;
  ENSURE("out.j_n", (size_t)J, &o.n);
  ENSURE("out.j_off", (size_t)J, &o.off);
  ENSURE("out.j_start_ts", (size_t)J, &o.start_ts);
  ENSURE("out.j_end_ts", (size_t)J, &o.end_ts);
  ENSURE("out.j_duration", (size_t)J, &o.duration);
  ENSURE("out.j_dwell", (size_t)J, &o.dwell);
  ENSURE("out.j_dist", (size_t)J, &o.dist);
  ENSURE("out.j_slat", (size_t)J, &o.slat);
  ENSURE("out.j_slon", (size_t)J, &o.slon);
  ENSURE("out.j_elat", (size_t)J, &o.elat);
  ENSURE("out.j_elon", (size_t)J, &o.elon);
  if (c->cfg.materialize_points) {
    ENSURE("out.p_perm", nv, &o.perm);
    ENSURE("out.p_d", nv, &o.d);
    ENSURE("out.p_vhat", nv, &o.vhat);
    ENSURE("out.p_accel", nv, &o.accel);
    ENSURE("out.p_dwell", nv, &o.dwell_pt);
    ENSURE("out.p_key", nv, &o.key);
    ENSURE("out.p_flags", nv, &o.flags);
    ENSURE("out.p_stop_ms", nv, &o.stop_ms);
    ENSURE("out.p_accel_v", nv, &o.accel_v);
  } else {
    o.perm = nullptr;
    o.d = nullptr;
    o.vhat = o.accel = nullptr;
    o.dwell_pt = nullptr;
    o.key = nullptr;
    o.flags = nullptr;
    o.stop_ms = nullptr;
    o.accel_v = nullptr;
  }
  ENSURE("run.sortkey", nv, &o.run_sortkey);
  ENSURE("run.cnt", nv, &o.run_cnt);
  ENSURE("run.sum", nv, &o.run_sum);
  ENSURE("run.min", nv, &o.run_min);
  ENSURE("run.max", nv, &o.run_max);
  o.run_cap = (uint32_t)nv;
  // work list, longest journey first, for the sort and the walk
  unsigned long long *szkey, *szsorted;
  uint32_t *order = nullptr, *work;
  ENSURE("j.szkey", (size_t)J, &szkey);
  ENSURE("j.work", 2, &work);
  CK(cudaMemsetAsync(work, 0, 8, c->st));
  if (J) {
    LAUNCH(ST_SIZES, (k_size_keys<<<(J + 255) / 256, 256, 0, c->st>>>(jn, J, szkey)));
    LAUNCH_CHECK();
    cvetl_status s = sort_pairs<unsigned long long>(c, "osort", szkey, nullptr, J, 0, 32, &szsorted, &order);
    if (s != CVETL_OK) return s;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool f32 = c->cfg.precision == CVETL_FP32;
    // Journeys above 8192 points (the list's first) take the fused journey kernel (sort and walk
    // in one CTA; their sort goes through global scratch either way); the others are ordered by
    // size class (each class a persistent grid over its part of the list), and the walk reads
    // their bucketed records through the ordered positions.
    uint32_t *bounds, *cwork;
    ENSURE("j.bounds", 5, &bounds);
    ENSURE("j.cwork", 4, &cwork);
    LAUNCH(ST_JOURNEY_SORT, (k_size_classes<<<1, 96, 0, c->st>>>(jn, order, J, bounds, cwork)));
    LAUNCH_CHECK();
    static const int occ[4] = {
        0, occupancy(k_journey_sort_class<kSortBlockB, 8192>, kSortBlockB, kSortSmemB),
        occupancy(k_journey_sort_class<kSortBlockC, 4096>, kSortBlockC, kSortSmemC),
        occupancy(k_journey_sort_class<kJSmallBlock, 512>, kJSmallBlock, kSortSmemD)};
    static const int occ_f32 = occupancy(k_journeys<Fp32Form, true, kJBlock>, kJBlock, kJSmem);
    static const int occ_f64 = occupancy(k_journeys<Fp64Form, true, kJBlock>, kJBlock, kJSmem);
#define FUSED(F, OCC) k_journeys<F, true, kJBlock><<<(uint32_t)(sms * OCC), kJBlock, kJSmem, c->st>>>( \
    rec, jn, joff, J, scrA, scrB, c->gp, c->bt, o, c->dstate, nullptr, JState{}, order, cwork, 0u, bounds + 1)
    if (f32) LAUNCH(ST_JOURNEYS, (FUSED(Fp32Form, occ_f32)));
    else LAUNCH(ST_JOURNEYS, (FUSED(Fp64Form, occ_f64)));
#undef FUSED
#define JCLS(NT, CAP, SM, K) k_journey_sort_class<NT, CAP><<<(uint32_t)(sms * occ[K]), NT, SM, c->st>>>( \
    rec, jn, joff, order, bounds, K, cwork + K, scrA, scrB, spos, c->dstate)
    LAUNCH(ST_JOURNEY_SORT, (JCLS(kSortBlockB, 8192, kSortSmemB, 1)));
    LAUNCH(ST_JOURNEY_SORT, (JCLS(kSortBlockC, 4096, kSortSmemC, 2)));
    LAUNCH(ST_JOURNEY_SORT, (JCLS(kJSmallBlock, 512, kSortSmemD, 3)));
#undef JCLS
    LAUNCH_CHECK();
    // the walk: a persistent grid of warps taking the rest of the list longest first
    // (the grid's threshold tables in shared memory when they fit)
    const size_t wsm = walk_thr_shared(c->gp.n_rows, c->gp.n_cols, c->bt.n_inst)
                           ? (size_t)(c->gp.n_rows + c->gp.n_cols + 2) * sizeof(unsigned long long)
                           : 0;
    static const int occ32 = occupancy(k_journey_walk<Fp32Form>, kWalkBlock, kWalkThrMax * 8);
    static const int occ64 = occupancy(k_journey_walk<Fp64Form>, kWalkBlock, kWalkThrMax * 8);
    if (f32) LAUNCH(ST_JOURNEY_WALK, (k_journey_walk<Fp32Form><<<(uint32_t)(sms * occ32), kWalkBlock, wsm, c->st>>>(
                                        rec, spos, jn, joff, J, c->gp, c->bt, o, c->dstate, order, work + 1, bounds + 1)));
    else LAUNCH(ST_JOURNEY_WALK, (k_journey_walk<Fp64Form><<<(uint32_t)(sms * occ64), kWalkBlock, wsm, c->st>>>(
                                     rec, spos, jn, joff, J, c->gp, c->bt, o, c->dstate, order, work + 1, bounds + 1)));
    LAUNCH_CHECK();
    if (o.perm) {  // features over earlier points of a journey (materialised points)
      LAUNCH(ST_POINT_EXTRAS, (k_point_extras<<<grid_for((size_t)J * 32, 256), 256, 0, c->st>>>(
                              jn, joff, J, c->ts, c->bt, o.perm, o.d, o.dwell_pt, o.flags, o.stop_ms, o.accel_v)));
      LAUNCH_CHECK();
    }
  }

  // load: runs ordered by (key, first sorted position), folded into the cell table
  uint32_t R = (uint32_t)c->n_valid;
  const uint32_t* Rd = &c->dstate->n_runs;
  if (exact) {
    cvetl_status s = read_state(c);
    if (s != CVETL_OK) return s;
    R = c->hstate->n_runs;
    Rd = nullptr;
  }
  unsigned long long* rkey;
  uint32_t* sidx;
  cvetl_status s = sort_pairs<unsigned long long>(c, "rsort", c->jo.run_sortkey, nullptr, R, 0, 64, &rkey, &sidx, Rd);
  if (s != CVETL_OK) return s;
  uint32_t *head, *cidx, *ctotal;
  ENSURE("cell.head", (size_t)R, &head);
  ENSURE("cell.idx", (size_t)R, &cidx);
  ENSURE("cell.total", 1, &ctotal);
  if (R) {
    LAUNCH(ST_CELL_HEADS, (k_cell_heads<<<grid_for(R, 256), 256, 0, c->st>>>(rkey, R, head, Rd)));
    LAUNCH_CHECK();
  }
  if ((s = scan_u32(c, head, R, cidx, ctotal, Rd)) != CVETL_OK) return s;
  CellOut& co = c->co;
  ENSURE("out.c_key", (size_t)R, &co.key);
  ENSURE("out.c_row", (size_t)R, &co.row);
  ENSURE("out.c_col", (size_t)R, &co.col);
  ENSURE("out.c_bin", (size_t)R, &co.bin);
  ENSURE("out.c_count", (size_t)R, &co.count);
  ENSURE("out.c_sum", (size_t)R, &co.sum);
  ENSURE("out.c_mean", (size_t)R, &co.mean);
  ENSURE("out.c_min", (size_t)R, &co.min);
  ENSURE("out.c_max", (size_t)R, &co.max);
  ENSURE("out.c_volume", (size_t)R, &co.volume);
  if (R) {
    LAUNCH(ST_CELL_WRITE, (k_cell_write<<<grid_for(R, 256), 256, 0, c->st>>>(
                              rkey, sidx, R, head, cidx, c->jo.run_cnt, c->jo.run_sum,
                              c->jo.run_min, c->jo.run_max, c->cfg.n_rows, c->cfg.n_cols, c->bt, co, Rd,
                              joff, J)));
    LAUNCH_CHECK();
  }
  if (c->bt.n_inst) {
    LAUNCH(ST_CELL_WRITE, (k_inst_begins<<<1, 32, 0, c->st>>>(skey, J, rkey, R, Rd, cidx, ctotal, c->bt,
                                                               c->inst_counts)));
    LAUNCH_CHECK();
  }
  c->cell_total = ctotal;
  return CVETL_OK;
}

// post_sizing as a CUDA graph, one per shape (rows, journeys, kept rows, hash table, buffer
// generation, input columns, batch table, precision, point columns, launch shapes). The first
// run of a shape executes eagerly (allocating what it needs) and is then captured; later runs of
// the shape launch the graph. A capture that fails leaves that shape eager.
cvetl_status run_graph(cvetl_ctx* c, const Hash& h, uint32_t* row_slot, unsigned long long* ukey,
                       uint32_t* uslot, uint32_t J) {
  cvetl_ctx::GraphKey k;
  memset(&k, 0, sizeof k);
  k.n = (uint64_t)c->n_rows;
  k.J = J;
  k.nv = c->n_valid;
  k.cap = h.cap;
  k.gen = c->buf_gen;
  k.cols[0] = c->jid;
  k.cols[1] = c->ts;
  k.cols[2] = c->lat;
  k.cols[3] = c->lon;
  k.cols[4] = c->spd;
  k.inst = c->bt.inst;
  k.n_inst = c->bt.n_inst;
  k.precision = c->cfg.precision;
  k.materialize = c->cfg.materialize_points;
  k.t0 = c->tune.journey_ctas;
  k.t1 = (c->tune.row_unroll * 1024 + c->tune.row_block) * 1024 + c->tune.scatter_block;
  k.t2 = c->tune.small_sort_max * 1024 + c->tune.small_journey_max;
  k.id_bits = c->id_bits;
  k.aligned = c->bt.cols && c->batch_aligned ? 1 : 0;
  for (auto& g : c->graphs) {
    if (!(g.key == k)) continue;
    if (!g.exec) return post_sizing(c, h, row_slot, ukey, uslot, J, false);
    CK(cudaGraphLaunch(g.exec, c->st));
    c->graph_replays += 1;
    for (int i = 0; i < ST_COUNT; ++i) {
      c->launches[i] += g.launches[i];
      c->total_launches += g.launches[i];
    }
    return CVETL_OK;
  }
  cvetl_status s = post_sizing(c, h, row_slot, ukey, uslot, J, false);
  if (s != CVETL_OK) return s;
  k.gen = c->buf_gen;  // the buffers as they stand after the eager run
  cvetl_ctx::GraphEntry e;
  e.key = k;
  e.exec = nullptr;
  memset(c->cap_launches, 0, sizeof c->cap_launches);
  cudaGraph_t graph = nullptr;
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
  }
  cudaStream_t user = c->st;
  cudaError_t ce = cudaErrorNotReady;
  cvetl_status cs = CVETL_ECUDA;
  if (c->cap_stream) {
    // nothing executes during a capture, so the private stream needs no ordering with the user's
    c->st = c->cap_stream;
    c->capturing = true;
    ce = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      const std::string saved = c->err;
      cs = post_sizing(c, h, row_slot, ukey, uslot, J, false);
      ce = cudaStreamEndCapture(c->st, &graph);
      if (cs != CVETL_OK) c->err = saved;  // the eager results stand
    }
    c->capturing = false;
    c->st = user;
  }
  if (ce == cudaSuccess && cs == CVETL_OK && graph && cudaGraphInstantiate(&e.exec, graph, 0) != cudaSuccess)
    e.exec = nullptr;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  memcpy(e.launches, c->cap_launches, sizeof e.launches);
  if (c->graphs.size() >= 8) {
    if (c->graphs.front().exec) cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.push_back(e);
  return CVETL_OK;
}

// ======================================================================================
extern "C" {

void cvetl_config_default(cvetl_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->lat_min = 36.0;
  cfg->lon_min = -95.8;
  cfg->cell_deg = 0.01;
  cfg->n_rows = 460;
  cfg->n_cols = 670;
  cfg->n_bins = 1440;
  cfg->t0_ms = 1620518400000LL;  // 2021-05-09 00:00:00 UTC
  cfg->bin_ms = 60000;
  cfg->v_stop_kmh = 1.0f;
  cfg->earth_radius_m = 6371000.0;
  cfg->precision = CVETL_FP64;
  cfg->materialize_points = 0;
  cfg->profile = 0;
  cfg->device = 0;
  cfg->mem_budget_bytes = 0;
  cfg->stream = nullptr;
  cfg->mode = CVETL_BATCH;
  cfg->lateness_ms = 30000;
}

int32_t cvetl_version(void) { return CVETL_VERSION; }

const char* cvetl_last_error(const cvetl_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

cvetl_status cvetl_create(const cvetl_config* cfg, cvetl_ctx** out) {
  cvetl_ctx* c = nullptr;
  if (!cfg || !out) return fail(nullptr, CVETL_EINVAL, "cvetl_create: NULL argument");
  if (cfg->n_rows <= 0 || cfg->n_cols <= 0 || cfg->n_bins <= 0 || cfg->bin_ms <= 0)
    return fail(nullptr, CVETL_EINVAL, "grid and bin sizes must be positive");
  if ((uint64_t)cfg->n_rows * (uint64_t)cfg->n_cols * (uint64_t)cfg->n_bins > 0xFFFFFFFFull)
    return fail(nullptr, CVETL_EINVAL, "n_rows * n_cols * n_bins must be below 2^32");
  if (!std::isfinite(cfg->lat_min) || !std::isfinite(cfg->lon_min) || !(cfg->cell_deg > 0.0) ||
      !std::isfinite(cfg->cell_deg) || !std::isfinite(cfg->earth_radius_m))
    return fail(nullptr, CVETL_EINVAL, "lat_min, lon_min, cell_deg and earth_radius_m must be finite, cell_deg > 0");
  if (cfg->mode != CVETL_BATCH && cfg->mode != CVETL_STREAM)
    return fail(nullptr, CVETL_EINVAL, "mode must be CVETL_BATCH or CVETL_STREAM");
  if (cfg->mode == CVETL_STREAM && cfg->lateness_ms < 0)
    return fail(nullptr, CVETL_EINVAL, "lateness_ms must be >= 0");
  if (cfg->precision != CVETL_FP64 && cfg->precision != CVETL_FP32)
    return fail(nullptr, CVETL_EINVAL, "precision must be CVETL_FP64 or CVETL_FP32");
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) return fail(nullptr, CVETL_ECUDA, "cudaSetDevice(%d): %s", cfg->device, cudaGetErrorString(e));
  c = new cvetl_ctx();
  c->cfg = *cfg;
  c->st = (cudaStream_t)cfg->stream;
  auto bail = [&](cvetl_status s) {
    g_create_error = c->err;
    cvetl_destroy(c);
    return s;
  };
  // keying tables
  std::vector<unsigned long long> rt(cfg->n_rows + 1), ct(cfg->n_cols + 1);
  for (int k = 0; k <= cfg->n_rows; ++k) rt[k] = threshold(cfg->lat_min, cfg->cell_deg, k);
  for (int k = 0; k <= cfg->n_cols; ++k) ct[k] = threshold(cfg->lon_min, cfg->cell_deg, k);
  cvetl_status s;
  if ((s = ensure(c, "grid.rows", rt.size(), &c->row_thr)) != CVETL_OK) return bail(s);
  if ((s = ensure(c, "grid.cols", ct.size(), &c->col_thr)) != CVETL_OK) return bail(s);
  if ((s = ensure(c, "state", 1, &c->dstate)) != CVETL_OK) return bail(s);
  // cosine table for the binary64 haversine: {lat0 = k * 0.01, cos(lat0 deg), sin(lat0 deg) * pi/180}
  std::vector<CosEntry> cos_tab(18001);
  for (int k = -9000; k <= 9000; ++k) {
    const double lat0 = (double)k * 0.01;
    const double rad = M_PI / 180.0;
    const double c0 = std::cos(lat0 * rad), s0r = std::sin(lat0 * rad) * rad;
    cos_tab[k + 9000] = CosEntry{lat0, c0, s0r, (float)c0, (float)s0r};
  }
  CosEntry* d_cos = nullptr;
  if ((s = ensure(c, "grid.cos", cos_tab.size(), &d_cos)) != CVETL_OK) return bail(s);
  if (cudaMemcpy(d_cos, cos_tab.data(), cos_tab.size() * sizeof(CosEntry), cudaMemcpyHostToDevice) != cudaSuccess) {
    fail(c, CVETL_ECUDA, "cvetl_create: cosine table upload failed");
    return bail(CVETL_ECUDA);
  }
  c->gp.cos_tab = d_cos;
  if (cudaMemcpy(c->row_thr, rt.data(), rt.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->col_thr, ct.data(), ct.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMallocHost(&c->hstate, sizeof(DevState)) != cudaSuccess) {
    fail(c, CVETL_ECUDA, "cvetl_create: device set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
    return bail(CVETL_ECUDA);
  }
  GridParams& g = c->gp;
  g.row_thr = c->row_thr;
  g.col_thr = c->col_thr;
  g.lat_min_f = (float)cfg->lat_min;
  g.lon_min_f = (float)cfg->lon_min;
  g.inv_cell_f = (float)(1.0 / cfg->cell_deg);
  g.n_rows = cfg->n_rows;
  g.n_cols = cfg->n_cols;
  g.n_bins = cfg->n_bins;
  g.t0_ms = cfg->t0_ms;
  g.bin_ms = cfg->bin_ms;
  unsigned __int128 span = (unsigned __int128)(uint64_t)cfg->n_bins * (uint64_t)cfg->bin_ms;
  g.t_span = span > (unsigned __int128)~0ull ? ~0ull : (unsigned long long)span;
  g.bin_magic = cfg->bin_ms == 1 ? 0ull : ~0ull / (unsigned long long)cfg->bin_ms + 1ull;  // ceil(2^64 / bin_ms)
  g.v_stop = cfg->v_stop_kmh;
  g.radius_m = cfg->earth_radius_m;
  g.asin_c1 = 2.0 * cfg->earth_radius_m;
  g.asin_c2 = g.asin_c1 / 6.0;
  g.asin_c3 = g.asin_c1 * 0.075;
  g.dist_k = cfg->earth_radius_m * (3.141592653589793 / 180.0);
  g.dist_kh = (float)g.dist_k;
  g.dist_kl = (float)(g.dist_k - (double)g.dist_kh);
  if (cudaFuncSetAttribute(k_journeys<Fp64Form, false, kJBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize, kJSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_journeys<Fp32Form, false, kJBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize, kJSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_journeys<Fp64Form, true, kJBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize, kJSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_journeys<Fp32Form, true, kJBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize, kJSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_journey_sort_class<kSortBlockB, 8192>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmemB) != cudaSuccess ||
      cudaFuncSetAttribute(k_journey_sort_class<kSortBlockC, 4096>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmemC) != cudaSuccess ||
      cudaFuncSetAttribute(k_journey_sort_class<kJSmallBlock, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmemD) != cudaSuccess ||
      cudaFuncSetAttribute(rs::k_onesweep<unsigned long long>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, rs::kTile * 12) != cudaSuccess ||
      cudaFuncSetAttribute(rs::k_onesweep<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           rs::kTile * 8) != cudaSuccess ||
      cudaFuncSetAttribute(k_cta_sort<unsigned long long, kCtaSortBlock>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cta_sort_smem<unsigned long long>()) != cudaSuccess ||
      cudaFuncSetAttribute(k_cta_sort<uint32_t, kCtaSortBlock>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cta_sort_smem<uint32_t>()) != cudaSuccess) {
    fail(c, CVETL_ECUDA, "cudaFuncSetAttribute failed: %s", cudaGetErrorString(cudaGetLastError()));
    return bail(CVETL_ECUDA);
  }
  *out = c;
  return CVETL_OK;
}

cvetl_status cvetl_destroy(cvetl_ctx* c) {
  if (!c) return CVETL_OK;
  cudaSetDevice(c->cfg.device);
  cudaStreamSynchronize(c->st);
  for (auto& kv : c->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  if (c->hstate) cudaFreeHost(c->hstate);
  for (auto& p : c->pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  if (c->copy_ev) cudaEventDestroy(c->copy_ev);
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return CVETL_OK;
}

cvetl_status cvetl_extract(cvetl_ctx* c, const cvetl_input* in) {
  if (!c) return CVETL_EINVAL;
  if (!in) return fail(c, CVETL_EINVAL, "cvetl_extract: NULL input");
  if (c->cfg.mode == CVETL_STREAM) {
    if (in->n < 0 || in->n > CVETL_MAX_RECORDS)
      return fail(c, CVETL_EINVAL, "n = %lld outside [0, %lld]", (long long)in->n, (long long)CVETL_MAX_RECORDS);
    if (in->n > 0 && (!in->jid || !in->ts || !in->lat || !in->lon || !in->speed))
      return fail(c, CVETL_EINVAL, "cvetl_extract: NULL column");
    cudaSetDevice(c->cfg.device);
    return stream_extract(c, in);
  }
  if (in->kind == CVETL_IN_CSV) return extract_csv(c, in);
  if (in->kind != CVETL_IN_COLUMNS) return fail(c, CVETL_EINVAL, "unknown input kind %d", in->kind);
  if (in->n < 0 || in->n > CVETL_MAX_RECORDS)
    return fail(c, CVETL_EINVAL, "n = %lld outside [0, %lld]", (long long)in->n, (long long)CVETL_MAX_RECORDS);
  if (in->n > 0 && (!in->jid || !in->ts || !in->lat || !in->lon || !in->speed))
    return fail(c, CVETL_EINVAL, "cvetl_extract: NULL column");
  cudaSetDevice(c->cfg.device);
  c->state = 0;
  const size_t n = (size_t)in->n;
  if (in->on_device) {
    c->jid = in->jid;
    c->ts = in->ts;
    c->lat = in->lat;
    c->lon = in->lon;
    c->spd = in->speed;
  } else {
    int64_t *jid, *ts;
    double *lat, *lon;
    float* spd;
    ENSURE("in.jid", n, &jid);
    ENSURE("in.ts", n, &ts);
    ENSURE("in.lat", n, &lat);
    ENSURE("in.lon", n, &lon);
    ENSURE("in.spd", n, &spd);
    if (n) {
      CK(cudaMemcpyAsync(jid, in->jid, n * 8, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(ts, in->ts, n * 8, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(lat, in->lat, n * 8, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(lon, in->lon, n * 8, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(spd, in->speed, n * 4, cudaMemcpyHostToDevice, c->st));
    }
    c->jid = jid;
    c->ts = ts;
    c->lat = lat;
    c->lon = lon;
    c->spd = spd;
  }
  const float* heading = in->heading;
  if (heading && !in->on_device) {
    float* hd;
    ENSURE("in.heading", n, &hd);
    if (n) CK(cudaMemcpyAsync(hd, in->heading, n * 4, cudaMemcpyHostToDevice, c->st));
    heading = hd;
  }
  c->n_in = in->n;
  c->n_rows = in->n;
  c->csv_malformed = 0;
  c->heading = heading;
  c->bt = Batch{};
  c->J = c->R = c->K = c->n_valid = 0;
  c->state = 1;
  return CVETL_OK;
}

cvetl_status cvetl_extract_batch(cvetl_ctx* c, const cvetl_instance* inst, int32_t n_inst, int32_t on_device) {
  if (!c) return CVETL_EINVAL;
  if (c->cfg.mode != CVETL_BATCH) return fail(c, CVETL_EINVAL, "cvetl_extract_batch needs a batch-mode context");
  if (!inst || n_inst < 1 || n_inst > kMaxInst)
    return fail(c, CVETL_EINVAL, "a batch holds 1 to %d instances", kMaxInst);
  int64_t rows = 0;
  uint64_t keys = 0;
  for (int i = 0; i < n_inst; ++i) {
    const cvetl_instance& q = inst[i];
    if (q.n < 0) return fail(c, CVETL_EINVAL, "instance %d: negative row count", i);
    if (q.n > 0 && (!q.jid || !q.ts || !q.lat || !q.lon || !q.speed))
      return fail(c, CVETL_EINVAL, "instance %d: NULL column", i);
    if (q.n_rows <= 0 || q.n_cols <= 0 || !std::isfinite(q.lat_min) || !std::isfinite(q.lon_min))
      return fail(c, CVETL_EINVAL, "instance %d: the grid needs finite origin and positive size", i);
    rows += q.n;
    keys += (uint64_t)q.n_rows * (uint64_t)q.n_cols * (uint64_t)c->cfg.n_bins;
  }
  if (rows > CVETL_MAX_RECORDS) return fail(c, CVETL_EINVAL, "the batch holds more than %lld rows", (long long)CVETL_MAX_RECORDS);
  if (keys > 0xFFFFFFFEull) return fail(c, CVETL_EINVAL, "the instances' keys (rows x cols x bins, summed) must stay below 2^32 - 1");
  cudaSetDevice(c->cfg.device);
  c->state = 0;
  const size_t n = (size_t)rows;
  // Device instances are read in place, through a table of their column pointers (the caller
  // keeps them unchanged until cvetl_transform returns); host instances are copied into the
  // context's concatenated columns.
  const bool in_place = on_device != 0;
  int64_t *jid = nullptr, *ts = nullptr;
  double *lat = nullptr, *lon = nullptr;
  float* spd = nullptr;
  BatchCols* dcols = nullptr;
  if (in_place) {
    ENSURE("batch.cols", (size_t)kMaxInst, &dcols);
  } else {
    ENSURE("in.jid", n, &jid);
    ENSURE("in.ts", n, &ts);
    ENSURE("in.lat", n, &lat);
    ENSURE("in.lon", n, &lon);
    ENSURE("in.spd", n, &spd);
  }
  // instance table: threshold tables and offsets (kept from the last batch when the instances'
  // grids, days and sizes repeat)
  std::vector<double> key;
  key.push_back(c->cfg.cell_deg);
  for (int i = 0; i < n_inst; ++i) {
    const cvetl_instance& q = inst[i];
    key.insert(key.end(), {q.lat_min, q.lon_min, (double)q.n_rows, (double)q.n_cols, (double)q.t0_ms, (double)q.n});
  }
  const bool same_tables = key == c->batch_key && c->bt.n_inst == n_inst && c->bt.inst != nullptr;
  std::vector<BatchInst> bi(n_inst);
  size_t groups = 0;  // instance-local row groups of the scatter
  std::vector<unsigned long long> thr;
  std::vector<size_t> thr_at(n_inst);
  c->inst_rows.assign(n_inst + 1, 0);
  c->inst_keys.assign(n_inst + 1, 0);
  std::vector<BatchCols> cols(n_inst);
  const auto al = [](const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; };
  bool aligned = in_place;
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].n > 0)
      aligned = aligned && al(inst[i].jid, 32) && al(inst[i].ts, 32) && al(inst[i].lat, 32) && al(inst[i].lon, 32) &&
                al(inst[i].speed, 16);
  c->batch_aligned = aligned;
  for (int i = 0; i < n_inst; ++i) {
    const cvetl_instance& q = inst[i];
    const size_t r0 = (size_t)c->inst_rows[i], m = (size_t)q.n;
    cols[i] = BatchCols{q.jid, q.ts, q.lat, q.lon, q.speed};
    if (m && !in_place) {
      CK(cudaMemcpyAsync(jid + r0, q.jid, m * 8, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(ts + r0, q.ts, m * 8, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(lat + r0, q.lat, m * 8, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(lon + r0, q.lon, m * 8, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(spd + r0, q.speed, m * 4, cudaMemcpyHostToDevice, c->st));
    }
    c->inst_rows[i + 1] = (int64_t)(r0 + m);
    c->inst_keys[i + 1] = c->inst_keys[i] + (int64_t)q.n_rows * q.n_cols * c->cfg.n_bins;
    if (same_tables) continue;
    thr_at[i] = thr.size();
    for (int k = 0; k <= q.n_rows; ++k) thr.push_back(threshold(q.lat_min, c->cfg.cell_deg, k));
    for (int k = 0; k <= q.n_cols; ++k) thr.push_back(threshold(q.lon_min, c->cfg.cell_deg, k));
    bi[i].lat_min_f = (float)q.lat_min;
    bi[i].lon_min_f = (float)q.lon_min;
    bi[i].n_rows = q.n_rows;
    bi[i].n_cols = q.n_cols;
    bi[i].t0_ms = q.t0_ms;
    bi[i].row_begin = (uint32_t)r0;
    bi[i].key_off = (uint32_t)c->inst_keys[i];
    bi[i].group_begin = (uint32_t)groups;
    groups += (m + kScatterRows - 1) / kScatterRows;
  }
  // the column table, in stream order before the kernels that read it (pageable source:
  // staged before the call returns)
  if (in_place) CK(cudaMemcpyAsync(dcols, cols.data(), cols.size() * sizeof(BatchCols), cudaMemcpyHostToDevice, c->st));
  if (same_tables) {
    Batch keep = c->bt;
    keep.cols = dcols;
    c->jid = jid;
    c->ts = ts;
    c->lat = lat;
    c->lon = lon;
    c->spd = spd;
    c->heading = nullptr;
    c->n_in = rows;
    c->n_rows = rows;
    c->csv_malformed = 0;
    c->J = c->R = c->K = c->n_valid = 0;
    c->bt = keep;
    c->inst_cells.clear();
    c->inst_journeys.clear();
    c->state = 1;
    return CVETL_OK;
  }
  unsigned long long* dthr;
  BatchInst* dbi;
  ENSURE("batch.thr", thr.size(), &dthr);
  ENSURE("batch.inst", (size_t)n_inst, &dbi);
  ENSURE("batch.counts", 2 * kMaxInst, &c->inst_counts);
  for (int i = 0; i < n_inst; ++i) {
    bi[i].row_thr = dthr + thr_at[i];
    bi[i].col_thr = dthr + thr_at[i] + inst[i].n_rows + 1;
  }
  // the tables are pageable host memory: copy synchronously so they may go out of scope
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(dthr, thr.data(), thr.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dbi, bi.data(), bi.size() * sizeof(BatchInst), cudaMemcpyHostToDevice));
  c->bt.n_inst = n_inst;
  c->bt.inst = dbi;
  c->bt.cols = dcols;
  c->batch_groups = groups;
  c->batch_key = key;
  c->jid = jid;
  c->ts = ts;
  c->lat = lat;
  c->lon = lon;
  c->spd = spd;
  c->heading = nullptr;
  c->n_in = rows;
  c->n_rows = rows;
  c->csv_malformed = 0;
  c->J = c->R = c->K = c->n_valid = 0;
  c->inst_cells.clear();
  c->inst_journeys.clear();
  c->state = 1;
  return CVETL_OK;
}

cvetl_status cvetl_batch_ranges(cvetl_ctx* c, int64_t* row_begin, int64_t* key_begin, int64_t* cell_begin,
                                int64_t* journey_begin, int32_t n) {
  if (!c) return CVETL_EINVAL;
  if (!c->bt.n_inst || c->state < 3 || c->inst_cells.empty())
    return fail(c, CVETL_ESTATE, "cvetl_batch_ranges needs a batch that went through cvetl_load");
  if (n != c->bt.n_inst + 1) return fail(c, CVETL_EINVAL, "the ranges have n_inst + 1 = %d entries", c->bt.n_inst + 1);
  for (int i = 0; i < n; ++i) {
    if (row_begin) row_begin[i] = c->inst_rows[i];
    if (key_begin) key_begin[i] = c->inst_keys[i];
    if (cell_begin) cell_begin[i] = c->inst_cells[i];
    if (journey_begin) journey_begin[i] = c->inst_journeys[i];
  }
  return CVETL_OK;
}

cvetl_status cvetl_tuning_get(cvetl_ctx* c, cvetl_tuning* out) {
  if (!c) return CVETL_EINVAL;
  if (!out) return fail(c, CVETL_EINVAL, "cvetl_tuning_get: NULL output");
  out->journey_ctas = c->tune.journey_ctas;
  out->row_unroll = c->tune.row_unroll;
  out->row_block = c->tune.row_block;
  out->small_sort_max = c->tune.small_sort_max;
  out->small_journey_max = c->tune.small_journey_max;
  out->scatter_block = c->tune.scatter_block;
  return CVETL_OK;
}

cvetl_status cvetl_tuning_set(cvetl_ctx* c, const cvetl_tuning* t) {
  if (!c) return CVETL_EINVAL;
  if (!t) return fail(c, CVETL_EINVAL, "cvetl_tuning_set: NULL tuning");
  if (t->journey_ctas < 0 || t->journey_ctas > 3) return fail(c, CVETL_EINVAL, "journey_ctas must be in [0, 3]");
  if (t->row_unroll != 2 && t->row_unroll != 4 && t->row_unroll != 8)
    return fail(c, CVETL_EINVAL, "row_unroll must be 2, 4 or 8");
  if (t->row_block != 128 && t->row_block != 256 && t->row_block != 512)
    return fail(c, CVETL_EINVAL, "row_block must be 128, 256 or 512");
  if (t->small_sort_max < 0 || t->small_sort_max > (int32_t)kCtaSortMax)
    return fail(c, CVETL_EINVAL, "small_sort_max must be in [0, %u]", kCtaSortMax);
  if (t->small_journey_max < 0 || t->small_journey_max > kJSmallMax)
    return fail(c, CVETL_EINVAL, "small_journey_max must be in [0, %d]", kJSmallMax);
  if (t->scatter_block != 128 && t->scatter_block != 256 && t->scatter_block != 512)
    return fail(c, CVETL_EINVAL, "scatter_block must be 128, 256 or 512");
  c->tune.journey_ctas = t->journey_ctas;
  c->tune.row_unroll = t->row_unroll;
  c->tune.row_block = t->row_block;
  c->tune.small_sort_max = t->small_sort_max;
  c->tune.small_journey_max = t->small_journey_max;
  c->tune.scatter_block = t->scatter_block;
  return CVETL_OK;
}

cvetl_status cvetl_autotune(cvetl_ctx* c, int32_t reps, cvetl_tuning* out, double* ms_best) {
  if (!c) return CVETL_EINVAL;
  if (c->cfg.mode != CVETL_BATCH) return fail(c, CVETL_EINVAL, "cvetl_autotune tunes batch-mode contexts");
  if (c->state < 1) return fail(c, CVETL_ESTATE, "cvetl_autotune needs a preceding cvetl_extract");
  cudaSetDevice(c->cfg.device);
  reps = std::max(1, std::min(10, (int)reps));
  // launch statistics are restored afterwards
  CK(cudaStreamSynchronize(c->st));
  int64_t launches[ST_COUNT], total = c->total_launches;
  double ms_saved[ST_COUNT];
  memcpy(launches, c->launches, sizeof launches);
  memcpy(ms_saved, c->ms, sizeof ms_saved);
  const int profile = c->cfg.profile;
  c->cfg.profile = 0;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cvetl_status st = CVETL_OK;
  auto run_once = [&](double* ms) -> cvetl_status {
    c->state = 1;
    CK(cudaEventRecord(a, c->st));
    cvetl_status s = cvetl_transform(c);
    if (s == CVETL_OK) s = cvetl_load(c);
    if (s != CVETL_OK) return s;
    CK(cudaEventRecord(b, c->st));
    CK(cudaEventSynchronize(b));
    float f = 0.f;
    CK(cudaEventElapsedTime(&f, a, b));
    *ms = f;
    return CVETL_OK;
  };
  auto measure = [&](double* med) -> cvetl_status {
    double t;
    cvetl_status s = run_once(&t);  // untimed: first use of this shape
    if (s != CVETL_OK) return s;
    std::vector<double> v;
    for (int r = 0; r < reps; ++r) {
      if ((s = run_once(&t)) != CVETL_OK) return s;
      v.push_back(t);
    }
    std::sort(v.begin(), v.end());
    *med = v[v.size() / 2];
    return CVETL_OK;
  };
  auto best = c->tune;
  double best_ms = 0.0;
  if ((st = measure(&best_ms)) == CVETL_OK) {
    const int ctas[] = {0, 1, 2, 3}, unroll[] = {2, 4, 8}, smax[] = {0, 1024, 2048, 4096}, block[] = {128, 256, 512},
              jmax[] = {0, 128, 256, 512};
    const int* cands[] = {ctas, unroll, smax, block, jmax, block};
    const int ncand[] = {4, 3, 4, 3, 4, 3};
    for (int field = 0; field < 6 && st == CVETL_OK; ++field) {
      const int* cand = cands[field];
      const int nc = ncand[field];
      for (int k = 0; k < nc && st == CVETL_OK; ++k) {
        auto t = best;
        int& f = field == 0 ? t.journey_ctas : field == 1 ? t.row_unroll : field == 2 ? t.small_sort_max
                 : field == 3 ? t.row_block : field == 4 ? t.small_journey_max : t.scatter_block;
        if (f == cand[k]) continue;
        f = cand[k];
        c->tune = t;
        double ms = 0.0;
        if ((st = measure(&ms)) != CVETL_OK) break;
        if (ms < 0.98 * best_ms) {
          best = t;
          best_ms = ms;
        }
      }
    }
  }
  c->tune = best;
  c->state = 1;
  cudaStreamSynchronize(c->st);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->cfg.profile = profile;
  memcpy(c->launches, launches, sizeof launches);
  memcpy(c->ms, ms_saved, sizeof ms_saved);
  c->total_launches = total;
  if (st != CVETL_OK) return st;
  if (out) cvetl_tuning_get(c, out);
  if (ms_best) *ms_best = best_ms;
  return CVETL_OK;
}

void cvetl_lattice_config_default(cvetl_lattice_config* lc) {
  if (!lc) return;
  memset(lc, 0, sizeof(*lc));
  lc->bin_ms = 300000;
  lc->n_bins = 288;
  lc->direction = CVETL_DXN_CARDINAL;
  lc->dense = 1;
  lc->normalize = 0;
}

cvetl_status cvetl_lattice_build(cvetl_ctx* c, const cvetl_lattice_config* lc, cvetl_lattice* out) {
  if (!c) return CVETL_EINVAL;
  if (!lc || !out) return fail(c, CVETL_EINVAL, "cvetl_lattice_build: NULL argument");
  if (c->cfg.mode != CVETL_BATCH || c->bt.n_inst) return fail(c, CVETL_EINVAL, "the lattice is built for a single batch");
  if (c->state < 3) return fail(c, CVETL_ESTATE, "cvetl_lattice_build needs a preceding cvetl_load");
  if (!c->heading) return fail(c, CVETL_EINVAL, "the lattice needs the heading column");
  if (lc->bin_ms <= 0 || lc->n_bins <= 0 || (lc->direction != CVETL_DXN_CARDINAL && lc->direction != CVETL_DXN_QUADRANT))
    return fail(c, CVETL_EINVAL, "lattice bins must be positive and the direction a CVETL_DXN_* value");
  const uint64_t cells = (uint64_t)c->cfg.n_rows * (uint64_t)c->cfg.n_cols;
  if ((uint64_t)lc->n_bins * 4u * cells > 0xFFFFFFFFull)
    return fail(c, CVETL_EINVAL, "n_bins * 4 * n_rows * n_cols must stay below 2^32");
  cudaSetDevice(c->cfg.device);
  const uint32_t n = (uint32_t)c->n_rows, J = c->J;
  LatticeParams lp;
  lp.bin_ms = lc->bin_ms;
  lp.n_bins = lc->n_bins;
  lp.direction = lc->direction;
  lp.rank_bits = std::max(1, 64 - __builtin_clzll((unsigned long long)std::max<uint32_t>(J, 2) - 1));
  unsigned __int128 span = (unsigned __int128)(uint64_t)lc->n_bins * (uint64_t)lc->bin_ms;
  lp.t_span = span > (unsigned __int128)~0ull ? ~0ull : (unsigned long long)span;
  lp.bin_magic = lc->bin_ms == 1 ? 0ull : ~0ull / (unsigned long long)lc->bin_ms + 1ull;
  const uint64_t max_lk = (uint64_t)lc->n_bins * 4u * cells - 1;
  const int end_bit = std::min(64, (max_lk ? 64 - __builtin_clzll(max_lk) : 1) + lp.rank_bits);
  unsigned long long *keys, *ctr;
  uint32_t* vals;
  ENSURE("lat.keys", (size_t)n, &keys);
  ENSURE("lat.vals", (size_t)n, &vals);
  ENSURE("lat.ctr", 4, &ctr);
  CK(cudaMemsetAsync(ctr, 0, 32, c->st));
  if (n) {
    LAUNCH(ST_LATTICE_KEYS, (k_lattice_keys<<<grid_for(n, 256), 256, 0, c->st>>>(
                           c->row_slot, c->slot_rank, c->ts, c->lat, c->lon, c->heading, n, c->spd, c->gp, lp, keys,
                           vals, ctr)));
    LAUNCH_CHECK();
  }
  unsigned long long* skey;
  uint32_t* sspd;  // the points' speeds in lattice order
  cvetl_status s = sort_pairs<unsigned long long>(c, "lsort", keys, vals, n, 0, end_bit, &skey, &sspd);
  if (s != CVETL_OK) return s;
  unsigned long long dropped = 0;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(&dropped, ctr, 8, cudaMemcpyDeviceToHost));
  const uint32_t m = (uint32_t)((uint64_t)c->n_valid - dropped);
  // cell starts: the segment heads counted per tile, the tile counts scanned, the heads' positions
  // written in order (the keys read twice, no per-key flag or index arrays)
  const uint32_t ntl = (m + kLatTile - 1) / kLatTile;
  uint32_t *tcnt, *toff, *total, *chan;
  ENSURE("lat.tcnt", (size_t)ntl + 1, &tcnt);
  ENSURE("lat.toff", (size_t)ntl + 1, &toff);
  ENSURE("lat.total", 1, &total);
  ENSURE("lat.chan", 16, &chan);
  CK(cudaMemsetAsync(chan, 0xFF, 32, c->st));
  CK(cudaMemsetAsync(chan + 8, 0, 32, c->st));
  if (m) {
    LAUNCH(ST_LATTICE, (k_lattice_tile_heads<<<ntl, 256, 0, c->st>>>(skey, m, lp.rank_bits, tcnt)));
    LAUNCH_CHECK();
  }
  if ((s = scan_u32(c, tcnt, ntl, toff, total)) != CVETL_OK) return s;
  uint32_t* start;
  ENSURE("lat.start", (size_t)m + 1, &start);
  if (m) {
    LAUNCH(ST_LATTICE, (k_lattice_tile_starts<<<ntl, 256, 0, c->st>>>(skey, m, lp.rank_bits, toff, total, start)));
    LAUNCH_CHECK();
  }
  LatticeOut& lo = c->lattice;
  ENSURE("lat.o_key", (size_t)m, &lo.key);
  ENSURE("lat.o_bin", (size_t)m, &lo.bin);
  ENSURE("lat.o_dxn", (size_t)m, &lo.dxn);
  ENSURE("lat.o_row", (size_t)m, &lo.row);
  ENSURE("lat.o_col", (size_t)m, &lo.col);
  ENSURE("lat.o_count", (size_t)m, &lo.count);
  ENSURE("lat.o_sum", (size_t)m, &lo.sum);
  ENSURE("lat.o_mean", (size_t)m, &lo.mean);
  ENSURE("lat.o_volume", (size_t)m, &lo.volume);
  ENSURE("lat.o_mean_norm", (size_t)m, &lo.mean_norm);
  ENSURE("lat.o_volume_norm", (size_t)m, &lo.volume_norm);
  uint32_t K = 0;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(&K, total, 4, cudaMemcpyDeviceToHost));
  if (!m) K = 0;
  if (K) {
    // cells longest first, so that the lanes of a warp fold cells of about the same length
    unsigned long long *lkey, *lsorted;
    uint32_t* order;
    ENSURE("lat.lenkey", (size_t)K, &lkey);
    LAUNCH(ST_LATTICE, (k_lattice_len_keys<<<grid_for(K, 256), 256, 0, c->st>>>(start, total, lkey)));
    LAUNCH_CHECK();
    if ((s = sort_pairs<unsigned long long>(c, "lorder", lkey, nullptr, K, 32, 64, &lsorted, &order)) != CVETL_OK)
      return s;
    LAUNCH(ST_LATTICE_FOLD, (k_lattice_fold<<<grid_for(K, 256), 256, 0, c->st>>>(
                           skey, sspd, start, order, total, lp.rank_bits, c->cfg.n_rows, c->cfg.n_cols, lo, chan)));
    LAUNCH_CHECK();
  }
  float* dense = nullptr;
  if (lc->dense) {
    const size_t cnt = (size_t)lc->n_bins * 8u * cells;
    ENSURE("lat.dense", cnt, &dense);
    CK(cudaMemsetAsync(dense, 0, cnt * 4, c->st));
  }
  if (K) {
    LAUNCH(ST_LATTICE, (k_lattice_norm<<<grid_for(K, 256), 256, 0, c->st>>>(K, chan, lo, c->cfg.n_rows, c->cfg.n_cols,
                                                                            dense, lc->normalize ? 1 : 0)));
    LAUNCH_CHECK();
  }
  uint32_t ch[16];
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(ch, chan, sizeof ch, cudaMemcpyDeviceToHost));
  if ((s = read_state(c)) != CVETL_OK) return s;
  memset(out, 0, sizeof(*out));
  out->n_cells = K;
  out->key = lo.key;
  out->bin = lo.bin;
  out->dxn = lo.dxn;
  out->row = lo.row;
  out->col = lo.col;
  out->count = lo.count;
  out->sum = lo.sum;
  out->mean = lo.mean;
  out->volume = lo.volume;
  out->mean_norm = lo.mean_norm;
  out->volume_norm = lo.volume_norm;
  out->n_dropped = (int64_t)dropped;
  out->dense = dense;
  out->n_bins = lc->n_bins;
  for (int k = 0; k < 8; ++k) {
    const bool seen = ch[k] != 0xFFFFFFFFu;
    auto dec = [](uint32_t u) {
      uint32_t b = (u & 0x80000000u) ? (u ^ 0x80000000u) : ~u;
      float f;
      memcpy(&f, &b, 4);
      return f;
    };
    out->ch_min[k] = seen ? dec(ch[k]) : 0.0f;
    out->ch_max[k] = seen ? dec(ch[8 + k]) : 0.0f;
  }
  return CVETL_OK;
}

cvetl_status cvetl_transform(cvetl_ctx* c) {
  if (!c) return CVETL_EINVAL;
  if (c->state != 1) return fail(c, CVETL_ESTATE, "cvetl_transform needs a preceding cvetl_extract");
  cudaSetDevice(c->cfg.device);
  if (c->cfg.mode == CVETL_STREAM) {
    cvetl_status s = stream_finalize(c, false);
    if (s != CVETL_OK) return s;
    c->state = 2;
    return CVETL_OK;
  }
  const uint32_t n = (uint32_t)c->n_rows;
  CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));

  // 1. count journeys (hash table of ids), growing the table if it overflows
  // start small (2^18 slots stay hot in L2) and grow when the ids do not fit at load <= 1/2
  uint32_t cap = next_pow2(2ull * (n > 256 ? n : 256));
  if (cap > (1u << 18)) cap = 1u << 18;
  if (c->hint_distinct)  // the last batch's journey count: skip the growth steps it needed
    cap = std::min(next_pow2(2ull * (n > 256 ? n : 256)), std::max(cap, next_pow2(2ull * c->hint_distinct + 2)));
  Hash h{};
  uint32_t* row_slot;
  ENSURE("row.slot", (size_t)n, &row_slot);
  for (;;) {
    ENSURE("hash.keys", (size_t)cap + 1, &h.keys);
    ENSURE("hash.cnt", (size_t)cap + 1, &h.cnt);
    ENSURE("hash.aux", (size_t)cap + 1, &h.aux);
    h.cap = cap;
    h.mask = cap - 1;
    CK(cudaMemsetAsync(h.keys, 0xFF, ((size_t)cap + 1) * 8, c->st));
    CK(cudaMemsetAsync(h.cnt, 0, ((size_t)cap + 1) * 4, c->st));
    CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));
    if (n) {
      const int U = c->tune.row_unroll, NT = c->tune.row_block;
#define HASH(U_, NT_) k_hash_count<U_, NT_><<<grid_for((n + U_ - 1) / U_, NT_, 2048 / NT_), NT_, 0, c->st>>>( \
    c->jid, c->lat, c->lon, c->spd, n, h, c->bt, row_slot, c->dstate)
#define HASH_NT(U_)                                                    \
      if (NT == 128) LAUNCH(ST_HASH, (HASH(U_, 128)));                 \
      else if (NT == 512) LAUNCH(ST_HASH, (HASH(U_, 512)));            \
      else LAUNCH(ST_HASH, (HASH(U_, 256)));
      if (U == 2) { HASH_NT(2) }
      else if (U == 8) { HASH_NT(8) }
      else { HASH_NT(4) }
#undef HASH_NT
#undef HASH
      LAUNCH_CHECK();
    }
    cvetl_status s = read_state(c);
    if (s != CVETL_OK) return s;
    if (c->hstate->err & kErrIdRange)
      return fail(c, CVETL_EINVAL, "a batch's journey ids must lie within [-2^57, 2^57)");
    bool overflow = (c->hstate->err & kErrHashOverflow) || (uint64_t)c->hstate->n_distinct * 2 > cap;
    if (!overflow) break;
    uint32_t limit = next_pow2(2ull * (n > 256 ? n : 256));
    if (cap >= limit) return fail(c, CVETL_ECUDA, "internal: hash table cannot hold the journey ids");
    cap = (cap * 4ull > limit) ? limit : cap * 4;
  }
  c->n_valid = (uint32_t)(n - c->hstate->n_malformed);
  c->hint_distinct = c->hstate->n_distinct;

  // 2. distinct ids in ascending order -> rank, size, bucket offset
  unsigned long long* ukey;
  uint32_t *uslot, *counter;
  ENSURE("j.ukey", (size_t)c->hstate->n_distinct + 1, &ukey);
  ENSURE("j.uslot", (size_t)c->hstate->n_distinct + 1, &uslot);
  ENSURE("j.counter", 1, &counter);
  CK(cudaMemsetAsync(counter, 0, 4, c->st));
  LAUNCH(ST_COLLECT, (k_collect_slots<<<grid_for((size_t)cap + 1, 256), 256, 0, c->st>>>(h, ukey, uslot, counter,
                                                                                        c->dstate)));
  LAUNCH_CHECK();
  uint32_t J = 0;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(&J, counter, 4, cudaMemcpyDeviceToHost));
  c->J = J;
  c->id_bits = key_span_bits(c);

  // 3. the rest of transform and load, with no host read until the end
  cvetl_status s = c->cfg.graph ? run_graph(c, h, row_slot, ukey, uslot, J)
                                : post_sizing(c, h, row_slot, ukey, uslot, J, true);
  if (s != CVETL_OK) return s;
  if ((s = read_state(c)) != CVETL_OK) return s;
  c->R = c->hstate->n_runs;
  uint32_t K = 0;
  CK(cudaMemcpy(&K, c->cell_total, 4, cudaMemcpyDeviceToHost));
  c->K = c->R ? K : 0;
  if (c->bt.n_inst) {  // first journey and cell row of each instance
    uint32_t cnt[2 * kMaxInst];
    CK(cudaMemcpy(cnt, c->inst_counts, sizeof cnt, cudaMemcpyDeviceToHost));
    const int m = c->bt.n_inst;
    c->inst_journeys.assign(m + 1, (int64_t)c->J);
    c->inst_cells.assign(m + 1, (int64_t)c->K);
    for (int i = 0; i < m; ++i) {
      c->inst_journeys[i] = cnt[i];
      c->inst_cells[i] = cnt[kMaxInst + i];
    }
  }
  c->state = 2;
  return CVETL_OK;
}

cvetl_status cvetl_load(cvetl_ctx* c) {
  if (!c) return CVETL_EINVAL;
  if (c->state != 2) return fail(c, CVETL_ESTATE, "cvetl_load needs a preceding cvetl_transform");
  cudaSetDevice(c->cfg.device);
  if (c->cfg.mode == CVETL_STREAM) {
    cvetl_status s = stream_fold(c);
    if (s != CVETL_OK) return s;
    c->state = 3;
    return CVETL_OK;
  }
  // batch mode: the load stage's kernels were queued with the transform's (one sequence with
  // a single read-back at its end); the cell table is complete here
  c->state = 3;
  return CVETL_OK;
}

cvetl_status cvetl_results(cvetl_ctx* c, cvetl_tables* r) {
  if (!c) return CVETL_EINVAL;
  if (!r) return fail(c, CVETL_EINVAL, "cvetl_results: NULL output");
  if (c->state < 1) return fail(c, CVETL_ESTATE, "cvetl_results needs a preceding cvetl_extract");
  cudaSetDevice(c->cfg.device);
  memset(r, 0, sizeof(*r));
  r->n_extracted = c->n_rows;
  r->x_jid = c->jid;
  r->x_ts = c->ts;
  r->x_lat = c->lat;
  r->x_lon = c->lon;
  r->x_speed = c->spd;
  r->x_heading = c->heading;
  r->n_in = c->n_in;
  if (c->cfg.mode == CVETL_STREAM) {  // tables of everything finalised so far
    auto& ss = c->ss;
    r->n_extracted = 0;
    r->x_jid = nullptr;
    r->x_ts = nullptr;
    r->x_lat = r->x_lon = nullptr;
    r->x_speed = r->x_heading = nullptr;
    if (c->state == 1 || c->state == 2)
      return fail(c, CVETL_ESTATE, "finish the window (transform, load) before reading results");
    cvetl_status s = stream_tables(c);
    if (s != CVETL_OK) return s;
    const CellOut& co = c->co;
    r->n_cells = c->K;
    r->cell_key = co.key; r->cell_row = co.row; r->cell_col = co.col; r->cell_bin = co.bin;
    r->cell_count = co.count; r->cell_sum = co.sum; r->cell_mean = co.mean;
    r->cell_min = co.min; r->cell_max = co.max;
    r->cell_volume = nullptr;  // unique journeys are not kept across windows
    const JourneyOut& o = c->jo;
    r->n_journeys = c->J;
    r->j_id = c->jid_sorted; r->j_n = o.n; r->j_offset = o.off; r->j_start_ts = o.start_ts;
    r->j_end_ts = o.end_ts; r->j_duration_ms = o.duration; r->j_distance_m = o.dist;
    r->j_dwell_ms = o.dwell; r->j_start_lat = o.slat; r->j_start_lon = o.slon;
    r->j_end_lat = o.elat; r->j_end_lon = o.elon;
    r->n_malformed = ss.tot_malformed;
    r->n_valid = ss.tot_final;
    r->n_out_of_grid = ss.tot_off;
    r->n_dup = ss.tot_dup;
    r->n_too_late = ss.tot_late;
    r->n_runs = ss.tot_runs;
    return CVETL_OK;
  }
  if (c->state < 3) {  // extracted only: tables come with cvetl_load
    r->n_malformed = c->csv_malformed;
    return CVETL_OK;
  }
  cvetl_status s = read_state(c);
  if (s != CVETL_OK) return s;
  const CellOut& co = c->co;
  r->n_cells = c->K;
  r->cell_key = co.key;
  r->cell_row = co.row;
  r->cell_col = co.col;
  r->cell_bin = co.bin;
  r->cell_count = co.count;
  r->cell_sum = co.sum;
  r->cell_mean = co.mean;
  r->cell_min = co.min;
  r->cell_max = co.max;
  r->cell_volume = co.volume;
  const JourneyOut& o = c->jo;
  r->n_journeys = c->J;
  r->j_id = c->jid_sorted;
  r->j_n = o.n;
  r->j_offset = o.off;
  r->j_start_ts = o.start_ts;
  r->j_end_ts = o.end_ts;
  r->j_duration_ms = o.duration;
  r->j_distance_m = o.dist;
  r->j_dwell_ms = o.dwell;
  r->j_start_lat = o.slat;
  r->j_start_lon = o.slon;
  r->j_end_lat = o.elat;
  r->j_end_lon = o.elon;
  if (c->cfg.materialize_points) {
    r->n_points = c->n_valid;
    r->p_perm = o.perm;
    r->p_d = o.d;
    r->p_vhat = o.vhat;
    r->p_accel = o.accel;
    r->p_dwell = o.dwell_pt;
    r->p_key = o.key;
    r->p_flags = o.flags;
    r->p_stop_ms = o.stop_ms;
    r->p_accel_v = o.accel_v;
  }
  r->n_malformed = c->csv_malformed + (int64_t)c->hstate->n_malformed;
  r->n_valid = c->n_valid;
  r->n_out_of_grid = (int64_t)c->hstate->n_offgrid;
  r->n_dup = (int64_t)c->hstate->n_dup;
  r->n_too_late = 0;
  r->n_runs = c->R;
  return CVETL_OK;
}

cvetl_status cvetl_flush(cvetl_ctx* c) {
  if (!c) return CVETL_EINVAL;
  if (c->cfg.mode != CVETL_STREAM) return fail(c, CVETL_ESTATE, "cvetl_flush is for stream mode");
  if (c->ss.flushed) return fail(c, CVETL_ESTATE, "the stream was already flushed");
  if (c->state == 1 || c->state == 2)
    return fail(c, CVETL_ESTATE, "finish the window (transform, load) before flushing");
  cudaSetDevice(c->cfg.device);
  cvetl_status s = stream_finalize(c, true);
  if (s != CVETL_OK) return s;
  if ((s = stream_fold(c)) != CVETL_OK) return s;
  c->ss.flushed = true;
  c->state = 3;
  return CVETL_OK;
}

cvetl_status cvetl_stats_get(cvetl_ctx* c, cvetl_stats* out) {
  if (!c) return CVETL_EINVAL;
  if (!out) return fail(c, CVETL_EINVAL, "cvetl_stats_get: NULL output");
  cudaSetDevice(c->cfg.device);
  CK(cudaStreamSynchronize(c->st));
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) c->ms[p.first] += ms;
    c->event_pool.push_back(p.second.first);
    c->event_pool.push_back(p.second.second);
  }
  c->pending.clear();
  memset(out, 0, sizeof(*out));
  out->n_stages = ST_COUNT;
  for (int i = 0; i < ST_COUNT; ++i) {
    out->name[i] = kStageNames[i];
    out->ms[i] = c->ms[i];
    out->launches[i] = c->launches[i];
  }
  out->total_launches = c->total_launches;
  out->device_bytes = (int64_t)c->held;
  out->graph_replays = c->graph_replays;
  return CVETL_OK;
}

cvetl_status cvetl_stats_reset(cvetl_ctx* c) {
  if (!c) return CVETL_EINVAL;
  cudaSetDevice(c->cfg.device);
  CK(cudaStreamSynchronize(c->st));
  for (auto& p : c->pending) {
    c->event_pool.push_back(p.second.first);
    c->event_pool.push_back(p.second.second);
  }
  c->pending.clear();
  for (int i = 0; i < ST_COUNT; ++i) {
    c->ms[i] = 0;
    c->launches[i] = 0;
  }
  c->total_launches = 0;
  return CVETL_OK;
}

cvetl_status cvetl_probe_fp64(int32_t kind, int32_t blocks, int32_t threads, int64_t iters, double* sink,
                              int64_t* ops, void* stream) {
  cvetl_ctx* c = nullptr;
  if (kind < kProbeFma || kind > kProbeMix) return fail(c, CVETL_EINVAL, "cvetl_probe_fp64: kind %d", kind);
  if (blocks < 1 || blocks > (1 << 20) || (threads != 64 && threads != 128 && threads != 256) || iters < 0)
    return fail(c, CVETL_EINVAL, "cvetl_probe_fp64: %d blocks of %d threads, %lld iterations", blocks, threads,
                (long long)iters);
  if (!sink) return fail(c, CVETL_EINVAL, "cvetl_probe_fp64: NULL sink");
  cudaStream_t st = (cudaStream_t)stream;
  const double b = 0.9999999999999, cc = 1e-9;
  switch (kind) {
    case kProbeFma: k_probe_fp64<kProbeFma><<<blocks, threads, 0, st>>>(iters, b, cc, sink); break;
    case kProbeAdd: k_probe_fp64<kProbeAdd><<<blocks, threads, 0, st>>>(iters, b, cc, sink); break;
    case kProbeMul: k_probe_fp64<kProbeMul><<<blocks, threads, 0, st>>>(iters, b, cc, sink); break;
    default: k_probe_fp64<kProbeMix><<<blocks, threads, 0, st>>>(iters, b, cc, sink); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, CVETL_ECUDA, "cvetl_probe_fp64: %s", cudaGetErrorString(e));
  if (ops) *ops = (int64_t)blocks * threads * iters * kProbeChains * probe_ops_per_iter(kind);
  return CVETL_OK;
}

}  // extern "C"

// The allocation-free sort entry point (its scratch array and set-up live in this file).
#include "noalloc_sort.cuh"
