// cvetl.cu — the C ABI (include/cvetl.h): context, device buffers and the launch sequence of
// the extract / transform / load kernels.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "cvetl.h"

#include "common.cuh"
#include "radix_sort.cuh"
#include "scan.cuh"
#include "extract.cuh"
#include "journey.cuh"
#include "cells.cuh"
#include "csv.cuh"

using namespace cvetl;

namespace {

enum Stage {
  ST_HASH, ST_COLLECT, ST_SORT_HIST, ST_SORT_PASS, ST_SIZES, ST_SCAN, ST_CURSORS, ST_SCATTER,
  ST_JOURNEYS, ST_CELL_HEADS, ST_CELL_WRITE, ST_CSV_COUNT, ST_CSV_PARSE, ST_COUNT
};
const char* kStageNames[ST_COUNT] = {"hash_count", "collect_slots", "radix_histogram",
                                     "radix_onesweep", "journey_sizes", "scan", "journey_cursors",
                                     "scatter", "journeys", "cell_heads", "cell_write",
                                     "csv_count", "csv_parse"};

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
  int64_t* jid_sorted = nullptr;
  // statistics
  int64_t launches[ST_COUNT] = {};
  double ms[ST_COUNT] = {};
  int64_t total_launches = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> event_pool;
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
template <typename T>
cvetl_status ensure(cvetl_ctx* c, const char* name, size_t count, T** out) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 256;
  DevBuf& b = c->bufs[name];
  if (b.bytes < bytes) {
    size_t grow = bytes + bytes / 8;
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
template <typename K>
cvetl_status sort_pairs(cvetl_ctx* c, const char* tag, K* keys, uint32_t* vals, uint32_t n,
                        int begin_bit, int end_bit, K** ko, uint32_t** vo) {
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
  if (vals) va = vals;
  else ENSURE((t + ".va").c_str(), n, &va);
  const uint32_t ntiles = (n + rs::kTile - 1) / rs::kTile;
  ENSURE("sort.hist", rs::kMaxPasses * rs::kRadix, &hist);
  ENSURE("sort.status", (size_t)ntiles * rs::kRadix, &status);
  ENSURE("sort.tiles", rs::kMaxPasses, &tiles);
  CK(cudaMemsetAsync(hist, 0, rs::kMaxPasses * rs::kRadix * 4, c->st));
  CK(cudaMemsetAsync(tiles, 0, rs::kMaxPasses * 4, c->st));
  LAUNCH(ST_SORT_HIST, (rs::k_histogram<K><<<grid_for(n, rs::kBlock, 4), rs::kBlock, 0, c->st>>>(
                           keys, n, begin_bit, passes, hist)));
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
                             hist + p * rs::kRadix, status, tiles + p, &c->dstate->err)));
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

cvetl_status scan_u32(cvetl_ctx* c, const uint32_t* in, uint32_t n, uint32_t* out, uint32_t* total_dev) {
  const uint32_t nb = (n + scan::kTile - 1) / scan::kTile;
  uint32_t* sums;
  ENSURE("scan.sums", nb + 1, &sums);
  if (n == 0) {
    CK(cudaMemsetAsync(total_dev, 0, 4, c->st));
    return CVETL_OK;
  }
  LAUNCH(ST_SCAN, (scan::k_tile_sums<<<nb, scan::kBlock, 0, c->st>>>(in, n, sums)));
  LAUNCH_CHECK();
  LAUNCH(ST_SCAN, (scan::k_scan_sums<<<1, scan::kBlock, 0, c->st>>>(sums, nb, total_dev)));
  LAUNCH_CHECK();
  LAUNCH(ST_SCAN, (scan::k_apply<<<nb, scan::kBlock, 0, c->st>>>(in, n, sums, out)));
  LAUNCH_CHECK();
  return CVETL_OK;
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

// CSV text -> parsed columns on the device (count pass sizes the columns; parse pass keeps
// file order through a decoupled look-back over tiles).
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
  unsigned long long* nl;
  ENSURE("csv.newlines", 1, &nl);
  CK(cudaMemsetAsync(nl, 0, 8, c->st));
  if (len) {
    LAUNCH(ST_CSV_COUNT, (k_csv_count<<<grid_for((len + 15) / 16, kCsvBlock), kCsvBlock, 0, c->st>>>(buf, len, nl)));
    LAUNCH_CHECK();
  }
  unsigned long long newlines = 0;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(&newlines, nl, 8, cudaMemcpyDeviceToHost));
  const size_t cap = len ? (size_t)newlines + 1 : 0;
  if (cap > (size_t)CVETL_MAX_RECORDS) return fail(c, CVETL_EINVAL, "the text holds more than %lld lines", (long long)CVETL_MAX_RECORDS);
  int64_t *jid, *ts;
  double *lat, *lon;
  float *spd, *hd;
  ENSURE("csv.jid", cap, &jid);
  ENSURE("csv.ts", cap, &ts);
  ENSURE("csv.lat", cap, &lat);
  ENSURE("csv.lon", cap, &lon);
  ENSURE("csv.spd", cap, &spd);
  ENSURE("csv.hd", cap, &hd);
  const uint32_t n_tiles = (uint32_t)((len + kCsvTile - 1) / kCsvTile);
  uint32_t *status, *tiles;
  ENSURE("csv.status", (size_t)n_tiles + 1, &status);
  ENSURE("csv.tiles", 1, &tiles);
  CK(cudaMemsetAsync(status, 0, ((size_t)n_tiles + 1) * 4, c->st));
  CK(cudaMemsetAsync(tiles, 0, 4, c->st));
  CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));
  if (n_tiles) {
    CsvOut o{jid, ts, lat, lon, spd, hd};
    LAUNCH(ST_CSV_PARSE, (k_csv_parse<<<n_tiles, kCsvBlock, 0, c->st>>>(buf, len, n_tiles, o, (uint32_t)cap,
                                                                         status, tiles, c->dstate)));
    LAUNCH_CHECK();
  }
  cvetl_status s = read_state(c);
  if (s != CVETL_OK) return s;
  c->n_in = (int64_t)c->hstate->n_lines;
  c->csv_malformed = (int64_t)c->hstate->n_malformed;
  c->n_rows = c->n_in - c->csv_malformed;
  c->jid = jid;
  c->ts = ts;
  c->lat = lat;
  c->lon = lon;
  c->spd = spd;
  c->heading = hd;
  c->J = c->R = c->K = c->n_valid = 0;
  c->state = 1;
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
    cos_tab[k + 9000] = CosEntry{lat0, std::cos(lat0 * rad), std::sin(lat0 * rad) * rad, 0.0};
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
  g.v_stop = cfg->v_stop_kmh;
  g.radius_m = cfg->earth_radius_m;
  g.asin_c1 = 2.0 * cfg->earth_radius_m;
  g.asin_c2 = g.asin_c1 / 6.0;
  g.asin_c3 = g.asin_c1 * 0.075;
  if (cudaFuncSetAttribute(k_journeys<Fp64Form>, cudaFuncAttributeMaxDynamicSharedMemorySize, kJSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_journeys<Fp32Form>, cudaFuncAttributeMaxDynamicSharedMemorySize, kJSmem) != cudaSuccess ||
      cudaFuncSetAttribute(rs::k_onesweep<unsigned long long>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, rs::kTile * 12) != cudaSuccess ||
      cudaFuncSetAttribute(rs::k_onesweep<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           rs::kTile * 8) != cudaSuccess) {
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
  delete c;
  return CVETL_OK;
}

cvetl_status cvetl_extract(cvetl_ctx* c, const cvetl_input* in) {
  if (!c) return CVETL_EINVAL;
  if (!in) return fail(c, CVETL_EINVAL, "cvetl_extract: NULL input");
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
  c->n_in = in->n;
  c->n_rows = in->n;
  c->csv_malformed = 0;
  c->heading = in->heading;
  c->J = c->R = c->K = c->n_valid = 0;
  c->state = 1;
  return CVETL_OK;
}

cvetl_status cvetl_transform(cvetl_ctx* c) {
  if (!c) return CVETL_EINVAL;
  if (c->state != 1) return fail(c, CVETL_ESTATE, "cvetl_transform needs a preceding cvetl_extract");
  cudaSetDevice(c->cfg.device);
  const uint32_t n = (uint32_t)c->n_rows;
  CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->st));

  // 1. count journeys (hash table of ids), growing the table if it overflows
  // start small (2^18 slots stay hot in L2) and grow when the ids do not fit at load <= 1/2
  uint32_t cap = next_pow2(2ull * (n > 256 ? n : 256));
  if (cap > (1u << 18)) cap = 1u << 18;
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
      LAUNCH(ST_HASH, (k_hash_count<<<grid_for((n + kUnroll - 1) / kUnroll, 256), 256, 0, c->st>>>(c->jid, c->lat, c->lon,
                                                                          c->spd, n, h, row_slot, c->dstate)));
      LAUNCH_CHECK();
    }
    cvetl_status s = read_state(c);
    if (s != CVETL_OK) return s;
    bool overflow = (c->hstate->err & kErrHashOverflow) || (uint64_t)c->hstate->n_distinct * 2 > cap;
    if (!overflow) break;
    uint32_t limit = next_pow2(2ull * (n > 256 ? n : 256));
    if (cap >= limit) return fail(c, CVETL_ECUDA, "internal: hash table cannot hold the journey ids");
    cap = (cap * 4ull > limit) ? limit : cap * 4;
  }
  c->n_valid = (uint32_t)(n - c->hstate->n_malformed);

  // 2. distinct ids in ascending order -> rank, size, bucket offset
  unsigned long long* ukey;
  uint32_t *uslot, *counter;
  ENSURE("j.ukey", (size_t)c->hstate->n_distinct + 1, &ukey);
  ENSURE("j.uslot", (size_t)c->hstate->n_distinct + 1, &uslot);
  ENSURE("j.counter", 1, &counter);
  CK(cudaMemsetAsync(counter, 0, 4, c->st));
  LAUNCH(ST_COLLECT, (k_collect_slots<<<grid_for((size_t)cap + 1, 256), 256, 0, c->st>>>(h, ukey, uslot, counter)));
  LAUNCH_CHECK();
  uint32_t J = 0;
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpy(&J, counter, 4, cudaMemcpyDeviceToHost));
  c->J = J;
  unsigned long long* skey;
  uint32_t* sslot;
  {
    cvetl_status s = sort_pairs<unsigned long long>(c, "jsort", ukey, uslot, J, 0, 64, &skey, &sslot);
    if (s != CVETL_OK) return s;
  }
  uint32_t *jn, *joff, *total;
  ENSURE("j.n32", (size_t)J, &jn);
  ENSURE("j.off32", (size_t)J, &joff);
  ENSURE("j.total", 1, &total);
  ENSURE("out.j_id", (size_t)J, &c->jid_sorted);
  if (J) {
    LAUNCH(ST_SIZES, (k_journey_sizes<<<(J + 255) / 256, 256, 0, c->st>>>(skey, sslot, J, h, jn, c->jid_sorted)));
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
  if (n) {
    LAUNCH(ST_SCATTER, (k_scatter<<<grid_for((n + kUnroll - 1) / kUnroll, 256), 256, 0, c->st>>>(
                           c->ts, c->lat, c->lon, c->spd, row_slot, n, h, rec)));
    LAUNCH_CHECK();
  }

  // 4. per-journey sort, kinematics, keys, journey table, cell runs
  Elem *scrA, *scrB;
  ENSURE("scr.a", nv, &scrA);
  ENSURE("scr.b", nv, &scrB);
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
  } else {
    o.perm = nullptr;
    o.d = nullptr;
    o.vhat = o.accel = nullptr;
    o.dwell_pt = nullptr;
    o.key = nullptr;
    o.flags = nullptr;
  }
  ENSURE("run.sortkey", nv, &o.run_sortkey);
  ENSURE("run.cnt", nv, &o.run_cnt);
  ENSURE("run.sum", nv, &o.run_sum);
  ENSURE("run.min", nv, &o.run_min);
  ENSURE("run.max", nv, &o.run_max);
  o.run_cap = (uint32_t)nv;
  if (J) {
    if (c->cfg.precision == CVETL_FP32) {
      LAUNCH(ST_JOURNEYS, (k_journeys<Fp32Form><<<J, kJBlock, kJSmem, c->st>>>(rec, jn, joff, J, scrA, scrB, c->gp, o, c->dstate)));
    } else {
      LAUNCH(ST_JOURNEYS, (k_journeys<Fp64Form><<<J, kJBlock, kJSmem, c->st>>>(rec, jn, joff, J, scrA, scrB, c->gp, o, c->dstate)));
    }
    LAUNCH_CHECK();
  }
  cvetl_status s = read_state(c);
  if (s != CVETL_OK) return s;
  c->R = c->hstate->n_runs;
  c->state = 2;
  return CVETL_OK;
}

cvetl_status cvetl_load(cvetl_ctx* c) {
  if (!c) return CVETL_EINVAL;
  if (c->state != 2) return fail(c, CVETL_ESTATE, "cvetl_load needs a preceding cvetl_transform");
  cudaSetDevice(c->cfg.device);
  const uint32_t R = c->R;
  unsigned long long* skey;
  uint32_t* sidx;
  cvetl_status s = sort_pairs<unsigned long long>(c, "rsort", c->jo.run_sortkey, nullptr, R, 0, 64, &skey, &sidx);
  if (s != CVETL_OK) return s;
  uint32_t *head, *cidx, *total;
  ENSURE("cell.head", (size_t)R, &head);
  ENSURE("cell.idx", (size_t)R, &cidx);
  ENSURE("cell.total", 1, &total);
  if (R) {
    LAUNCH(ST_CELL_HEADS, (k_cell_heads<<<(R + 255) / 256, 256, 0, c->st>>>(skey, R, head)));
    LAUNCH_CHECK();
  }
  if ((s = scan_u32(c, head, R, cidx, total)) != CVETL_OK) return s;
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
  if (R) {
    LAUNCH(ST_CELL_WRITE, (k_cell_write<<<(R + 255) / 256, 256, 0, c->st>>>(
                              skey, sidx, R, head, cidx, c->jo.run_cnt, c->jo.run_sum,
                              c->jo.run_min, c->jo.run_max, c->cfg.n_rows, c->cfg.n_cols, co)));
    LAUNCH_CHECK();
  }
  if ((s = read_state(c)) != CVETL_OK) return s;
  uint32_t K = 0;
  CK(cudaMemcpy(&K, total, 4, cudaMemcpyDeviceToHost));
  c->K = R ? K : 0;
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
  return fail(c, CVETL_ESTATE, "streaming mode is not built in this version");
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

}  // extern "C"

// The allocation-free sort entry point (its scratch array and set-up live in this file).
#include "noalloc_sort.cuh"
