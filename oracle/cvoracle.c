/*
 * cvoracle.c — plain, slow, single-threaded CPU oracle of the connected-vehicle ETL path.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's CPU
 * baseline, never by the product path. It shares no code with the CUDA library.
 *
 * Every step follows a plain definition, in the order the steps are listed in the header,
 * with no blocking, fusion or reordering. Citations are to the paper's sections, tables and
 * algorithms (arXiv 2305.07454). Where the paper is silent, the reading taken is stated.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC -o liboracle.so cvoracle.c -lm
 */
#include "cvoracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Extract: CSV grammar.                                                                  */
/* The paper's data are per-vehicle CSV text files (Methods, "Connected Vehicle Dataset"; */
/* Table 1). It gives no grammar or malformed-row rule; the reading used here:           */
/*   row      = 6 fields separated by ','; one trailing '\r' is stripped;                 */
/*   integer  = -?[0-9]{1,18}                (journey id, timestamp in ms)               */
/*   decimal  = -?[0-9]+(\.[0-9]+)?  with at most 15 digits in total, no exponent        */
/*   value    = double(M) / 10^k, one round-to-nearest division, M the digit string as an */
/*              integer and k the number of fraction digits (both exact in binary64)      */
/*   range    = |lat| <= 90 and |lon| <= 180                                              */
/* Any violation drops the row and counts it as malformed; an empty line is malformed.   */
/* ------------------------------------------------------------------------------------ */

static const double kPow10[16] = {1e0, 1e1, 1e2, 1e3, 1e4, 1e5, 1e6, 1e7,
                                  1e8, 1e9, 1e10, 1e11, 1e12, 1e13, 1e14, 1e15};

int orc_parse_integer(const char* s, int64_t len, int64_t* out) {
  int64_t i = 0;
  int neg = 0;
  if (i < len && s[i] == '-') { neg = 1; i++; }
  int64_t ndig = len - i;
  if (ndig < 1 || ndig > 18) return 0;
  int64_t v = 0;
  for (; i < len; i++) {
    char c = s[i];
    if (c < '0' || c > '9') return 0;
    v = v * 10 + (c - '0');
  }
  *out = neg ? -v : v;
  return 1;
}

int orc_parse_decimal(const char* s, int64_t len, double* out) {
  int64_t i = 0;
  int neg = 0;
  if (i < len && s[i] == '-') { neg = 1; i++; }
  int64_t n_int = 0, n_frac = 0;
  int64_t m = 0;
  while (i < len && s[i] >= '0' && s[i] <= '9') { m = m * 10 + (s[i] - '0'); n_int++; i++;
    if (n_int > 15) return 0; }
  if (n_int == 0) return 0;
  if (i < len) {
    if (s[i] != '.') return 0;
    i++;
    while (i < len && s[i] >= '0' && s[i] <= '9') { m = m * 10 + (s[i] - '0'); n_frac++; i++;
      if (n_int + n_frac > 15) return 0; }
    if (n_frac == 0) return 0;
    if (i != len) return 0;
  }
  double v = (double)m / kPow10[n_frac];
  *out = neg ? -v : v;
  return 1;
}

/* Parses one line (without its '\n'). Returns 1 if well formed. */
static int parse_row(const char* s, int64_t len, int64_t* jid, int64_t* ts, double* lat,
                     double* lon, float* speed, float* heading) {
  if (len > 0 && s[len - 1] == '\r') len--;
  if (len == 0) return 0;
  int64_t start[6], flen[6];
  int nf = 0;
  int64_t b = 0;
  for (int64_t i = 0; i <= len; i++) {
    if (i == len || s[i] == ',') {
      if (nf == 6) return 0; /* more than 6 fields */
      start[nf] = b;
      flen[nf] = i - b;
      nf++;
      b = i + 1;
    }
  }
  if (nf != 6) return 0;
  double la, lo, sp, hd;
  if (!orc_parse_integer(s + start[0], flen[0], jid)) return 0;
  if (!orc_parse_integer(s + start[1], flen[1], ts)) return 0;
  if (!orc_parse_decimal(s + start[2], flen[2], &la)) return 0;
  if (!orc_parse_decimal(s + start[3], flen[3], &lo)) return 0;
  if (!orc_parse_decimal(s + start[4], flen[4], &sp)) return 0;
  if (!orc_parse_decimal(s + start[5], flen[5], &hd)) return 0;
  if (!(fabs(la) <= 90.0) || !(fabs(lo) <= 180.0)) return 0;
  *lat = la;
  *lon = lo;
  *speed = (float)sp;
  *heading = (float)hd;
  return 1;
}

int64_t orc_parse_csv(const char* buf, int64_t len, int64_t cap, int64_t* jid, int64_t* ts,
                      double* lat, double* lon, float* speed, float* heading,
                      int64_t* n_lines, int64_t* n_malformed) {
  int64_t lines = 0, bad = 0;
  int64_t b = 0;
  while (b < len) {
    int64_t e = b;
    while (e < len && buf[e] != '\n') e++;
    if (lines >= cap) return -1; /* the caller's columns are too short */
    int64_t j, t;
    double la, lo;
    float sp, hd;
    if (parse_row(buf + b, e - b, &j, &t, &la, &lo, &sp, &hd)) {
      jid[lines] = j; ts[lines] = t; lat[lines] = la; lon[lines] = lo;
      speed[lines] = sp; heading[lines] = hd;
    } else {
      /* a record without a position: the extract drops it as malformed */
      jid[lines] = 0; ts[lines] = 0; lat[lines] = NAN; lon[lines] = NAN;
      speed[lines] = NAN; heading[lines] = NAN;
      bad++;
    }
    lines++;
    b = e + 1; /* skip the '\n'; a final line without '\n' ends at len */
  }
  *n_lines = lines;
  *n_malformed = bad;
  return lines;
}

/* ------------------------------------------------------------------------------------ */
/* Transform: kinematics.                                                                 */
/* ------------------------------------------------------------------------------------ */

/* Haversine great-circle distance (reading: the paper is silent on distance; the sphere */
/* of radius R, coordinates differenced in degrees first, then the asin form).          */
double orc_haversine_m(double lat1, double lon1, double lat2, double lon2, double radius_m) {
  const double rad = M_PI / 180.0;
  double dphi = (lat2 - lat1) * rad;
  double dlam = (lon2 - lon1) * rad;
  double phi1 = lat1 * rad;
  double phi2 = lat2 * rad;
  double s_phi = sin(dphi / 2.0);
  double s_lam = sin(dlam / 2.0);
  double h = s_phi * s_phi + cos(phi1) * cos(phi2) * s_lam * s_lam;
  double r = sqrt(h);
  if (r > 1.0) r = 1.0;
  return 2.0 * radius_m * asin(r);
}

/* Algorithm 2, steps 4-5: (coordinate - minimum) // step, read as floor of the IEEE     */
/* round-to-nearest quotient of the round-to-nearest difference.                         */
int32_t orc_grid_index(double x, double x_min, double step, int32_t n) {
  if (!isfinite(x)) return -1;
  double q = (x - x_min) / step;
  double f = floor(q);
  if (!(f >= 0.0) || !(f < (double)n)) return -1;
  return (int32_t)f;
}

/* Algorithm 2, step 2: time // step, read as an integer floor division of the offset   */
/* from the start of the day (ms) by the bin width (ms).                                 */
int32_t orc_time_bin(int64_t ts, int64_t t0_ms, int64_t bin_ms, int32_t n_bins) {
  __int128 a = (__int128)ts - (__int128)t0_ms;
  __int128 q = a / bin_ms;
  if ((a % bin_ms != 0) && (a < 0)) q -= 1; /* floor, bin_ms > 0 */
  if (q < 0 || q >= n_bins) return -1;
  return (int32_t)q;
}

/* ------------------------------------------------------------------------------------ */
/* Sorting helpers (single-threaded; static state is fine for this plain program).       */
/* ------------------------------------------------------------------------------------ */
static const int64_t* g_jid;
static const int64_t* g_ts;
static const uint32_t* g_key;

/* Order by (journey id, timestamp, input index): the stable sort by (journey, time). */
static int cmp_jid_ts_idx(const void* a, const void* b) {
  uint32_t i = *(const uint32_t*)a, j = *(const uint32_t*)b;
  if (g_jid[i] != g_jid[j]) return g_jid[i] < g_jid[j] ? -1 : 1;
  if (g_ts[i] != g_ts[j]) return g_ts[i] < g_ts[j] ? -1 : 1;
  return i < j ? -1 : (i > j ? 1 : 0);
}

/* Order sorted positions by (key, position): the stable sort by key. */
static int cmp_key_pos(const void* a, const void* b) {
  uint32_t i = *(const uint32_t*)a, j = *(const uint32_t*)b;
  if (g_key[i] != g_key[j]) return g_key[i] < g_key[j] ? -1 : 1;
  return i < j ? -1 : (i > j ? 1 : 0);
}

static int valid_record(double lat, double lon, float speed) {
  /* The binary path applies the CSV grammar's value rules: finite, |lat| <= 90,
   * |lon| <= 180, finite speed. */
  return isfinite(lat) && isfinite(lon) && isfinite(speed) && fabs(lat) <= 90.0 &&
         fabs(lon) <= 180.0;
}

int orc_run(const orc_params* p, int64_t n, const int64_t* jid, const int64_t* ts,
            const double* lat, const double* lon, const float* speed, orc_points* pts,
            orc_journeys* jr, orc_cells* cl, orc_counters* cnt) {
  if (!p || n < 0 || n > 0xFFFFFFFELL || !pts || !jr || !cl || !cnt) return 1;
  if (p->n_rows <= 0 || p->n_cols <= 0 || p->n_bins <= 0 || p->bin_ms <= 0) return 1;
  if ((uint64_t)p->n_rows * (uint64_t)p->n_cols * (uint64_t)p->n_bins > 0xFFFFFFFFull) return 1;
  memset(cnt, 0, sizeof(*cnt));
  cnt->n_in = n;

  /* 1. Extract (column filter, Accelerated ETL step (2)) with validation. */
  uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  float* spd = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
  if (!order || !spd) { free(order); free(spd); return 2; }
  int64_t nv = 0;
  for (int64_t i = 0; i < n; i++) {
    /* 2. Canonicalise: -0.0 speed becomes +0.0. */
    spd[i] = (speed[i] == 0.0f) ? 0.0f : speed[i];
    if (valid_record(lat[i], lon[i], speed[i])) order[nv++] = (uint32_t)i;
  }
  cnt->n_malformed = n - nv;
  cnt->n_valid = nv;

  /* 3. Sort by (journey id, timestamp); ties keep input order. */
  g_jid = jid;
  g_ts = ts;
  qsort(order, (size_t)nv, sizeof(uint32_t), cmp_jid_ts_idx);

  const double R = p->earth_radius_m;
  int64_t run_stop = 0;     /* dwell of the current run of stop steps */
  double v_prev = 0.0;      /* implied speed of the previous step, m/s */
  int v_prev_ok = 0;        /* the previous step had dt > 0 */
  for (int64_t k = 0; k < nv; k++) {
    uint32_t i = order[k];
    pts->perm[k] = i;
    uint8_t f = 0;
    double d = 0.0, vh = 0.0, ac = 0.0, av = 0.0;
    int64_t dwell = 0;
    /* 4. Journey start / step. */
    int start = (k == 0) || (jid[order[k - 1]] != jid[i]);
    if (start) {
      f |= ORC_F_START;
    } else {
      uint32_t q = order[k - 1];
      int64_t dt = (int64_t)((uint64_t)ts[i] - (uint64_t)ts[q]);
      if (dt == 0) f |= ORC_F_DUP;
      /* 5. Haversine step distance. */
      d = orc_haversine_m(lat[q], lon[q], lat[i], lon[i], R);
      if (dt > 0) {
        double dt_s = (double)dt / 1000.0;
        /* 6. Implied speed in km/h. */
        vh = d / dt_s * 3.6;
        /* 7. Acceleration from the sensor speeds, m/s^2. */
        ac = (((double)spd[i] - (double)spd[q]) / 3.6) / dt_s;
      }
      /* 8. Dwell: both endpoints below the stop speed. */
      if (spd[q] < p->v_stop_kmh && spd[i] < p->v_stop_kmh) {
        f |= ORC_F_STOP;
        dwell = dt;
      }
      /* Run-length dwell (reading): the time since the current stop began is the dwell summed
       * over the consecutive stop steps ending here. Acceleration from the implied speeds
       * (reading): the difference of this step's and the previous step's implied speed in m/s
       * over this step's dt, when both steps have dt > 0. */
      run_stop = (f & ORC_F_STOP) ? run_stop + dwell : 0;
      if (dt > 0) {
        const double dt_s = (double)dt / 1000.0;
        const double v = d / dt_s;
        if (v_prev_ok) av = (v - v_prev) / dt_s;
        v_prev = v;
        v_prev_ok = 1;
      } else {
        v_prev_ok = 0;
      }
    }
    if (start) {
      run_stop = 0;
      v_prev_ok = 0;
    }
    /* 9. Key: Algorithm 2 bins unrolled into one global index. */
    int32_t r = orc_grid_index(lat[i], p->lat_min, p->cell_deg, p->n_rows);
    int32_t c = orc_grid_index(lon[i], p->lon_min, p->cell_deg, p->n_cols);
    int32_t b = orc_time_bin(ts[i], p->t0_ms, p->bin_ms, p->n_bins);
    uint32_t key = ORC_KEY_INVALID;
    if (r >= 0 && c >= 0 && b >= 0) {
      key = (uint32_t)(((uint64_t)b * (uint64_t)p->n_rows + (uint64_t)r) * (uint64_t)p->n_cols +
                       (uint64_t)c);
    } else {
      f |= ORC_F_OFFGRID;
      cnt->n_out_of_grid++;
    }
    if (f & ORC_F_DUP) cnt->n_dup++;
    pts->d[k] = d;
    pts->vhat[k] = vh;
    pts->accel[k] = ac;
    pts->dwell[k] = dwell;
    pts->key[k] = key;
    pts->flags[k] = f;
    pts->stop_ms[k] = run_stop;
    pts->accel_v[k] = av;
  }

  /* 10. Journey summaries, in journey-id order, sequential sums in sorted order. */
  int64_t nj = 0;
  for (int64_t k = 0; k < nv; k++) {
    uint32_t i = order[k];
    if (pts->flags[k] & ORC_F_START) {
      jr->jid[nj] = jid[i];
      jr->n[nj] = 0;
      jr->start_ts[nj] = ts[i];
      jr->distance_m[nj] = 0.0;
      jr->dwell_ms[nj] = 0;
      jr->start_lat[nj] = lat[i];
      jr->start_lon[nj] = lon[i];
      nj++;
    }
    int64_t j = nj - 1;
    jr->n[j] += 1;
    jr->end_ts[j] = ts[i];
    jr->duration_ms[j] = (int64_t)((uint64_t)ts[i] - (uint64_t)jr->start_ts[j]);
    jr->distance_m[j] += pts->d[k];
    jr->dwell_ms[j] += pts->dwell[k];
    jr->end_lat[j] = lat[i];
    jr->end_lon[j] = lon[i];
  }
  cnt->n_journeys = nj;

  /* 11. Cell x bin aggregates over valid keys, in key order (groupby count / sum / mean and
   * count unique journeys, Table 3; min and max added). Sorted positions are stably ordered
   * by key, so the sum runs over each key's points in (journey, time) order. */
  uint32_t* byk = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nv > 0 ? nv : 1));
  if (!byk) { free(order); free(spd); return 2; }
  int64_t m = 0;
  for (int64_t k = 0; k < nv; k++)
    if (pts->key[k] != ORC_KEY_INVALID) byk[m++] = (uint32_t)k;
  g_key = pts->key;
  qsort(byk, (size_t)m, sizeof(uint32_t), cmp_key_pos);
  int64_t nc = 0;
  for (int64_t t = 0; t < m; t++) {
    uint32_t k = byk[t];
    uint32_t key = pts->key[k];
    float s = spd[order[k]];
    if (t == 0 || pts->key[byk[t - 1]] != key) {
      cl->key[nc] = key;
      uint32_t cells = (uint32_t)p->n_rows * (uint32_t)p->n_cols;
      cl->bin[nc] = (int32_t)(key / cells);
      cl->row[nc] = (int32_t)((key % cells) / (uint32_t)p->n_cols);
      cl->col[nc] = (int32_t)(key % (uint32_t)p->n_cols);
      cl->count[nc] = 0;
      cl->sum[nc] = 0.0;
      cl->min[nc] = s;
      cl->max[nc] = s;
      cl->volume[nc] = 0;
      nc++;
    }
    int64_t c = nc - 1;
    /* a key's points come in (journey, time) order: a new journey starts at each change */
    if (cl->count[c] == 0 || jid[order[byk[t - 1]]] != jid[order[k]]) cl->volume[c] += 1;
    cl->count[c] += 1;
    cl->sum[c] += (double)s;
    if (s < cl->min[c]) cl->min[c] = s;
    if (s > cl->max[c]) cl->max[c] = s;
  }
  for (int64_t c = 0; c < nc; c++) cl->mean[c] = cl->sum[c] / (double)cl->count[c];
  cnt->n_cells = nc;

  free(byk);
  free(order);
  free(spd);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Lattice: the paper stores each 5-minute batch as an image of 8 channels, speed and     */
/* volume in the four cardinal directions (Results, the channel images; Algorithm 2,     */
/* step 3, direction = heading // dxn_step), with volume as the count of unique journeys */
/* (Table 3, "Reduction - Count Unique (Volume)") and min-max normalised channels        */
/* (Table 3, "Normalize"; the paper names the operation without a formula: min-max per   */
/* channel over its occupied cells is the reading). Speed is the mean point speed.       */
/* ------------------------------------------------------------------------------------ */

/* Cardinal reading: a heading within 45 degrees of north is N, and so on clockwise. The   */
/* printed heading // 90 gives quadrants that are not centred on the cardinal directions; */
/* it is kept as ORC_DXN_QUADRANT.                                                        */
int32_t orc_direction(float heading, int32_t mode) {
  const double h = (double)heading;
  if (!isfinite(h)) return -1;
  double r = fmod(h + (mode == ORC_DXN_CARDINAL ? 45.0 : 0.0), 360.0);
  if (r < 0.0) r += 360.0;
  if (r >= 360.0) r = 0.0;
  return (int32_t)floor(r / 90.0);
}

static const uint32_t* g_lkey;

/* Order lattice entries (input indices) by (lattice key, journey id, input index). */
static int cmp_lkey_jid_idx(const void* a, const void* b) {
  uint32_t i = *(const uint32_t*)a, j = *(const uint32_t*)b;
  if (g_lkey[i] != g_lkey[j]) return g_lkey[i] < g_lkey[j] ? -1 : 1;
  if (g_jid[i] != g_jid[j]) return g_jid[i] < g_jid[j] ? -1 : 1;
  return i < j ? -1 : (i > j ? 1 : 0);
}

int orc_lattice(const orc_params* p, const orc_lattice_params* lp, int64_t n, const int64_t* jid,
                const int64_t* ts, const double* lat, const double* lon, const float* speed,
                const float* heading, orc_lattice_cells* out, int64_t* n_cells, int64_t* n_dropped,
                float* ch_min, float* ch_max) {
  if (!p || !lp || n < 0 || n > 0xFFFFFFFELL || !out || !n_cells || !n_dropped || !ch_min || !ch_max) return 1;
  if (lp->bin_ms <= 0 || lp->n_bins <= 0 || p->n_rows <= 0 || p->n_cols <= 0) return 1;
  if ((uint64_t)lp->n_bins * 4u * (uint64_t)p->n_rows * (uint64_t)p->n_cols > 0xFFFFFFFFull) return 1;
  uint32_t* lkey = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  uint32_t* ent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  if (!lkey || !ent) { free(lkey); free(ent); return 2; }
  int64_t m = 0, dropped = 0;
  /* 1. Key every kept row: (bin, direction, row, col) unrolled, like the cell key. */
  for (int64_t i = 0; i < n; i++) {
    if (!valid_record(lat[i], lon[i], speed[i])) continue;
    const int32_t d = orc_direction(heading[i], lp->direction);
    const int32_t b = orc_time_bin(ts[i], p->t0_ms, lp->bin_ms, lp->n_bins);
    const int32_t r = orc_grid_index(lat[i], p->lat_min, p->cell_deg, p->n_rows);
    const int32_t c = orc_grid_index(lon[i], p->lon_min, p->cell_deg, p->n_cols);
    if (d < 0 || b < 0 || r < 0 || c < 0) { dropped++; continue; }
    lkey[i] = (((uint32_t)b * 4u + (uint32_t)d) * (uint32_t)p->n_rows + (uint32_t)r) * (uint32_t)p->n_cols + (uint32_t)c;
    ent[m++] = (uint32_t)i;
  }
  /* 2. Group by key; inside a key by journey, then input order. */
  g_lkey = lkey;
  g_jid = jid;
  qsort(ent, (size_t)m, sizeof(uint32_t), cmp_lkey_jid_idx);
  /* 3. Per key: count, speed sum in that order, mean, unique journeys. */
  int64_t k = 0;
  for (int64_t a = 0; a < m;) {
    const uint32_t key = lkey[ent[a]];
    uint32_t cnt = 0, vol = 0;
    double sum = 0.0;
    int64_t e = a;
    for (; e < m && lkey[ent[e]] == key; e++) {
      const uint32_t i = ent[e];
      const float s = (speed[i] == 0.0f) ? 0.0f : speed[i];
      cnt += 1;
      sum += (double)s;
      if (e == a || jid[ent[e - 1]] != jid[i]) vol += 1;
    }
    const uint32_t cells = (uint32_t)p->n_rows * (uint32_t)p->n_cols;
    out->key[k] = key;
    out->bin[k] = (int32_t)(key / (cells * 4u));
    out->dxn[k] = (int32_t)((key / cells) % 4u);
    out->row[k] = (int32_t)((key % cells) / (uint32_t)p->n_cols);
    out->col[k] = (int32_t)(key % (uint32_t)p->n_cols);
    out->count[k] = cnt;
    out->sum[k] = sum;
    out->mean[k] = (float)(sum / (double)cnt);
    out->volume[k] = vol;
    k++;
    a = e;
  }
  /* 4. Min-max per channel (2d: mean speed, 2d + 1: volume) over the occupied cells. */
  int seen[8] = {0};
  for (int c = 0; c < 8; c++) ch_min[c] = ch_max[c] = 0.0f;
  for (int64_t q = 0; q < k; q++) {
    const int d = out->dxn[q];
    const float v[2] = {out->mean[q], (float)out->volume[q]};
    for (int t = 0; t < 2; t++) {
      const int c = 2 * d + t;
      if (!seen[c] || v[t] < ch_min[c]) ch_min[c] = v[t];
      if (!seen[c] || v[t] > ch_max[c]) ch_max[c] = v[t];
      seen[c] = 1;
    }
  }
  for (int64_t q = 0; q < k; q++) {
    const int d = out->dxn[q];
    const float mn0 = ch_min[2 * d], mx0 = ch_max[2 * d], mn1 = ch_min[2 * d + 1], mx1 = ch_max[2 * d + 1];
    out->mean_norm[q] = (mx0 > mn0) ? (out->mean[q] - mn0) / (mx0 - mn0) : 0.0f;
    out->volume_norm[q] = (mx1 > mn1) ? ((float)out->volume[q] - mn1) / (mx1 - mn1) : 0.0f;
  }
  *n_cells = k;
  *n_dropped = dropped;
  free(lkey);
  free(ent);
  return 0;
}
