/*
 * cvgen.c — seeded synthetic connected-vehicle records (see cvgen.h).
 *
 * Random numbers: splitmix64 seeds a xoshiro256** stream per (seed, journey, purpose);
 * normals by Box-Muller; lognormal and truncated Zipf lengths by inversion. Each journey
 * draws from its own streams, so the output does not depend on the thread count.
 * Record order: a keyed Feistel permutation of [0, 2^k) with cycle walking onto [0, n).
 *
 * Build: gcc -O2 -pthread -shared -fPIC -o libcvgen.so cvgen.c -lm
 */
#include "cvgen.h"

#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define DAY_MS 86400000LL

/* ---------------- random numbers ---------------- */
static inline uint64_t splitmix64(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline uint64_t mix64(uint64_t a, uint64_t b) {
  uint64_t s = a ^ (b * 0xD1B54A32D192ED03ull);
  return splitmix64(&s);
}
typedef struct { uint64_t s[4]; int has_spare; double spare; } rng_t;
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static void rng_init(rng_t* r, uint64_t seed, uint64_t stream, uint64_t purpose) {
  uint64_t sm = mix64(mix64(seed, stream), purpose);
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&sm);
  r->has_spare = 0;
}
static inline uint64_t rng_u64(rng_t* r) {
  uint64_t* s = r->s;
  uint64_t result = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl(s[3], 45);
  return result;
}
/* uniform in [0, 1) with 53 random bits */
static inline double rng_unif(rng_t* r) { return (double)(rng_u64(r) >> 11) * 0x1.0p-53; }
/* integer uniform in [lo, hi] */
static inline int64_t rng_int(rng_t* r, int64_t lo, int64_t hi) {
  return lo + (int64_t)(rng_unif(r) * (double)(hi - lo + 1));
}
static double rng_normal(rng_t* r) {
  if (r->has_spare) { r->has_spare = 0; return r->spare; }
  double u1 = rng_unif(r), u2 = rng_unif(r);
  if (u1 < 1e-300) u1 = 1e-300;
  double m = sqrt(-2.0 * log(u1));
  r->spare = m * sin(2.0 * M_PI * u2);
  r->has_spare = 1;
  return m * cos(2.0 * M_PI * u2);
}

/* ---------------- keyed permutation ---------------- */
typedef struct { int half; uint64_t mask; uint64_t key[4]; } feistel_t;
static void feistel_init(feistel_t* f, int bits, uint64_t seed, uint64_t purpose) {
  if (bits < 2) bits = 2;
  if (bits & 1) bits++;
  f->half = bits / 2;
  f->mask = (f->half == 64) ? ~0ull : ((1ull << f->half) - 1);
  uint64_t s = mix64(seed, purpose);
  for (int i = 0; i < 4; i++) f->key[i] = splitmix64(&s);
}
static inline uint64_t feistel_apply(const feistel_t* f, uint64_t x) {
  uint64_t l = (x >> f->half) & f->mask, r = x & f->mask;
  for (int i = 0; i < 4; i++) {
    uint64_t nl = r;
    r = l ^ (mix64(r, f->key[i]) & f->mask);
    l = nl;
  }
  return (l << f->half) | r;
}
/* permutation of [0, n) by cycle walking */
static inline uint64_t perm_index(const feistel_t* f, uint64_t x, uint64_t n) {
  do { x = feistel_apply(f, x); } while (x >= n);
  return x;
}
static int bits_for(uint64_t n) {
  int b = 0;
  while (b < 64 && (1ull << b) < n) b++;
  return b;
}

/* ---------------- journey plan ---------------- */
typedef struct {
  int64_t jid, len, day, start_ms;
  int64_t count, offset;
  int has_stop;
  int64_t stop_at, stop_ms;
} journey_t;

void cvgen_default(cvgen_params* p) {
  memset(p, 0, sizeof(*p));
  p->seed = 1;
  p->n_journeys = 1000;
  p->len_dist = 0;
  p->median_len = 150.0;
  p->sigma = 0.759;
  p->zipf_s = 1.5;
  p->min_len = 1;
  p->max_len = 200000;
  p->day_start_ms = 1620518400000LL; /* 2021-05-09 00:00:00 UTC, the day of Table 1 */
  p->n_days = 1;
  p->lat_lo = 36.0; p->lat_hi = 40.6; p->lon_lo = -95.8; p->lon_hi = -89.1;
  p->dup_frac = 0.001;
  p->outlier_frac = 0.0005;
  p->stop_prob = 0.05;
  p->negzero_frac = 0.5;
  p->jid_mode = 0;
  p->shuffle = 1;
  p->threads = 0;
}

static int check_params(const cvgen_params* p) {
  if (p->n_journeys < 0 || p->min_len < 1 || p->max_len < p->min_len || p->n_days < 1) return 0;
  if (!(p->lat_hi > p->lat_lo) || !(p->lon_hi > p->lon_lo)) return 0;
  if (p->jid_mode == 0 && p->n_journeys > (1LL << 31)) return 0;
  return 1;
}

static double start_of_day_ms(rng_t* r) {
  /* Diurnal start-time density: a 30% uniform floor plus two peaks, N(8 h, 1.5 h) and
   * N(17 h, 1.5 h), 35% each, truncated to the day. */
  for (;;) {
    double u = rng_unif(r), t;
    if (u < 0.30) t = rng_unif(r) * 24.0;
    else if (u < 0.65) t = 8.0 + 1.5 * rng_normal(r);
    else t = 17.0 + 1.5 * rng_normal(r);
    if (t >= 0.0 && t < 24.0) return t * 3600000.0;
  }
}

static journey_t* make_plan(const cvgen_params* p) {
  int64_t J = p->n_journeys;
  journey_t* jr = (journey_t*)calloc((size_t)(J > 0 ? J : 1), sizeof(journey_t));
  if (!jr) return NULL;
  feistel_t fj;
  feistel_init(&fj, p->jid_mode == 0 ? 32 : 64, p->seed, 0x4A1Dull);
  rng_t r;
  rng_init(&r, p->seed, 0, 0x91A4ull);
  for (int64_t j = 0; j < J; j++) {
    journey_t* q = &jr[j];
    q->jid = (p->jid_mode == 0) ? (int64_t)perm_index(&fj, (uint64_t)j, 1ull << 31)
                                : (int64_t)feistel_apply(&fj, (uint64_t)j);
    double len;
    if (p->len_dist == 0) {
      len = floor(p->median_len * exp(p->sigma * rng_normal(&r)) + 0.5);
    } else {
      double a = (double)p->min_len, b = (double)p->max_len + 1.0, s = p->zipf_s;
      double u = rng_unif(&r);
      double x = pow(pow(a, 1.0 - s) + u * (pow(b, 1.0 - s) - pow(a, 1.0 - s)), 1.0 / (1.0 - s));
      len = floor(x);
    }
    if (len < (double)p->min_len) len = (double)p->min_len;
    if (len > (double)p->max_len) len = (double)p->max_len;
    q->len = (int64_t)len;
    q->day = (p->n_days > 1) ? rng_int(&r, 0, p->n_days - 1) : 0;
    q->start_ms = (int64_t)start_of_day_ms(&r);
    q->has_stop = rng_unif(&r) < p->stop_prob;
    q->stop_at = rng_int(&r, 0, q->len - 1);
    q->stop_ms = rng_int(&r, 10000, 120000);
  }
  return jr;
}

/* Time stream of one journey: returns the step to the next record (0 = duplicate). */
static inline int64_t next_dt(rng_t* tr, double dup_frac) {
  if (rng_unif(tr) < dup_frac) return 0;
  int64_t dt = rng_int(tr, 300, 1000) + (int64_t)llround(20.0 * rng_normal(tr));
  return dt < 1 ? 1 : dt;
}

static int64_t journey_count(const cvgen_params* p, const journey_t* q, int64_t j) {
  rng_t tr;
  rng_init(&tr, p->seed, (uint64_t)j, 0x7131ull);
  int64_t day_end = (q->day + 1) * DAY_MS;
  int64_t t = q->day * DAY_MS + q->start_ms, k = 1;
  while (k < q->len) {
    int64_t dt = next_dt(&tr, p->dup_frac);
    if (t + dt >= day_end) break;
    t += dt;
    k++;
  }
  return k;
}

typedef struct {
  const cvgen_params* p;
  journey_t* jr;
  int64_t n;
  feistel_t fp;
  int64_t *jid, *ts;
  double *lat, *lon;
  float *speed, *heading;
  atomic_llong next;
  int phase;
} work_t;

static void gen_journey(work_t* w, int64_t j) {
  const cvgen_params* p = w->p;
  journey_t* q = &w->jr[j];
  rng_t tr, mr;
  rng_init(&tr, p->seed, (uint64_t)j, 0x7131ull);
  rng_init(&mr, p->seed, (uint64_t)j, 0x30E1ull);
  double lat = p->lat_lo + rng_unif(&mr) * (p->lat_hi - p->lat_lo);
  double lon = p->lon_lo + rng_unif(&mr) * (p->lon_hi - p->lon_lo);
  double hdg = rng_unif(&mr) * 360.0;
  double spd = 20.0 + rng_unif(&mr) * 90.0;
  int64_t t = p->day_start_ms + q->day * DAY_MS + q->start_ms;
  int64_t stop_until = -1;
  int64_t prev_out = -1;
  for (int64_t k = 0; k < q->count; k++) {
    int64_t dt = (k == 0) ? 0 : next_dt(&tr, p->dup_frac);
    uint64_t g = (uint64_t)(q->offset + k);
    int64_t o = p->shuffle ? (int64_t)perm_index(&w->fp, g, (uint64_t)w->n) : (int64_t)g;
    if (k > 0 && dt == 0) { /* exact duplicate of the previous record */
      w->jid[o] = w->jid[prev_out]; w->ts[o] = w->ts[prev_out];
      w->lat[o] = w->lat[prev_out]; w->lon[o] = w->lon[prev_out];
      w->speed[o] = w->speed[prev_out]; w->heading[o] = w->heading[prev_out];
      prev_out = o;
      continue;
    }
    if (k > 0) {
      t += dt;
      int stopped = t < stop_until;
      if (!stopped && q->has_stop && k == q->stop_at) { stop_until = t + q->stop_ms; stopped = 1; }
      hdg += 5.0 * rng_normal(&mr);
      spd += 2.0 * rng_normal(&mr);
      if (spd < 0.0) spd = 0.0;
      if (spd > 130.0) spd = 130.0;
      if (!stopped) {
        double dist = spd / 3.6 * (double)dt / 1000.0; /* flat-earth step, metres */
        double h = hdg * (M_PI / 180.0);
        lat += dist * cos(h) / 111320.0;
        lon += dist * sin(h) / (111320.0 * cos(lat * (M_PI / 180.0)));
        if (lat > p->lat_hi) { lat = 2.0 * p->lat_hi - lat; hdg = 180.0 - hdg; }
        if (lat < p->lat_lo) { lat = 2.0 * p->lat_lo - lat; hdg = 180.0 - hdg; }
        if (lon > p->lon_hi) { lon = 2.0 * p->lon_hi - lon; hdg = -hdg; }
        if (lon < p->lon_lo) { lon = 2.0 * p->lon_lo - lon; hdg = -hdg; }
      }
      hdg = fmod(hdg, 360.0);
      if (hdg < 0.0) hdg += 360.0;
      float out_spd = stopped ? 0.0f : (float)spd;
      w->speed[o] = out_spd;
    } else {
      w->speed[o] = (float)spd;
    }
    double olat = lat, olon = lon;
    double u = rng_unif(&mr);
    if (u < p->outlier_frac) { /* a point written just outside the box */
      double e = 0.0005 + 0.01 * rng_unif(&mr);
      switch ((int)(rng_unif(&mr) * 4.0)) {
        case 0: olat = p->lat_hi + e; break;
        case 1: olat = p->lat_lo - e; break;
        case 2: olon = p->lon_hi + e; break;
        default: olon = p->lon_lo - e; break;
      }
    }
    if (w->speed[o] == 0.0f && rng_unif(&mr) < p->negzero_frac) w->speed[o] = -0.0f;
    w->jid[o] = q->jid;
    w->ts[o] = t;
    w->lat[o] = olat;
    w->lon[o] = olon;
    w->heading[o] = (float)hdg;
    prev_out = o;
  }
}

static void* worker(void* arg) {
  work_t* w = (work_t*)arg;
  const int64_t J = w->p->n_journeys, chunk = 64;
  for (;;) {
    int64_t a = atomic_fetch_add(&w->next, chunk);
    if (a >= J) break;
    int64_t b = a + chunk < J ? a + chunk : J;
    for (int64_t j = a; j < b; j++) {
      if (w->phase == 0) w->jr[j].count = journey_count(w->p, &w->jr[j], j);
      else gen_journey(w, j);
    }
  }
  return NULL;
}

static int n_threads(int32_t req) {
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  if (c < 1) c = 1;
  if (req > 0 && req < c) c = req;
  if (c > 256) c = 256;
  return (int)c;
}

static void run_phase(work_t* w, int phase) {
  w->phase = phase;
  atomic_store(&w->next, 0);
  int nt = n_threads(w->p->threads);
  pthread_t th[256];
  int started = 0;
  for (int i = 0; i < nt; i++)
    if (pthread_create(&th[i], NULL, worker, w) == 0) started++; else break;
  if (started == 0) worker(w);
  for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
}

static int64_t plan_counts(const cvgen_params* p, journey_t* jr) {
  work_t w;
  memset(&w, 0, sizeof(w));
  w.p = p;
  w.jr = jr;
  run_phase(&w, 0);
  int64_t total = 0;
  for (int64_t j = 0; j < p->n_journeys; j++) { jr[j].offset = total; total += jr[j].count; }
  return total;
}

int64_t cvgen_count(const cvgen_params* p) {
  if (!p || !check_params(p)) return -1;
  journey_t* jr = make_plan(p);
  if (!jr) return -2;
  int64_t n = plan_counts(p, jr);
  free(jr);
  return n;
}

int cvgen_fill(const cvgen_params* p, int64_t n, int64_t* jid, int64_t* ts, double* lat,
               double* lon, float* speed, float* heading) {
  if (!p || !check_params(p)) return 1;
  journey_t* jr = make_plan(p);
  if (!jr) return 2;
  int64_t total = plan_counts(p, jr);
  if (total != n) { free(jr); return 3; }
  work_t w;
  memset(&w, 0, sizeof(w));
  w.p = p; w.jr = jr; w.n = n;
  w.jid = jid; w.ts = ts; w.lat = lat; w.lon = lon; w.speed = speed; w.heading = heading;
  feistel_init(&w.fp, bits_for((uint64_t)(n > 1 ? n : 2)), p->seed, 0x5EEDull);
  run_phase(&w, 1);
  free(jr);
  return 0;
}

/* ---------------- CSV ---------------- */
static int fmt_uint(char* o, uint64_t v) {
  char t[24];
  int k = 0;
  do { t[k++] = (char)('0' + v % 10); v /= 10; } while (v);
  for (int i = 0; i < k; i++) o[i] = t[k - 1 - i];
  return k;
}
static int fmt_int(char* o, int64_t v) {
  if (v < 0) { o[0] = '-'; return 1 + fmt_uint(o + 1, (uint64_t)0 - (uint64_t)v); }
  return fmt_uint(o, (uint64_t)v);
}
/* |x| rounded to dec decimals, with a '-' when the sign bit is set */
static int fmt_fixed(char* o, double x, int dec) {
  int k = 0;
  if (signbit(x)) o[k++] = '-';
  double ax = fabs(x);
  double scale = 1.0;
  for (int i = 0; i < dec; i++) scale *= 10.0;
  uint64_t m = (uint64_t)llround(ax * scale);
  uint64_t ip = m, fp = 0;
  uint64_t p10 = 1;
  for (int i = 0; i < dec; i++) p10 *= 10;
  ip = m / p10;
  fp = m % p10;
  k += fmt_uint(o + k, ip);
  if (dec > 0) {
    o[k++] = '.';
    char t[24];
    for (int i = dec - 1; i >= 0; i--) { t[i] = (char)('0' + fp % 10); fp /= 10; }
    memcpy(o + k, t, (size_t)dec);
    k += dec;
  }
  return k;
}

/* Formats row i into o (at least 160 bytes). *bad receives 1 if the row was corrupted. */
static int fmt_row(char* o, int64_t i, const int64_t* jid, const int64_t* ts, const double* lat,
                   const double* lon, const float* speed, const float* heading, uint64_t seed,
                   double mfrac, int* bad) {
  rng_t r;
  rng_init(&r, seed, (uint64_t)i, 0xC5Full);
  int dec = (rng_unif(&r) < 0.5) ? 6 : 7;
  int kind = -1;
  if (rng_unif(&r) < mfrac) kind = (int)(rng_unif(&r) * 7.0);
  *bad = kind >= 0;
  int k = 0;
  k += fmt_int(o + k, jid[i]);
  o[k++] = ',';
  int ts_at = k;
  k += fmt_int(o + k, ts[i]);
  o[k++] = ',';
  if (kind == 4) k += fmt_fixed(o + k, lat[i], 15);        /* 16+ digit mantissa */
  else if (kind == 6) k += fmt_fixed(o + k, 90.5 + fabs(lat[i] - (double)(int64_t)lat[i]), dec);
  else k += fmt_fixed(o + k, lat[i], dec);
  o[k++] = ',';
  k += fmt_fixed(o + k, lon[i], dec);
  o[k++] = ',';
  if (kind == 1) { /* empty field */ }
  else if (kind == 5) { memcpy(o + k, "nan", 3); k += 3; }
  else k += fmt_fixed(o + k, (double)speed[i], 2);
  if (kind != 0) { /* kind 0 drops the last field */
    o[k++] = ',';
    k += fmt_fixed(o + k, (double)heading[i], 1);
  }
  if (kind == 2) { memcpy(o + k, ",0", 2); k += 2; }
  if (kind == 3) o[ts_at + 1] = 'x'; /* a non-digit inside the timestamp */
  o[k++] = '\n';
  return k;
}

typedef struct {
  const int64_t *jid, *ts;
  const double *lat, *lon;
  const float *speed, *heading;
  int64_t n;
  uint64_t seed;
  double mfrac;
  int nchunks;
  int64_t* chunk_bytes;
  int64_t* chunk_bad;
  char* out;
  atomic_int next;
  int phase;
} csv_work_t;

static void* csv_worker(void* arg) {
  csv_work_t* w = (csv_work_t*)arg;
  char row[256];
  for (;;) {
    int c = atomic_fetch_add(&w->next, 1);
    if (c >= w->nchunks) break;
    int64_t a = w->n * c / w->nchunks, b = w->n * (c + 1) / w->nchunks;
    if (w->phase == 0) {
      int64_t bytes = 0, bad = 0;
      for (int64_t i = a; i < b; i++) {
        int isbad;
        bytes += fmt_row(row, i, w->jid, w->ts, w->lat, w->lon, w->speed, w->heading, w->seed,
                         w->mfrac, &isbad);
        bad += isbad;
      }
      w->chunk_bytes[c] = bytes;
      w->chunk_bad[c] = bad;
    } else {
      char* o = w->out + w->chunk_bytes[c];
      for (int64_t i = a; i < b; i++) {
        int isbad;
        o += fmt_row(o, i, w->jid, w->ts, w->lat, w->lon, w->speed, w->heading, w->seed,
                     w->mfrac, &isbad);
      }
    }
  }
  return NULL;
}

int64_t cvgen_csv(const int64_t* jid, const int64_t* ts, const double* lat, const double* lon,
                  const float* speed, const float* heading, int64_t n, uint64_t seed,
                  double malformed_frac, int32_t threads, char* out, int64_t cap,
                  int64_t* n_malformed) {
  if (n < 0) return -1;
  csv_work_t w;
  memset(&w, 0, sizeof(w));
  w.jid = jid; w.ts = ts; w.lat = lat; w.lon = lon; w.speed = speed; w.heading = heading;
  w.n = n; w.seed = seed; w.mfrac = malformed_frac;
  w.nchunks = (int)((n + 65535) / 65536);
  if (w.nchunks < 1) w.nchunks = 1;
  w.chunk_bytes = (int64_t*)calloc((size_t)w.nchunks + 1, sizeof(int64_t));
  w.chunk_bad = (int64_t*)calloc((size_t)w.nchunks + 1, sizeof(int64_t));
  if (!w.chunk_bytes || !w.chunk_bad) { free(w.chunk_bytes); free(w.chunk_bad); return -2; }
  w.out = out;
  int nt = n_threads(threads);
  pthread_t th[256];
  for (int phase = 0; phase < (out ? 2 : 1); phase++) {
    w.phase = phase;
    atomic_store(&w.next, 0);
    int started = 0;
    for (int i = 0; i < nt; i++)
      if (pthread_create(&th[i], NULL, csv_worker, &w) == 0) started++; else break;
    if (started == 0) csv_worker(&w);
    for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
    if (phase == 0) { /* chunk byte counts -> offsets */
      int64_t total = 0, bad = 0;
      for (int c = 0; c < w.nchunks; c++) {
        int64_t b = w.chunk_bytes[c];
        w.chunk_bytes[c] = total;
        total += b;
        bad += w.chunk_bad[c];
      }
      w.chunk_bytes[w.nchunks] = total;
      if (n_malformed) *n_malformed = bad;
      if (out && total > cap) { free(w.chunk_bytes); free(w.chunk_bad); return -3; }
    }
  }
  int64_t total = w.chunk_bytes[w.nchunks];
  free(w.chunk_bytes);
  free(w.chunk_bad);
  return total;
}
