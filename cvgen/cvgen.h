/*
 * cvgen.h — seeded synthetic connected-vehicle records.
 *
 * Stands in for the Missouri DOT connected-vehicle dataset described in the paper
 * (arXiv 2305.07454, Methods, "Connected Vehicle Dataset"; Table 1), which is not
 * available. It produces shuffled records (journey id, timestamp ms, latitude, longitude,
 * speed km/h, heading deg) of statewide shape: lognormal or Zipf journey lengths,
 * sub-second sampling, a diurnal start-time curve, random-walk trajectories inside a
 * bounding box, exact duplicate records, stop runs and points just outside the box.
 *
 * This module only draws inputs. It contains none of the ETL method's arithmetic, and both
 * the CPU oracle and the CUDA library consume the same bytes it writes.
 */
#ifndef CVGEN_H
#define CVGEN_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint64_t seed;
  int64_t n_journeys;
  int32_t len_dist;     /* 0: lognormal(median_len, sigma); 1: Zipf(zipf_s) on [min_len, max_len] */
  double median_len;
  double sigma;
  double zipf_s;
  int64_t min_len, max_len;
  int64_t day_start_ms; /* UTC ms of the first day's midnight */
  int32_t n_days;       /* journeys start on a uniformly drawn day and end by its midnight */
  double lat_lo, lat_hi, lon_lo, lon_hi;
  double dup_frac;      /* probability that a record repeats its predecessor exactly */
  double outlier_frac;  /* probability that a record is written just outside the box */
  double stop_prob;     /* probability that a journey holds one stop run */
  double negzero_frac;  /* share of exact-zero speeds written as -0.0 */
  int32_t jid_mode;     /* 0: distinct ids in [0, 2^31); 1: distinct ids over all of int64 */
  int32_t shuffle;      /* 1: records in a keyed pseudo-random order; 0: journey order */
  int32_t threads;      /* worker threads (0 = all online cores) */
} cvgen_params;

/* Fills *p with the small-workload defaults (1,000 journeys, median 150 points). */
void cvgen_default(cvgen_params* p);

/* Number of records the parameters produce. Negative on bad parameters. */
int64_t cvgen_count(const cvgen_params* p);

/* Writes exactly cvgen_count(p) records. Returns 0 on success. */
int cvgen_fill(const cvgen_params* p, int64_t n, int64_t* jid, int64_t* ts, double* lat,
               double* lon, float* speed, float* heading);

/* CSV serialisation of columns: lat/lon with 6 or 7 decimals (drawn per row), speed with 2,
 * heading with 1, integers in decimal, no header, '\n' line ends. A share malformed_frac of
 * rows is corrupted, uniformly over seven kinds (missing field, empty field, extra field,
 * non-digit character, 16-digit mantissa, "nan", latitude out of range).
 * With out == NULL returns the byte count; otherwise writes it (cap bytes available) and
 * returns it, and *n_malformed receives the number of corrupted rows. Negative on error. */
int64_t cvgen_csv(const int64_t* jid, const int64_t* ts, const double* lat, const double* lon,
                  const float* speed, const float* heading, int64_t n, uint64_t seed,
                  double malformed_frac, int32_t threads, char* out, int64_t cap,
                  int64_t* n_malformed);

#ifdef __cplusplus
}
#endif
#endif
