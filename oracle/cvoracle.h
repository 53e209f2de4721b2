/*
 * cvoracle.h — plain, single-threaded CPU oracle of the connected-vehicle ETL hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library. The product path (the CUDA library) never calls it and
 * shares no code, header or table with it.
 *
 * What it computes (arXiv 2305.07454, "Accelerating Statewide Connected Vehicles Big
 * (Sensor Fusion) Data ETL Pipelines on GPUs"):
 *   - extract: CSV rows of (journey_id, timestamp, latitude, longitude, speed, heading)
 *     (Methods, "Connected Vehicle Dataset": per-vehicle CSV text; Table 1 shows the
 *     columns) filtered to the columns of interest (Accelerated ETL section, step (2));
 *   - transform: order by journey and time, per-point kinematics, and the floor-division
 *     binning of Algorithm 2 (time bin, latitude bin, longitude bin) unrolled into one
 *     global positional index (Accelerated ETL section, steps (3)-(4));
 *   - load: groupby count / sum / mean (Table 3 "Data Binning", "Reduction - Sum") plus
 *     min / max per lattice cube (steps (5)-(6)), and per-journey summaries.
 * The paper gives no per-journey kinematics; those definitions are readings stated at
 * each function in cvoracle.c.
 *
 * Arithmetic: IEEE binary64 with round-to-nearest, compiled with -ffp-contract=off and
 * without -ffast-math, so each written operation is one correctly rounded operation.
 */
#ifndef CVORACLE_H
#define CVORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_KEY_INVALID 0xFFFFFFFFu

/* per-point flags */
#define ORC_F_START   0x01u /* first point of its journey */
#define ORC_F_DUP     0x02u /* same timestamp as its predecessor in the journey */
#define ORC_F_OFFGRID 0x04u /* outside the grid or the day's time bins */
#define ORC_F_STOP    0x08u /* both this point and its predecessor are below the stop speed */

typedef struct {
  double lat_min, lon_min, cell_deg;
  int32_t n_rows, n_cols, n_bins;
  int64_t t0_ms, bin_ms;
  float v_stop_kmh;
  double earth_radius_m;
} orc_params;

/* Per-point outputs, in sorted order, each of length n_valid. */
typedef struct {
  uint32_t* perm;   /* input index of the sorted point */
  double* d;        /* haversine step distance, metres */
  double* vhat;     /* implied speed, km/h */
  double* accel;    /* acceleration, m/s^2 */
  int64_t* dwell;   /* dwell time of the step, ms */
  uint32_t* key;    /* unrolled cell x bin key, or ORC_KEY_INVALID */
  uint8_t* flags;   /* ORC_F_* */
  int64_t* stop_ms; /* time since the current stop began: dwell summed over the run of stop steps */
  double* accel_v;  /* acceleration from the implied speeds, m/s^2 (0 unless both steps have dt > 0) */
} orc_points;

/* Journey table, one row per distinct journey id, ascending id. Capacity >= n_valid. */
typedef struct {
  int64_t* jid;
  int64_t* n;
  int64_t* start_ts;
  int64_t* end_ts;
  int64_t* duration_ms;
  double* distance_m;
  int64_t* dwell_ms;
  double* start_lat;
  double* start_lon;
  double* end_lat;
  double* end_lon;
} orc_journeys;

/* Cell x bin table, one row per occupied key, ascending key. Capacity >= n_valid. */
typedef struct {
  uint32_t* key;
  int32_t* row;
  int32_t* col;
  int32_t* bin;
  uint32_t* count;
  double* sum;
  double* mean;
  float* min;
  float* max;
  uint32_t* volume; /* unique journeys (Table 3, "Reduction - Count Unique (Volume)") */
} orc_cells;

typedef struct {
  int64_t n_in;         /* records handed to the run */
  int64_t n_malformed;  /* records dropped by validation */
  int64_t n_valid;      /* records kept */
  int64_t n_out_of_grid;
  int64_t n_dup;
  int64_t n_journeys;
  int64_t n_cells;
} orc_counters;

/* Decimal field -> double, per the CSV grammar. Returns 1 and sets *out if the field is a
 * well-formed decimal, else 0. */
int orc_parse_decimal(const char* s, int64_t len, double* out);
/* Integer field -> int64, per the CSV grammar. */
int orc_parse_integer(const char* s, int64_t len, int64_t* out);

/* Parse CSV text. Every line is a row, in file order (its extracted-row index is its line
 * number); a line that breaks the grammar becomes the row (0, 0, NaN, NaN, NaN, NaN), which
 * the extract drops as malformed. The columns must have room for every line. Returns the
 * number of rows (-1 if cap is too small); *n_lines and *n_malformed are set. */
int64_t orc_parse_csv(const char* buf, int64_t len, int64_t cap,
                      int64_t* jid, int64_t* ts, double* lat, double* lon,
                      float* speed, float* heading,
                      int64_t* n_lines, int64_t* n_malformed);

/* Great-circle distance in metres between two points given in degrees. */
double orc_haversine_m(double lat1, double lon1, double lat2, double lon2, double radius_m);
/* floor((x - x_min) / step) as an int if it lies in [0, n) and x is finite; else -1. */
int32_t orc_grid_index(double x, double x_min, double step, int32_t n);
/* floor((ts - t0) / bin_ms) if it lies in [0, n_bins); else -1. */
int32_t orc_time_bin(int64_t ts, int64_t t0_ms, int64_t bin_ms, int32_t n_bins);

/* The whole path. Returns 0 on success, non-zero on bad arguments or allocation failure. */
int orc_run(const orc_params* p, int64_t n,
            const int64_t* jid, const int64_t* ts, const double* lat, const double* lon,
            const float* speed,
            orc_points* pts, orc_journeys* jr, orc_cells* cl, orc_counters* cnt);

/* ---- Lattice (the paper's 8-channel spatio-temporal image; Results, the 5-minute channel
 * images of speed and volume in four cardinal directions; Algorithm 2, step 3; Table 3,
 * "Count Unique (Volume)" and "Normalize"). */
#define ORC_DXN_CARDINAL 0 /* floor(((h + 45) mod 360) / 90): 0 N, 1 E, 2 S, 3 W (reading) */
#define ORC_DXN_QUADRANT 1 /* floor((h mod 360) / 90): Algorithm 2's heading // 90 as printed */

/* Direction channel of a heading in degrees; -1 for a non-finite heading. */
int32_t orc_direction(float heading, int32_t mode);

typedef struct {
  int64_t bin_ms;     /* lattice time bin, from the run's t0_ms (300000: 5 minutes) */
  int32_t n_bins;     /* 288 for a day of 5-minute bins */
  int32_t direction;  /* ORC_DXN_* */
} orc_lattice_params;

/* One row per occupied (bin, direction, row, col), ascending key; capacity >= kept rows. */
typedef struct {
  uint32_t* key;      /* ((bin * 4 + dxn) * n_rows + row) * n_cols + col */
  int32_t *bin, *dxn, *row, *col;
  uint32_t* count;    /* points */
  double* sum;        /* speed sum, sequential in (journey id, input index) order */
  float* mean;        /* (float)(sum / count): channel 2 * dxn */
  uint32_t* volume;   /* distinct journeys: channel 2 * dxn + 1 */
  float* mean_norm;   /* min-max normalised per channel over the occupied cells */
  float* volume_norm;
} orc_lattice_cells;

/* The lattice of the kept rows (the same row rule as orc_run) that have a finite heading and
 * fall inside the grid and the lattice's bins. ch_min / ch_max: per channel over its
 * occupied cells (0 for a channel without cells). Returns 0 on success. */
int orc_lattice(const orc_params* p, const orc_lattice_params* lp, int64_t n, const int64_t* jid,
                const int64_t* ts, const double* lat, const double* lon, const float* speed,
                const float* heading, orc_lattice_cells* out, int64_t* n_cells, int64_t* n_dropped,
                float* ch_min, float* ch_max);

#ifdef __cplusplus
}
#endif
#endif
