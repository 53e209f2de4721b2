/*
 * cvetl.h — C ABI of the connected-vehicle ETL library (libcvetl.so, CUDA, sm_103a).
 *
 * The library runs the data-parallel hot path of the connected-vehicle extract-transform-
 * load pipeline of arXiv 2305.07454 ("Accelerating Statewide Connected Vehicles Big
 * (Sensor Fusion) Data ETL Pipelines on GPUs"), following the paper's extract / transform /
 * load framing (Introduction, definition of ETL):
 *
 *   extract    records (journey id, timestamp, latitude, longitude, speed, heading) from
 *              binary columns or CSV text (Methods, "Connected Vehicle Dataset"; Table 1),
 *              keeping the columns of interest (Accelerated ETL section, step (2));
 *   transform  order by (journey id, timestamp), per-point kinematics, and the floor-
 *              division bins of Algorithm 2 unrolled into one global positional index
 *              (Accelerated ETL section, steps (3)-(4));
 *   load       per cell x time-bin count / sum / mean (Table 3 "Data Binning", "Reduction -
 *              Sum") plus min / max, and per-journey summaries (steps (5)-(6)).
 *
 * Every step runs in the library's own CUDA kernels on one GPU. There is no CPU fallback: a
 * call that cannot run on the device returns an error.
 *
 * Conventions
 *  - Every call returns a cvetl_status and never aborts or throws across the ABI.
 *    cvetl_last_error() returns the context's last error text.
 *  - Calls are stream-ordered on config.stream (a cudaStream_t; NULL = the legacy default
 *    stream). The caller owns input buffers. Host inputs are copied during cvetl_extract;
 *    device inputs are read in place, so the caller keeps them alive and unchanged until the
 *    work of cvetl_transform has completed on the stream.
 *  - Result arrays are device memory owned by the context. They stay valid until the next
 *    cvetl_extract or cvetl_destroy.
 *  - Call order per batch: cvetl_extract -> cvetl_transform -> cvetl_load -> cvetl_results.
 *    A call out of order returns CVETL_ESTATE and changes nothing.
 *  - One context per host thread. Different contexts may run concurrently on different
 *    streams.
 *  - Sizes: at most CVETL_MAX_RECORDS records per batch.
 */
#ifndef CVETL_H
#define CVETL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CVETL_VERSION 1
#define CVETL_MAX_RECORDS 1073741823LL /* 2^30 - 1 */
#define CVETL_KEY_INVALID 0xFFFFFFFFu

typedef struct cvetl_ctx cvetl_ctx;

typedef enum {
  CVETL_OK = 0,
  CVETL_EINVAL = 1,   /* bad argument (NULL pointer, bad size, bad configuration) */
  CVETL_ENOMEM = 2,   /* device allocation failed */
  CVETL_EFULL = 3,    /* the request would exceed config.mem_budget_bytes; state unchanged */
  CVETL_ESTATE = 4,   /* call out of order */
  CVETL_ECUDA = 5,    /* a CUDA runtime error; see cvetl_last_error */
  CVETL_ETIMEOUT = 6, /* a bounded device-side wait gave up; results are not valid */
  CVETL_EPARSE = 7    /* reserved for unrecoverable input errors */
} cvetl_status;

enum { CVETL_FP64 = 0, CVETL_FP32 = 1 };
enum { CVETL_IN_COLUMNS = 0, CVETL_IN_CSV = 1 };
enum { CVETL_BATCH = 0, CVETL_STREAM = 1 };

/* per-point flags */
#define CVETL_F_START 0x01u   /* first point of its journey */
#define CVETL_F_DUP 0x02u     /* same timestamp as its predecessor in the journey */
#define CVETL_F_OFFGRID 0x04u /* outside the grid or the day's time bins (key invalid) */
#define CVETL_F_STOP 0x08u    /* this point and its predecessor both below v_stop_kmh */

typedef struct {
  /* Grid of Algorithm 2: row = floor((lat - lat_min) / cell_deg), col likewise for lon,
   * valid when 0 <= row < n_rows and 0 <= col < n_cols. */
  double lat_min, lon_min, cell_deg; /* 36.0, -95.8, 0.01 */
  int32_t n_rows, n_cols;            /* 460, 670 */
  /* Time bins: bin = floor((ts - t0_ms) / bin_ms), valid when 0 <= bin < n_bins. */
  int32_t n_bins;                    /* 1440 */
  int64_t t0_ms, bin_ms;             /* 2021-05-09 00:00:00 UTC in ms, 60000 */
  float v_stop_kmh;                  /* 1.0: dwell threshold */
  double earth_radius_m;             /* 6371000.0 */
  int32_t precision;                 /* CVETL_FP64: distances in binary64. CVETL_FP32: coordinates
                                        differenced in binary64, the haversine and per-point
                                        arithmetic in float32, distance and speed sums in
                                        compensated float32 (keys, counts, order unchanged) */
  int32_t materialize_points;        /* 1: keep per-point columns in the results */
  int32_t profile;                   /* 1: time every kernel with CUDA events */
  int32_t device;                    /* CUDA device ordinal */
  size_t mem_budget_bytes;           /* device memory the context may hold; 0 = unlimited */
  void* stream;                      /* cudaStream_t */
  int32_t mode;                      /* CVETL_BATCH (one batch per extract) or CVETL_STREAM */
  int64_t lateness_ms;               /* stream mode: how late a record may arrive (30000) */
  int32_t graph;                     /* batch mode, 1: after the journey count is read back, the
                                        rest of transform and load runs as a CUDA graph, captured
                                        on the first run of a shape (rows, journeys, kept rows,
                                        buffers, inputs, launch shapes) and replayed when the
                                        shape repeats; per-kernel profile times are not taken for
                                        replays. Buffers that depend on the run count are then
                                        sized for one run per kept point. */
} cvetl_config;

typedef struct {
  int32_t kind;       /* CVETL_IN_COLUMNS or CVETL_IN_CSV */
  int32_t on_device;  /* 1: the pointers below are device memory */
  int64_t n;          /* rows (CVETL_IN_COLUMNS) */
  /* CVETL_IN_COLUMNS: six columns of n rows. heading may be NULL (it is not used). */
  const int64_t* jid;
  const int64_t* ts;
  const double* lat;
  const double* lon;
  const float* speed;
  const float* heading;
  /* CVETL_IN_CSV: csv_len bytes of text (see the grammar at cvetl_extract). */
  const char* csv;
  size_t csv_len;
  /* stream mode: the end of the window's arrival interval (ms, same clock as ts); after the
   * window the watermark is window_end_ms - lateness_ms */
  int64_t window_end_ms;
} cvetl_input;

typedef struct {
  /* cell x bin table, ascending key (device pointers, n_cells rows) */
  int64_t n_cells;
  const uint32_t* cell_key;
  const int32_t* cell_row;
  const int32_t* cell_col;
  const int32_t* cell_bin;
  const uint32_t* cell_count;
  const double* cell_sum;
  const double* cell_mean;
  const float* cell_min;
  const float* cell_max;
  const uint32_t* cell_volume;  /* unique journeys (Table 3, count unique); NULL in stream mode */
  /* journey table, ascending journey id (device pointers, n_journeys rows) */
  int64_t n_journeys;
  const int64_t* j_id;
  const int64_t* j_n;
  const int64_t* j_offset;      /* sorted position of the journey's first point */
  const int64_t* j_start_ts;
  const int64_t* j_end_ts;
  const int64_t* j_duration_ms;
  const double* j_distance_m;
  const int64_t* j_dwell_ms;
  const double* j_start_lat;
  const double* j_start_lon;
  const double* j_end_lat;
  const double* j_end_lon;
  /* per-point columns in sorted order (NULL unless materialize_points; n_points rows) */
  int64_t n_points;
  const uint32_t* p_perm;  /* extracted-row index of the sorted point */
  const double* p_d;       /* haversine step distance, m */
  const float* p_vhat;     /* implied speed, km/h */
  const float* p_accel;    /* acceleration, m/s^2 */
  const int64_t* p_dwell;  /* dwell of the step, ms */
  const uint32_t* p_key;   /* unrolled cell x bin key or CVETL_KEY_INVALID */
  const uint8_t* p_flags;  /* CVETL_F_* */
  const int64_t* p_stop_ms; /* time since the current stop began: dwell summed over consecutive stop steps */
  const float* p_accel_v;   /* acceleration from the implied speeds of this and the previous step, m/s^2
                               (binary64, 0 unless both steps have dt > 0) */
  /* extracted columns (device; the CSV path's parsed rows, or the caller's columns), n_extracted rows */
  int64_t n_extracted;
  const int64_t* x_jid;
  const int64_t* x_ts;
  const double* x_lat;
  const double* x_lon;
  const float* x_speed;
  const float* x_heading;  /* NULL when the caller's binary columns had no heading */
  /* counters */
  int64_t n_in;          /* rows handed to cvetl_extract */
  int64_t n_malformed;   /* rows dropped by validation */
  int64_t n_valid;       /* rows kept */
  int64_t n_out_of_grid; /* kept rows whose key is invalid */
  int64_t n_dup;         /* kept rows flagged CVETL_F_DUP */
  int64_t n_too_late;    /* always 0 in batch mode */
  int64_t n_runs;        /* runs of equal consecutive keys folded by the load stage */
} cvetl_tables;

#define CVETL_MAX_STAGES 32
typedef struct {
  int32_t n_stages;
  const char* name[CVETL_MAX_STAGES];   /* kernel / stage names (static strings) */
  double ms[CVETL_MAX_STAGES];          /* summed CUDA-event time (profile = 1) */
  int64_t launches[CVETL_MAX_STAGES];   /* kernel launches */
  int64_t total_launches;               /* all of this context's kernel launches */
  int64_t device_bytes;                 /* device memory the context holds now */
  int64_t graph_replays;                /* CUDA graph launches (config.graph) */
} cvetl_stats;

/* Fills *cfg with the statewide defaults listed beside each field. */
void cvetl_config_default(cvetl_config* cfg);

/* Creates a context. Validates the configuration: positive grid and bin sizes,
 * n_rows * n_cols * n_bins <= 2^32 - 1 (so every key fits in 32 bits and differs from
 * CVETL_KEY_INVALID), finite lat_min / lon_min, cell_deg > 0. Returns CVETL_EINVAL on a bad
 * configuration, CVETL_ECUDA if the device cannot be used. *out is set only on success. */
cvetl_status cvetl_create(const cvetl_config* cfg, cvetl_ctx** out);

/* Extract (Methods, "Connected Vehicle Dataset"; Accelerated ETL step (2)).
 * CVETL_IN_COLUMNS: takes n rows. A row is kept when lat, lon and speed are finite,
 * |lat| <= 90 and |lon| <= 180; otherwise it is counted in n_malformed. Speed -0.0 is read
 * as +0.0.
 * CVETL_IN_CSV: csv_len bytes of text (host or device; a device buffer that is not 16-byte
 * aligned is copied). Grammar (the paper's CSV files, Table 1, have no stated grammar; this is
 * the library's): lines end at '\n' (one trailing '\r' is stripped, the last line may lack
 * '\n'); a row is exactly six ','-separated fields jid,ts,lat,lon,speed,heading; jid and ts
 * match -?[0-9]{1,18}; the others match -?[0-9]+(\.[0-9]+)? with at most 15 digits and take the
 * binary64 value nearest to the decimal (speed and heading then rounded to float32);
 * |lat| <= 90 and |lon| <= 180. Every line is a row and its row index is its line number
 * (0-based, file order); any other line (empty lines included) becomes the row
 * (0, 0, NaN, NaN, NaN, NaN), which is dropped and counted in n_malformed; n_in counts lines.
 * Replaces the context's previous batch. Returns CVETL_EINVAL for NULL columns or
 * n outside [0, CVETL_MAX_RECORDS], CVETL_EFULL if the budget is exceeded. */
cvetl_status cvetl_extract(cvetl_ctx* ctx, const cvetl_input* in);

/* Transform (Accelerated ETL steps (3)-(4); Algorithm 2). Orders the kept rows by
 * (journey id, timestamp, extracted-row index), then for each point computes: the journey
 * start flag; dt = ts - ts_prev; the haversine step distance on a sphere of radius
 * earth_radius_m; implied speed d / dt * 3.6 km/h and acceleration (speed - speed_prev) /
 * 3.6 / dt m/s^2 when dt > 0 (else 0); dwell = dt when both speeds are below v_stop_kmh;
 * and the key (bin * n_rows + row) * n_cols + col with row, col, bin the floor-division
 * bins of Algorithm 2 (row and col taken from the IEEE binary64 quotient of the binary64
 * difference). Also builds the journey table. */
cvetl_status cvetl_transform(cvetl_ctx* ctx);

/* Load (Accelerated ETL steps (5)-(6); Table 3). Groups points with a valid key into the
 * cell x bin table: count, sum of speed (binary64), min, max, mean = sum / count. */
cvetl_status cvetl_load(cvetl_ctx* ctx);

/* Results of the last batch: device pointers owned by the context, sizes and counters.
 * After cvetl_extract alone it reports the extracted columns and n_in (the cell, journey and
 * point tables are empty until cvetl_load). Synchronises ctx->stream (it reads the sizes). */
cvetl_status cvetl_results(cvetl_ctx* ctx, cvetl_tables* out);

/* Batch of instances (the paper runs one statewide day at a time; this takes many days and
 * regions of very uneven size in one pass of every kernel). An instance has its own grid
 * origin and size and its own day; cell_deg, n_bins, bin_ms, the thresholds and the precision
 * are the context's. */
typedef struct {
  double lat_min, lon_min;  /* grid origin of the instance */
  int32_t n_rows, n_cols;   /* its grid size */
  int64_t t0_ms;            /* start of its first time bin */
  int64_t n;                /* rows */
  const int64_t* jid;
  const int64_t* ts;
  const double* lat;
  const double* lon;
  const float* speed;
} cvetl_instance;

#define CVETL_MAX_INSTANCES 32

/* Extract for a batch (batch-mode context): the instances' rows are taken in instance order
 * (all host or all device columns, per on_device), and cvetl_transform / cvetl_load then
 * treat every instance as its own batch in one pass: a journey is (instance, journey id), a
 * point is keyed on its instance's grid and day. The result tables hold the instances one after
 * another: journeys by (instance, id), cells by (instance, key) with each instance's own keys,
 * rows and columns (cvetl_batch_ranges gives each instance's slice). Materialised per-point keys
 * are offset by the instance's first key. Counters are totals.
 * CVETL_EINVAL for n_inst outside [1, CVETL_MAX_INSTANCES], a NULL column, a bad grid, more than
 * CVETL_MAX_RECORDS rows, or keys (sum of n_rows * n_cols * n_bins) reaching 2^32 - 1; the
 * journey ids of a batch must lie within [-2^57, 2^57) (cvetl_transform returns CVETL_EINVAL
 * otherwise). Host columns are copied before the call returns; device columns are read in
 * place through a table of their pointers (not copied), so, as for cvetl_extract, the caller
 * keeps them alive and unchanged until the work of cvetl_transform (and of cvetl_autotune, which
 * repeats it) has completed on the stream. */
cvetl_status cvetl_extract_batch(cvetl_ctx* ctx, const cvetl_instance* inst, int32_t n_inst, int32_t on_device);

/* Slices of a loaded batch, n = n_inst + 1 entries per array (any array may be NULL): the first
 * extracted row, first key, first cell row and first journey row of each instance, the last
 * entry being the total. CVETL_ESTATE unless the last batch was a cvetl_extract_batch taken
 * through cvetl_load. */
cvetl_status cvetl_batch_ranges(cvetl_ctx* ctx, int64_t* row_begin, int64_t* key_begin, int64_t* cell_begin,
                                int64_t* journey_begin, int32_t n);

/* Launch shapes. They change how the work is spread over the GPU, never a result bit. */
typedef struct {
  int32_t journey_ctas;    /* 0: one CTA per journey, longest journey first (default); 1..3: that
                              many persistent CTAs per SM taking journeys from the longest-first
                              work list */
  int32_t row_unroll;      /* rows per thread per iteration of the counting pass and the scatter:
                              2, 4 (default) or 8 */
  int32_t small_sort_max;  /* sorts of up to this many pairs run in one thread block (0..4096,
                              default 4096), larger ones device-wide */
  int32_t row_block;       /* threads per block of the counting pass (and of the scatter of
                              unaligned columns): 128, 256 (default) or 512 */
  int32_t small_journey_max; /* journeys of up to this many points (0..512, default 512) take
                                64-thread CTAs of a second journey kernel, the rest the 256-thread
                                one; 0: every journey takes a 256-thread CTA */
  int32_t scatter_block;   /* threads per block of the scatter of aligned columns (16 consecutive
                              rows per thread): 128 (default), 256 or 512 */
} cvetl_tuning;

cvetl_status cvetl_tuning_get(cvetl_ctx* ctx, cvetl_tuning* out);
/* CVETL_EINVAL for a value outside the ranges above (the context keeps its shapes). */
cvetl_status cvetl_tuning_set(cvetl_ctx* ctx, const cvetl_tuning* t);

/* Autotuner (batch-mode contexts). Times cvetl_transform + cvetl_load on the extracted rows
 * with CUDA events for candidate shapes: each field in turn over its candidates (journey_ctas
 * 0..3, row_unroll 2/4/8, small_sort_max 0/1024/2048/4096, row_block 128/256/512,
 * small_journey_max 0/128/256/512, scatter_block 128/256/512) with the others fixed, the median of
 * `reps` timed runs (1..10) after one untimed run per candidate, a candidate kept only when at
 * least 2% faster. The context keeps the fastest shapes; *out (may be NULL) receives them and
 * *ms_best (may be NULL) their median time. Needs a preceding cvetl_extract or
 * cvetl_extract_batch (CVETL_ESTATE otherwise) whose inputs stay valid during the call, and
 * leaves the context extracted: call cvetl_transform and cvetl_load next. Launch statistics are
 * left as they were. */
cvetl_status cvetl_autotune(cvetl_ctx* ctx, int32_t reps, cvetl_tuning* out, double* ms_best);

/* Lattice (the paper's multidimensional spatio-temporal output: each lattice time bin is an
 * image of 8 channels, speed and volume in the four cardinal directions, Results; direction
 * by Algorithm 2, step 3; volume as unique journeys, Table 3 "Count Unique (Volume)"; min-max
 * normalised channels, Table 3 "Normalize"). Channel 2d is the mean point speed and channel
 * 2d + 1 the number of unique journeys of direction d in a cell and lattice bin. */
enum {
  CVETL_DXN_CARDINAL = 0, /* floor(((heading + 45) mod 360) / 90): 0 N, 1 E, 2 S, 3 W */
  CVETL_DXN_QUADRANT = 1  /* floor((heading mod 360) / 90), the printed heading // 90 */
};

typedef struct {
  int64_t bin_ms;     /* lattice bin from config.t0_ms (300000: 5 minutes) */
  int32_t n_bins;     /* 288 */
  int32_t direction;  /* CVETL_DXN_* */
  int32_t dense;      /* 1: also write the dense tensor (n_bins * 8 * n_rows * n_cols floats) */
  int32_t normalize;  /* 1: the dense tensor holds the normalised channels */
} cvetl_lattice_config;

typedef struct {
  /* occupied (bin, direction, cell), ascending key = ((bin * 4 + dxn) * n_rows + row) * n_cols + col */
  int64_t n_cells;
  const uint32_t* key;
  const int32_t *bin, *dxn, *row, *col;
  const uint32_t* count;    /* points */
  const double* sum;        /* speed sum, in (journey, extracted-row) order */
  const float* mean;        /* (float)(sum / count) */
  const uint32_t* volume;   /* unique journeys */
  const float* mean_norm;   /* (mean - min) / (max - min) of its channel over the occupied cells, 0 if max = min */
  const float* volume_norm;
  int64_t n_dropped;        /* kept rows without a finite heading or outside the grid or the lattice bins */
  const float* dense;       /* [n_bins][8][n_rows][n_cols] (zero where unoccupied), or NULL */
  int32_t n_bins;
  float ch_min[8], ch_max[8]; /* per channel over its occupied cells (0 for an empty channel) */
} cvetl_lattice;

void cvetl_lattice_config_default(cvetl_lattice_config* lc);

/* Builds the lattice of the last batch (batch mode, one instance, after cvetl_load; the
 * extracted rows need headings: binary columns with a heading column, or CSV). Kept rows are
 * keyed by lattice bin, direction and cell (the same thresholds as the cell keys) and grouped
 * with the library's radix sort by (key, journey rank), ties in extracted-row order; one thread
 * per cell then folds its points in that order. Device arrays stay valid until the next
 * cvetl_extract or cvetl_lattice_build. CVETL_ESTATE before cvetl_load; CVETL_EINVAL for a
 * stream context, a batch of instances, missing headings or a bad configuration. */
cvetl_status cvetl_lattice_build(cvetl_ctx* ctx, const cvetl_lattice_config* lc, cvetl_lattice* out);

/* Stream mode (config.mode = CVETL_STREAM; the paper runs batches only, this serves windows of
 * records as they arrive). Per window: cvetl_extract appends the window's rows (binary columns)
 * to a pending store on the device; cvetl_transform finalises every pending point whose
 * timestamp is at or below the watermark W = window_end_ms - lateness_ms, in (journey,
 * timestamp, arrival) order, each journey continuing from its device-resident last point, open
 * run and running sums; cvetl_load folds the window's closed runs into the device-resident
 * cell table. A row whose timestamp is below the previous window's watermark when it arrives
 * is dropped and counted in n_too_late. cvetl_results reports the tables of everything
 * finalised so far. cvetl_flush finalises every pending point and closes every open run (end of
 * the stream); afterwards the tables equal those of one batch over the same rows (integers,
 * min and max exactly, sums within rounding) and the stream accepts no more windows.
 * Windows must come in order of window_end_ms. In stream mode cvetl_extract returns without
 * waiting for the GPU (host columns are copied before it returns); its drop counters and any
 * device error of the append are read, and reported, by the window's cvetl_transform.
 * In batch mode cvetl_flush returns CVETL_ESTATE. */
cvetl_status cvetl_flush(cvetl_ctx* ctx);

/* Per-kernel launch counts and (with profile = 1) CUDA-event times, summed since the
 * context was created or since cvetl_stats_reset. Synchronises ctx->stream. */
cvetl_status cvetl_stats_get(cvetl_ctx* ctx, cvetl_stats* out);
cvetl_status cvetl_stats_reset(cvetl_ctx* ctx);

/* Frees the context and all its device memory. NULL is accepted. */
cvetl_status cvetl_destroy(cvetl_ctx* ctx);

/* Last error text of the context (or of the last failed cvetl_create when ctx is NULL). */
const char* cvetl_last_error(const cvetl_ctx* ctx);

int32_t cvetl_version(void);

/* ---- Serving runtime ---------------------------------------------------------------------
 * The paper processes whole days as batches; the server serves windows of records as they
 * arrive, with continuous batching across feeds. A feed is one stream-mode context (its own
 * non-blocking CUDA stream, open-journey state and running cell table on the device). Each
 * submitted window or flush is a request with a ticket. n_slots worker threads take requests
 * from one FIFO queue: the requests of one feed run one at a time in submission order, the
 * requests of different feeds run at the same time on their own streams, so windows that
 * arrive while others are on the GPU start as soon as a slot and the memory budget allow.
 * Admission by memory: a request reserves kServeBytesPerRow (CVETL_SERVE_BYTES_PER_ROW) per
 * row while it runs; it is admitted when the memory the feeds hold plus the reservations of
 * the running requests plus its own fits in mem_budget_bytes, or when nothing else runs.
 * Admission is first come, first served: when the oldest request that its feed's order allows
 * does not fit, no later request starts before it. */
#define CVETL_SERVE_BYTES_PER_ROW 320
#define CVETL_SERVE_MAX_SLOTS 64

typedef struct cvetl_server cvetl_server;

typedef struct {
  int32_t n_slots;          /* requests on the GPU at once (worker threads), 1..CVETL_SERVE_MAX_SLOTS */
  int32_t device;           /* CUDA device ordinal */
  size_t mem_budget_bytes;  /* device memory of all feeds plus running reservations; 0 = unlimited */
} cvetl_server_config;

typedef struct {
  int32_t status;     /* cvetl_status of the request */
  int32_t feed;
  int32_t kind;       /* 0 window, 1 flush */
  int32_t slot;       /* the worker that ran it */
  int64_t n;          /* rows of the window */
  int64_t submit_ns;  /* steady clock (CLOCK_MONOTONIC) at submission */
  int64_t start_ns;   /* at admission */
  int64_t done_ns;    /* when its work had completed on the GPU */
  int32_t peak_in_flight; /* most requests running at once at any time so far (server-wide) */
  char message[164];  /* error text when status != CVETL_OK */
} cvetl_ticket_info;

/* Creates the server and its n_slots worker threads. CVETL_EINVAL for n_slots outside
 * [1, CVETL_SERVE_MAX_SLOTS]. */
cvetl_status cvetl_server_create(const cvetl_server_config* cfg, cvetl_server** out);

/* Adds a feed: a stream-mode context created from *cfg (mode, stream, device and
 * mem_budget_bytes are set by the server) on a new non-blocking stream. *feed gets its index. */
cvetl_status cvetl_server_add_feed(cvetl_server* s, const cvetl_config* cfg, int32_t* feed);

/* Queues one window of binary columns (in->kind = CVETL_IN_COLUMNS, host or device pointers,
 * in->window_end_ms set) for a feed; returns at once with *ticket. The caller keeps the
 * columns alive and unchanged until cvetl_server_wait on the ticket returns (host columns in
 * pinned memory are copied asynchronously). CVETL_EINVAL for a bad feed or input,
 * CVETL_EFULL when the window alone exceeds the budget, CVETL_ESTATE after the feed's flush. */
cvetl_status cvetl_server_submit(cvetl_server* s, int32_t feed, const cvetl_input* in, uint64_t* ticket);

/* Queues the end of a feed's stream (cvetl_flush): after it the feed takes no more windows. */
cvetl_status cvetl_server_submit_flush(cvetl_server* s, int32_t feed, uint64_t* ticket);

/* Waits for a ticket and releases it; *info (may be NULL) receives its record. Returns the
 * request's own status, or CVETL_EINVAL for an unknown ticket. */
cvetl_status cvetl_server_wait(cvetl_server* s, uint64_t ticket, cvetl_ticket_info* info);

/* Waits until no request is queued or running. */
cvetl_status cvetl_server_drain(cvetl_server* s);

/* The feed's context, for cvetl_results / cvetl_stats_get while the feed has no request queued
 * or running (CVETL_ESTATE otherwise); do not submit to the feed while using it. */
cvetl_status cvetl_server_feed(cvetl_server* s, int32_t feed, cvetl_ctx** ctx);

/* Runs what is running to completion, fails what is still queued with CVETL_ESTATE (their
 * tickets are dropped), joins the workers and destroys the feeds. NULL is accepted. */
cvetl_status cvetl_server_destroy(cvetl_server* s);

/* Last error text of a server call (not of a request: see cvetl_ticket_info.message). */
const char* cvetl_server_last_error(const cvetl_server* s);

/* Binary64 issue-rate probe (a measurement aid with no counterpart in the paper: the FP64 form
 * of the journey kernels runs part of its per-point arithmetic on the binary64 pipe, whose rate
 * this measures). Launches
 * `blocks` CTAs of `threads` (64, 128 or 256) threads on `stream`, each thread running 8
 * independent chains of `iters` iterations of one binary64 operation kind: 0 fma, 1 add,
 * 2 multiply, 3 a mix of 4 adds, 5 multiplies and 4 fma. sink: device
 * memory for blocks * threads doubles (caller-owned; receives the chains' sums). *ops (may be
 * NULL) receives the binary64 operations the launch performs. The call only enqueues: the
 * caller times it with events on the stream. CVETL_EINVAL on a bad argument, CVETL_ECUDA on a
 * launch error (text via cvetl_last_error(NULL)). */
cvetl_status cvetl_probe_fp64(int32_t kind, int32_t blocks, int32_t threads, int64_t iters, double* sink,
                              int64_t* ops, void* stream);

/* Allocation-free radix sort (the paper has no counterpart; it serves callers that may not
 * allocate device memory: code inside a host framework that owns the device memory pool and
 * forbids side allocations, and latency-critical loops where a cudaMalloc / cudaFree, which can
 * synchronise the device, would stall the work).
 * Stable sort of n 64-bit keys by bits [begin_bit, end_bit) (bits outside that range take no
 * part in the order): keys_out receives the keys, unchanged, in that order and perm_out[i] the
 * input position of the i-th key (keys equal in the range keep input order). All three arrays
 * are device memory owned by the caller; keys_out must not be keys_in. Work is queued on
 * `stream` (a cudaStream_t) and the call synchronises it before returning (it reads a device
 * error word back into host memory), so the call cannot be captured into a CUDA graph: on a
 * stream that is capturing it returns CVETL_ESTATE without touching the capture.
 * Scratch: a fixed device array of about 3 MB inside the library, one per device that loads
 * it, held until the process exits; the call allocates nothing (no cudaMalloc, no cudaFree).
 * The first call on each device looks up that array's device address and sets the kernel's
 * shared-memory limit (safe when several host threads make their first call at once).
 * Calls share the array and clear what must start at zero; calls that overlap on the GPU
 * (other streams, other threads) race on it, so serialise them.
 * Errors (text via cvetl_last_error(NULL)): CVETL_EINVAL when n is outside
 * [0, CVETL_NOALLOC_MAX_PAIRS], the bit range is not within [0, 64), an array is NULL or
 * keys_out == keys_in; CVETL_ESTATE when the stream is capturing; CVETL_ECUDA on a CUDA error;
 * CVETL_ETIMEOUT if a bounded device-side wait gave up (the outputs are then not valid). */
#define CVETL_NOALLOC_MAX_PAIRS 262144
cvetl_status cvetl_sort_u64_noalloc(const uint64_t* keys_in, uint64_t* keys_out, uint32_t* perm_out,
                                    int64_t n, int32_t begin_bit, int32_t end_bit, void* stream);

#ifdef __cplusplus
}
#endif
#endif
