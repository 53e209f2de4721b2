"""CUDA path against the CPU oracle, element by element, through the C ABI."""
import ctypes

import numpy as np
import pytest

import cvgen
from parity import close, compare, exact

pytestmark = pytest.mark.gpu

T0 = 1620518400000


def run_gpu(cols, device=True, materialize=True, tuning=None, **cfg):
    import torch

    import paper_2305_07454_b300 as P

    t = {k: torch.from_numpy(np.ascontiguousarray(cols[k])) for k in ("jid", "ts", "lat", "lon", "speed")}
    if device:
        t = {k: v.cuda() for k, v in t.items()}
    with P.Pipeline(materialize_points=int(materialize), **cfg) as p:
        if tuning:
            p.tuning = tuning
        return p.run(t)


def synth(sizes, seed, jids=None, dup_frac=0.0, t_start=T0 + 3_600_000):
    """Shuffled journeys of exactly the given sizes (test-local inputs, no method arithmetic)."""
    rng = np.random.default_rng(seed)
    parts = []
    for j, m in enumerate(sizes):
        jid = int(jids[j]) if jids is not None else int(rng.integers(0, 2 ** 40))
        dt = rng.integers(300, 1000, m)
        dt[0] = 0
        if dup_frac:
            dt[1:][rng.random(m - 1) < dup_frac] = 0
        ts = t_start + int(rng.integers(0, 3_600_000)) + np.cumsum(dt)
        lat = 38.0 + np.cumsum(rng.normal(0, 2e-5, m))
        lon = -92.0 + np.cumsum(rng.normal(0, 2e-5, m))
        spd = np.abs(rng.normal(40, 30, m)).astype(np.float32)
        spd[rng.random(m) < 0.05] = 0.0
        spd[rng.random(m) < 0.02] = -0.0
        if dup_frac:  # exact duplicates: copy the predecessor's values
            for i in np.flatnonzero(dt == 0)[1:] if m > 1 else []:
                lat[i], lon[i], spd[i] = lat[i - 1], lon[i - 1], spd[i - 1]
        parts.append(dict(jid=np.full(m, jid, np.int64), ts=ts.astype(np.int64), lat=lat, lon=lon, speed=spd))
    cols = {k: np.concatenate([p[k] for p in parts]) if parts else np.empty(0, t)
            for k, t in (("jid", np.int64), ("ts", np.int64), ("lat", np.float64), ("lon", np.float64),
                         ("speed", np.float32))}
    perm = rng.permutation(cols["jid"].shape[0])
    return {k: np.ascontiguousarray(v[perm]) for k, v in cols.items()}


def test_small_day(orc, small_day):
    compare(run_gpu(small_day), orc.run(small_day))


def test_fp64_form_distances_are_binary64_close(orc, small_day):
    """The FP64 form evaluates every term above 2^-22 relative in binary64 and only a sum of
    small corrections in float32 (a bound of about 1e-14 relative): per-point distances within
    1e-13 relative of the oracle's libm haversine, journey sums within 1e-12."""
    g, o = run_gpu(small_day), orc.run(small_day)
    close("point d", g["points"]["d"], o["points"]["d"], rel=1e-13, abs_=1e-12)
    close("journey distance", g["journeys"]["distance_m"], o["journeys"]["distance_m"], rel=1e-12)
    d_g, d_o = g["points"]["d"], o["points"]["d"]
    nz = d_o > 0
    print("max relative error of d:", float(np.max(np.abs(d_g[nz] - d_o[nz]) / d_o[nz])))


def test_small_day_host_input_matches(orc, small_day):
    a = run_gpu(small_day, device=False)
    compare(a, orc.run(small_day))


@pytest.mark.parametrize("seed", [2, 3])
def test_input_order_does_not_change_any_bit(small_day, seed):
    base = run_gpu(small_day)
    perm = np.random.default_rng(seed).permutation(small_day["jid"].shape[0])
    shuffled = {k: np.ascontiguousarray(v[perm]) for k, v in small_day.items()}
    got = run_gpu(shuffled)
    for part in ("cells", "journeys"):
        for k in base[part]:
            exact(f"{part} {k}", got[part][k], base[part][k])
    for k in ("d", "vhat", "accel", "dwell", "key", "flags"):
        exact("point " + k, got["points"][k], base["points"][k])
    # the sorted records are the same records in the same order; exact duplicates tie on
    # (journey, time) and follow input order, so their indices may trade places
    back = perm[got["points"]["perm"]]
    for k in small_day:
        exact("sorted " + k, small_day[k][back], small_day[k][base["points"]["perm"]])


def test_empty_input(orc):
    cols = synth([], 1)
    g = run_gpu(cols)
    assert g["counters"]["n_valid"] == 0 and g["counters"]["n_journeys"] == 0 and g["counters"]["n_cells"] == 0
    compare(g, orc.run(cols), points=False)


@pytest.mark.parametrize("sizes", [[1], [2], [255, 256, 257], [4095, 4096, 4097], [1, 8193, 3, 20000]])
def test_journey_sizes_around_tile_edges(orc, sizes):
    cols = synth(sizes, seed=sum(sizes), dup_frac=0.01)
    compare(run_gpu(cols), orc.run(cols))


@pytest.mark.parametrize("n_journeys", [1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097])
def test_journey_counts_around_the_block_sort_limit(orc, n_journeys):
    """Up to 4096 pairs take the one-block sort (its default limit; 256 threads up to 1024 pairs,
    1024 threads above), more the device-wide radix sort (journey ids and, with about one run per
    journey, the runs)."""
    rng = np.random.default_rng(n_journeys)
    cols = synth(list(rng.integers(1, 4, n_journeys)), seed=n_journeys)
    compare(run_gpu(cols), orc.run(cols))


def test_one_long_journey_many_chunks(orc):
    cols = synth([70001], seed=9, dup_frac=0.003)
    compare(run_gpu(cols), orc.run(cols))


SHORT_SIZES = [1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513, 4097]


@pytest.mark.parametrize("split", [0, 128, 512])
@pytest.mark.parametrize("dup_frac", [0.01, 0.6])
def test_short_journeys_in_64_thread_ctas(orc, split, dup_frac):
    """Journeys of up to `split` points take the 64-thread journey kernel, the rest the
    256-thread one; sizes around the 64-thread walk's ranges and the shape limits, and, at
    dup_frac 0.6, time buckets crowded past the bucket sort's limit (the 64-thread kernel then
    sorts (timestamp, row) pairs)."""
    cols = synth(SHORT_SIZES * 3, seed=17 + split, dup_frac=dup_frac)
    compare(run_gpu(cols, tuning=dict(small_journey_max=split)), orc.run(cols))


SORT_EDGES = [512, 513, 2048, 2049, 4096, 4097, 6143, 8192, 8193, 16384, 30001]


@pytest.mark.parametrize("dup_frac", [0.01, 0.6])
def test_journey_sort_size_classes(orc, dup_frac):
    """The batch path takes each journey by size class: up to 512, 4096 and 8192 points sorted
    with the timestamps held in shared memory and then walked one warp per journey, larger ones by
    the fused journey kernel; journeys on either side of every class edge, and at dup_frac 0.6 with
    time buckets crowded past the staged sort's limit (each class then falls back to the general
    sort)."""
    cols = synth(SORT_EDGES, seed=31 + int(dup_frac * 10), dup_frac=dup_frac)
    compare(run_gpu(cols), orc.run(cols))


def test_long_journeys_with_long_runs(orc):
    """Journeys above 8192 points (the fused kernel: each of 256 threads walks a contiguous range
    of the sorted points and the run fragments are stitched across ranges), with stretches that
    cross many ranges: a parked vehicle (one cell and bin for 5,000 points: a run spanning whole
    ranges), an off-grid stretch (invalid keys across ranges) and exact duplicates; both forms,
    with and without the per-point columns."""
    rng = np.random.default_rng(41)
    sizes = [8193, 10240, 10241, 12288, 20000, 45000]
    parts = []
    for j, m in enumerate(sizes):
        dt = rng.integers(300, 1000, m)
        dt[0] = 0
        dt[1:][rng.random(m - 1) < 0.01] = 0
        ts = T0 + 3_600_000 + int(rng.integers(0, 3_600_000)) + np.cumsum(dt)
        lat = 38.0 + np.cumsum(rng.normal(0, 2e-5, m))
        lon = -92.0 + np.cumsum(rng.normal(0, 2e-5, m))
        a, b = m // 5, m // 5 + 5000  # parked
        lat[a:b], lon[a:b] = lat[a], lon[a]
        c, d = (3 * m) // 5, (3 * m) // 5 + 3000  # off the grid (north of the box)
        lat[c:d] += 5.0
        spd = np.abs(rng.normal(40, 30, m)).astype(np.float32)
        spd[a:b] = 0.0
        parts.append(dict(jid=np.full(m, 7000 + j, np.int64), ts=ts.astype(np.int64), lat=lat, lon=lon, speed=spd))
    cols = {k: np.concatenate([q[k] for q in parts]) for k in parts[0]}
    perm = rng.permutation(cols["jid"].shape[0])
    cols = {k: np.ascontiguousarray(v[perm]) for k, v in cols.items()}
    o = orc.run(cols)
    compare(run_gpu(cols), o)
    import paper_2305_07454_b300 as P

    compare(run_gpu(cols, precision=P.FP32), o, rel=1e-4)  # the float32 form
    # without the per-point columns (the bench's configuration)
    compare(run_gpu(cols, materialize=False), o, points=False)


def test_very_long_journeys(orc):
    """Journeys of 120,000, 150,001 (40% exact duplicates) and 400,001 points: above the
    time-bucket sort's limit of 98,304 points, each is sorted by one CTA's radix sort through
    global scratch, its keys holding 17-19 position bits."""
    cols = synth([120000, 400001], seed=43)
    o = orc.run(cols)
    compare(run_gpu(cols, materialize=False), o, points=False)
    dup = synth([150001], seed=44, dup_frac=0.4)
    compare(run_gpu(dup, materialize=False), orc.run(dup), points=False)


def test_timestamps_spanning_the_int64_range(orc):
    """Timestamps spread over the whole int64 range: the sort keys (time offset and bucket
    position) no longer fit 64 bits and every journey is sorted as (timestamp, row) pairs, in both
    kernel shapes (steps of about 2^60 ms; every point falls outside the day's bins)."""
    rng = np.random.default_rng(23)
    sizes = [3, 60, 200, 511, 900, 5000]
    cols = synth(sizes, seed=23)
    ts = rng.integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, cols["ts"].shape[0], dtype=np.int64)
    ts[:2] = [np.iinfo(np.int64).min, np.iinfo(np.int64).max]
    cols["ts"] = ts
    o = orc.run(cols)
    for split in (0, 512):
        compare(run_gpu(cols, tuning=dict(small_journey_max=split)), o)


def test_duplicate_heavy_ties_follow_input_order(orc):
    cols = synth([300, 5000], seed=5, dup_frac=0.5)
    compare(run_gpu(cols), orc.run(cols))


def test_sentinel_like_ids_and_full_int64_range(orc):
    ids = [-1, -(2 ** 63), 2 ** 63 - 1, 0, 1, -2]
    cols = synth([10, 20, 30, 40, 50, 60], seed=4, jids=ids)
    compare(run_gpu(cols), orc.run(cols))
    wide = cvgen.generate(cvgen.params("small_day", seed=4, n_journeys=300, jid_mode=1))
    compare(run_gpu(wide), orc.run(wide))


def test_malformed_offgrid_and_negative_zero(orc):
    cols = synth([500, 700], seed=6)
    n = cols["jid"].shape[0]
    rng = np.random.default_rng(0)
    i = rng.choice(n, 60, replace=False)
    cols["lat"][i[:10]] = np.nan
    cols["lon"][i[10:20]] = np.inf
    cols["lat"][i[20:25]] = 90.0000001
    cols["lon"][i[25:30]] = -180.5
    cols["speed"][i[30:35]] = np.nan
    cols["lat"][i[35:40]] = 35.5          # below the grid
    cols["lon"][i[40:45]] = -89.0999999   # just east of the grid
    cols["ts"][i[45:50]] = T0 - 5        # before the day
    cols["ts"][i[50:55]] = T0 + 86_400_000  # after the last bin
    cols["speed"][i[55:60]] = -0.0
    o = orc.run(cols)
    assert o["counters"]["n_malformed"] == 35 and o["counters"]["n_out_of_grid"] >= 20
    compare(run_gpu(cols), o)


def test_cell_edges_exactly(orc):
    """Points placed exactly on 0.01 deg edges: the binary64 quotient decides the side."""
    k = np.arange(0, 460)
    lat = 36.0 + k * 0.01
    lon = np.full_like(lat, -95.8 + 0.37)
    n = lat.shape[0]
    cols = dict(jid=np.arange(n, dtype=np.int64), ts=np.full(n, T0 + 1000, np.int64), lat=lat,
                lon=lon, speed=np.ones(n, np.float32))
    compare(run_gpu(cols), orc.run(cols))


@pytest.mark.parametrize("bin_ms,n_bins", [(1, 13000), (7, 9000), (1000, 7200), (60000, 1440),
                                            (2 ** 31 - 1, 2), (2 ** 32 + 5, 1)])
def test_time_bins_of_any_width(orc, bin_ms, n_bins):
    """Algorithm 2's time bin, floor((ts - t0) / bin_ms), for bin widths from 1 ms to past 2^32
    ms: spans below 2^32 take the multiply-high division, wider ones the 64-bit division."""
    import oracle

    cols = synth([300, 1000, 37, 5000], seed=11)
    cfg = dict(bin_ms=bin_ms, n_bins=n_bins, t0_ms=int(cols["ts"].min()) - 5)
    compare(run_gpu(cols, **cfg), orc.run(cols, oracle.default_params(**cfg)))


def test_aggregates_only_mode_matches(orc, small_day):
    g = run_gpu(small_day, materialize=False)
    assert "points" not in g
    compare(g, orc.run(small_day), points=False)


def test_call_order_and_budget_errors(small_day):
    import torch

    import paper_2305_07454_b300 as P

    with P.Pipeline() as p:
        with pytest.raises(P.CvetlError) as e:
            p.transform()
        assert e.value.status == P.ESTATE
        with pytest.raises(P.CvetlError) as e:
            p.load()
        assert e.value.status == P.ESTATE
    with P.Pipeline(mem_budget_bytes=1 << 20) as p:
        t = {k: torch.from_numpy(np.ascontiguousarray(small_day[k])).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
        p.extract(t)
        with pytest.raises(P.CvetlError) as e:
            p.transform()
        assert e.value.status == P.EFULL


def test_stats_count_launches(small_day):
    import torch

    import paper_2305_07454_b300 as P

    t = {k: torch.from_numpy(np.ascontiguousarray(small_day[k])).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
    with P.Pipeline(profile=1) as p:
        p.run(t, to_host=False)
        s = p.stats()
    assert s["total_launches"] > 10
    # journeys above 8192 points: the fused journey kernel; the rest: the size-class bounds and one
    # persistent sort launch per size class, then the walk
    assert s["stages"]["journeys"]["launches"] == 1
    assert s["stages"]["journey_sort"]["launches"] == 4 and s["stages"]["journey_sort"]["ms"] > 0
    assert s["stages"]["journey_walk"]["launches"] == 1 and s["stages"]["journey_walk"]["ms"] > 0


def test_results_into_pinned_buffers(small_day):
    """results(out=...) fills pinned host buffers with the same tables as the plain host copy,
    and buffers smaller than a table grow."""
    import torch

    import paper_2305_07454_b300 as P

    t = {k: torch.from_numpy(np.ascontiguousarray(small_day[k])).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
    with P.Pipeline(materialize_points=1) as p:
        p.run(t, to_host=False)
        a = p.results(to_host=True)
        host = p.host_tables(cells=1, journeys=1, points=1)
        b = p.results(to_host=True, out=host)
        assert b["cells"]["key"].shape == a["cells"]["key"].shape
        for part in ("cells", "journeys", "points"):
            for k in a[part]:
                exact(part + " " + k, b[part][k], a[part][k])
        assert b["counters"] == a["counters"]
