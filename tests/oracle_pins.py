"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each ``pin_*`` function raises AssertionError on a violation. They are collected by
``test_oracle_pins.py`` and re-run against deliberately broken copies of the oracle by
``test_oracle_mutants.py``, to show that a plausible mistake anywhere in the oracle fails
at least one of them. None of them re-types the oracle's formulas: they use closed forms,
an independent great-circle formula, exact integer arithmetic, CPython's correctly rounded
float parser, numpy library routines and brute force on tiny inputs.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import numpy as np

R = 6371000.0
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def vincenty_sphere_m(lat1, lon1, lat2, lon2, radius=R):
    """Great-circle distance by the atan2 (Vincenty, sphere) formula: independent of the
    haversine form and well conditioned for every separation."""
    p1, p2 = np.radians(lat1), np.radians(lat2)
    dl = np.radians(lon2 - lon1)
    num = np.hypot(np.cos(p2) * np.sin(dl),
                   np.cos(p1) * np.sin(p2) - np.sin(p1) * np.cos(p2) * np.cos(dl))
    den = np.sin(p1) * np.sin(p2) + np.cos(p1) * np.cos(p2) * np.cos(dl)
    return radius * np.arctan2(num, den)


# ---------------------------------------------------------------- haversine
def pin_haversine_closed_forms(o):
    rng = np.random.default_rng(11)
    # along a meridian: d = R |dphi|
    for _ in range(200):
        a, b = rng.uniform(-89.0, 89.0, 2)
        lon = rng.uniform(-180, 180)
        want = R * abs(math.radians(b) - math.radians(a))
        got = o.haversine_m(a, lon, b, lon, R)
        assert _rel(got, want) < 1e-11 or abs(got - want) < 1e-6, (a, b, got, want)
    # along the equator: d = R |dlambda| for |dlambda| <= 180 deg
    for _ in range(200):
        a, b = rng.uniform(-90.0, 90.0, 2)
        want = R * abs(math.radians(b) - math.radians(a))
        got = o.haversine_m(0.0, a, 0.0, b, R)
        assert _rel(got, want) < 1e-11 or abs(got - want) < 1e-6, (a, b, got, want)
    # identity, symmetry, antipodes, one degree of latitude
    for _ in range(100):
        la, lo, lb, lob = rng.uniform(-80, 80), rng.uniform(-170, 170), rng.uniform(-80, 80), rng.uniform(-170, 170)
        assert o.haversine_m(la, lo, la, lo, R) == 0.0
        assert _rel(o.haversine_m(la, lo, lb, lob, R), o.haversine_m(lb, lob, la, lo, R)) < 1e-15
    assert _rel(o.haversine_m(0.0, 0.0, 0.0, 180.0, R), math.pi * R) < 1e-15
    assert _rel(o.haversine_m(30.0, 10.0, -30.0, -170.0, R), math.pi * R) < 1e-12
    assert round(o.haversine_m(37.0, -92.0, 38.0, -92.0, R), 2) == 111194.93
    # against the independent atan2 form, at mid latitudes, steps from 10 m to 200 km
    lat1 = rng.uniform(36.0, 40.6, 2000)
    lon1 = rng.uniform(-95.8, -89.1, 2000)
    step = 10.0 ** rng.uniform(-4, 0.3, 2000)
    ang = rng.uniform(0, 2 * math.pi, 2000)
    lat2 = lat1 + step * np.cos(ang)
    lon2 = lon1 + step * np.sin(ang)
    want = vincenty_sphere_m(lat1, lon1, lat2, lon2)
    for i in range(2000):
        got = o.haversine_m(lat1[i], lon1[i], lat2[i], lon2[i], R)
        assert _rel(got, want[i]) < 1e-8, (i, got, want[i])


# ---------------------------------------------------------------- keys
def pin_grid_index(o):
    # exact rational floor for 6-decimal latitudes m / 1e6 away from cell edges
    rng = np.random.default_rng(12)
    m = rng.integers(35_500_000, 41_000_000, 20000)
    for mi in m:
        x = mi / 1e6
        num = int(mi) - 36_000_000  # (x - 36) in micro-degrees
        k, rem = divmod(num, 10_000)
        got = o.grid_index(x, 36.0, 0.01, 460)
        exp = k if 0 <= k < 460 else -1
        if rem == 0:  # exactly on an edge: either side is a correct rounding
            assert got in (exp, k - 1 if 0 <= k - 1 < 460 else -1), (x, got, exp)
        else:
            assert got == exp, (x, got, exp)
    # longitudes likewise (negative coordinates)
    m = rng.integers(-96_000_000, -89_000_000, 20000)
    for mi in m:
        x = mi / 1e6
        num = int(mi) + 95_800_000
        k, rem = divmod(num, 10_000)
        got = o.grid_index(x, -95.8, 0.01, 670)
        exp = k if 0 <= k < 670 else -1
        if rem == 0:
            assert got in (exp, k - 1 if 0 <= k - 1 < 670 else -1), (x, got, exp)
        else:
            assert got == exp, (x, got, exp)
    # monotone across edges, at consecutive doubles
    for k in (1, 57, 166, 459):
        x = 36.0 + k * 0.01
        xs = [x]
        for _ in range(8):
            xs.insert(0, np.nextafter(xs[0], -np.inf))
            xs.append(np.nextafter(xs[-1], np.inf))
        idx = [o.grid_index(v, 36.0, 0.01, 460) for v in xs]
        assert idx == sorted(idx) and idx[0] == k - 1 and idx[-1] == k, (k, idx)
    # out of range and non-finite
    assert o.grid_index(35.999999, 36.0, 0.01, 460) == -1
    assert o.grid_index(36.0, 36.0, 0.01, 460) == 0
    assert o.grid_index(40.61, 36.0, 0.01, 460) == -1
    assert o.grid_index(40.6 + 1e-9, 36.0, 0.01, 460) == -1
    assert o.grid_index(40.599999, 36.0, 0.01, 460) == 459
    for bad in (float("nan"), float("inf"), -float("inf")):
        assert o.grid_index(bad, 36.0, 0.01, 460) == -1


def pin_time_bin(o):
    t0, w, nb = 1620518400000, 60000, 1440
    rng = np.random.default_rng(13)
    offs = list(rng.integers(-3 * 86400000, 3 * 86400000, 5000)) + [-1, 0, 59999, 60000, 86399999, 86400000, -60000, -60001]
    for off in offs:
        ts = t0 + int(off)
        q = (ts - t0) // w  # Python integer floor division
        exp = q if 0 <= q < nb else -1
        assert o.time_bin(ts, t0, w, nb) == exp, (off, exp)
    assert o.time_bin(-(2 ** 63), t0, w, nb) == -1
    assert o.time_bin(2 ** 63 - 1, t0, w, nb) == -1


# ---------------------------------------------------------------- extract
def pin_parse_fields(o):
    rng = np.random.default_rng(14)
    for _ in range(3000):
        nd = int(rng.integers(1, 16))
        ni = int(rng.integers(1, nd + 1))
        digits = "".join(str(d) for d in rng.integers(0, 10, nd))
        s = digits[:ni] + ("." + digits[ni:] if ni < nd else "")
        if rng.random() < 0.5:
            s = "-" + s
        got = o.parse_decimal(s)
        assert got is not None and got == float(s), (s, got)  # CPython's correctly rounded parse
    for good in ("0", "-0", "0.0", "007.5", "123456789012345", "1.23456789012345", "-90.000000"):
        assert o.parse_decimal(good) == float(good), good
    for bad in ("", "-", "1.", ".5", "+1", "1e5", "nan", "inf", " 1", "1 ", "1.2.3", "--1",
                "1234567890123456", "1.234567890123456", "12a4", "0x10", "1,0"):
        assert o.parse_decimal(bad) is None, bad
    for good, v in (("0", 0), ("-12", -12), ("123456789012345678", 123456789012345678), ("0001", 1)):
        assert o.parse_integer(good) == v, good
    for bad in ("", "-", "1234567890123456789", "1.0", "+5", "1e3", " 7"):
        assert o.parse_integer(bad) is None, bad


def pin_table1(o):
    with open(os.path.join(GOLDEN, "table1_expected.json")) as f:
        exp = json.load(f)
    with open(os.path.join(GOLDEN, "table1.csv"), "rb") as f:
        buf = f.read()
    cols, nl, nm = o.parse_csv(buf)
    assert nl == exp["n_lines"] and nm == exp["n_malformed"]
    r = o.run(cols)
    assert list(r["points"]["perm"]) == exp["perm"]
    assert list(r["points"]["flags"]) == exp["flags"]
    for k, v in exp["journeys"].items():
        assert list(r["journeys"][k]) == v, k
    for k in ("key", "row", "col", "bin", "count"):
        assert list(r["cells"][k]) == exp["cells"][k], k
    spd = np.array([np.float32(float(s)) for s in exp["cells"]["speed_decimal"]], np.float32)
    assert np.array_equal(r["cells"]["min"], spd) and np.array_equal(r["cells"]["max"], spd)
    assert np.array_equal(r["cells"]["sum"], spd.astype(np.float64) * np.array(exp["cells"]["count"]))


def pin_csv_roundtrip(o, cols):
    import cvgen

    buf, injected = cvgen.to_csv(cols, seed=5, malformed_frac=0.01)
    got, nl, nm = o.parse_csv(buf)
    n = cols["jid"].shape[0]
    assert nl == n and nm == injected and got["jid"].shape[0] == n
    # every line is a row; the malformed ones carry no position
    bad = np.isnan(got["lat"])
    assert int(bad.sum()) == injected and np.all(np.isnan(got["lon"][bad])) and np.all(got["jid"][bad] == 0)
    got = {k: v[~bad] for k, v in got.items()}
    # kept rows are the generator's rows, in file order, rounded to their printed precision
    cj, ct, gj, gt = cols["jid"].tolist(), cols["ts"].tolist(), got["jid"].tolist(), got["ts"].tolist()
    src = np.empty(len(gj), np.int64)
    i = 0
    for k in range(len(gj)):
        while not (cj[i] == gj[k] and ct[i] == gt[k]):
            i += 1
        src[k] = i
        i += 1
    assert np.all(np.abs(cols["lat"][src] - got["lat"]) <= 5.0000001e-7)
    assert np.all(np.abs(cols["lon"][src] - got["lon"]) <= 5.0000001e-7)
    assert np.all(np.abs(cols["speed"][src] - got["speed"]) <= 0.0051)


# ---------------------------------------------------------------- whole path
def pin_invariants(o, cols):
    r = o.run(cols)
    c, p, j, cl = r["counters"], r["points"], r["journeys"], r["cells"]
    n = cols["jid"].shape[0]
    nv = c["n_valid"]
    assert c["n_in"] == n and nv + c["n_malformed"] == n
    # conservation
    assert int(cl["count"].sum()) + c["n_out_of_grid"] == nv
    assert int(j["n"].sum()) == nv
    assert int(np.count_nonzero(p["key"] == 0xFFFFFFFF)) == c["n_out_of_grid"]
    # permutation is a bijection onto the valid records
    perm = p["perm"].astype(np.int64)
    assert np.unique(perm).shape[0] == nv
    # sortedness and stability
    sj, st = cols["jid"][perm], cols["ts"][perm]
    assert np.all((sj[1:] > sj[:-1]) | ((sj[1:] == sj[:-1]) & (st[1:] > st[:-1])) |
                  ((sj[1:] == sj[:-1]) & (st[1:] == st[:-1]) & (perm[1:] > perm[:-1])))
    assert np.all(np.diff(j["jid"]) > 0)
    # journey starts, durations, dwell
    starts = np.flatnonzero(p["flags"] & 1)
    assert np.array_equal(sj[starts], j["jid"])
    bounds = np.append(starts, nv)
    dt = np.diff(st)
    for k in range(0, len(starts), max(1, len(starts) // 200)):
        a, b = bounds[k], bounds[k + 1]
        assert j["duration_ms"][k] == int(dt[a:b - 1].sum()) == j["end_ts"][k] - j["start_ts"][k]
        assert 0 <= j["dwell_ms"][k] <= j["duration_ms"][k]
    # flags agree with the data
    dup = np.zeros(nv, bool)
    dup[1:] = (sj[1:] == sj[:-1]) & (st[1:] == st[:-1])
    assert np.array_equal((p["flags"] & 2) != 0, dup) and c["n_dup"] == int(dup.sum())
    # cell aggregates
    assert np.all(np.diff(cl["key"].astype(np.int64)) > 0)
    assert np.all(cl["min"] <= cl["mean"] + 1e-9) and np.all(cl["mean"] <= cl["max"] + 1e-9)
    assert np.all(cl["key"] == (cl["bin"].astype(np.int64) * 460 + cl["row"]) * 670 + cl["col"])


def pin_library_cross_check(o, cols):
    """numpy.lexsort for the order; numpy grouping for count / sum / min / max."""
    r = o.run(cols)
    p, cl = r["points"], r["cells"]
    n = cols["jid"].shape[0]
    idx = np.arange(n)
    valid = np.isfinite(cols["lat"]) & np.isfinite(cols["lon"]) & np.isfinite(cols["speed"])
    order = np.lexsort((idx[valid], cols["ts"][valid], cols["jid"][valid]))
    assert np.array_equal(idx[valid][order], p["perm"].astype(np.int64))
    keys = p["key"]
    spd = cols["speed"][p["perm"]].astype(np.float32)
    spd = np.where(spd == 0, np.float32(0), spd)
    ok = keys != 0xFFFFFFFF
    kk, ss = keys[ok], spd[ok]
    o2 = np.argsort(kk, kind="stable")
    kk, ss = kk[o2], ss[o2]
    uk, first, cnt = np.unique(kk, return_index=True, return_counts=True)
    assert np.array_equal(uk, cl["key"]) and np.array_equal(cnt, cl["count"])
    assert np.array_equal(np.minimum.reduceat(ss, first), cl["min"])
    assert np.array_equal(np.maximum.reduceat(ss, first), cl["max"])
    sums = np.add.reduceat(ss.astype(np.float64), first)
    assert np.all(np.abs(sums - cl["sum"]) <= 1e-12 * np.abs(sums) + 1e-9)
    # unique journeys per key: distinct (key, journey) pairs counted per key
    jj = cols["jid"][p["perm"]][ok][o2]
    pairs = np.unique(np.stack([kk.astype(np.int64), jj]), axis=1)
    uk2, vol = np.unique(pairs[0], return_counts=True)
    assert np.array_equal(uk2, cl["key"].astype(np.int64)) and np.array_equal(vol, cl["volume"])
    assert (cl["volume"] <= cl["count"]).all()
    # journey table from the same lexsort: each journey's first and last record in (time, row)
    # order give its start and end time and position (latitude and longitude both move along
    # the generated journeys, so a swapped or misplaced coordinate shows)
    j = r["journeys"]
    sj = cols["jid"][valid][order]
    head = np.flatnonzero(np.concatenate([[True], sj[1:] != sj[:-1]]))
    tail = np.append(head[1:], sj.shape[0]) - 1
    assert np.array_equal(j["jid"], sj[head]) and np.array_equal(j["n"], tail - head + 1)
    for name, src in (("ts", cols["ts"]), ("lat", cols["lat"]), ("lon", cols["lon"])):
        s = src[valid][order]
        assert np.array_equal(j["start_" + name], s[head]), name
        assert np.array_equal(j["end_" + name], s[tail]), name
    moved = j["start_lon"] != j["end_lon"]
    assert moved.mean() > 0.5  # the check above sees longitude move in most journeys


def _independent_groups(cols):
    """Grouping with plain Python containers: journeys as lists sorted by (ts, index)."""
    groups = {}
    for i in range(len(cols["jid"])):
        groups.setdefault(int(cols["jid"][i]), []).append((int(cols["ts"][i]), i, float(cols["speed"][i])))
    for v in groups.values():
        v.sort()
    return groups


def pin_bruteforce_orders(o):
    base = dict(
        jid=np.array([7, 3, 7, 3, 7, 9, 7], np.int64),
        ts=np.array([1620520000500, 1620520000000, 1620520000000, 1620520000900, 1620520000500, 1620519999000, 1620520061000], np.int64),
        lat=np.array([37.00001, 38.5, 37.0, 38.5003, 37.00001, 40.61, 37.01], np.float64),
        lon=np.array([-92.0, -91.0, -92.0, -91.0004, -92.0, -90.0, -92.0], np.float64),
        speed=np.array([0.5, 40.0, 0.0, 41.0, 0.5, 10.0, 60.0], np.float32),
    )
    n = 7
    ref = None
    groups = _independent_groups(base)
    for perm in itertools.permutations(range(n)):
        perm = np.array(perm)
        cols = {k: v[perm] for k, v in base.items()}
        r = o.run(cols)
        back = perm[r["points"]["perm"]]
        sig = (tuple(back), tuple(r["points"]["flags"]), tuple(r["points"]["key"]),
               tuple(np.round(r["points"]["d"], 9)), tuple(r["points"]["dwell"]),
               tuple(r["journeys"]["n"]), tuple(r["journeys"]["duration_ms"]),
               tuple(r["cells"]["key"]), tuple(r["cells"]["count"]),
               tuple(np.round(r["cells"]["sum"], 9)))
        if ref is None:
            ref = sig
            # independent grouping: journey sizes, durations and order
            assert list(r["journeys"]["jid"]) == sorted(groups)
            assert list(r["journeys"]["n"]) == [len(groups[k]) for k in sorted(groups)]
            assert list(r["journeys"]["duration_ms"]) == [groups[k][-1][0] - groups[k][0][0] for k in sorted(groups)]
        else:
            # identical outputs for every input order (the two identical records of journey
            # 7 keep their input order, so they map to different base indices; every value
            # is equal)
            assert sig[1:] == ref[1:]


def pin_kinematics_hand(o):
    t = 1620532122000
    # one journey on a meridian: 0.001 deg steps every 500 ms, a stop, a duplicate, a 1 ms step
    cols = dict(
        jid=np.array([5, 5, 5, 5, 5, 5], np.int64),
        ts=np.array([t, t + 500, t + 1000, t + 1000, t + 3000, t + 3001], np.int64),
        lat=np.array([37.0, 37.001, 37.002, 37.002, 37.002, 37.002], np.float64),
        lon=np.array([-92.5, -92.5, -92.5, -92.5, -92.5, -92.5], np.float64),
        speed=np.array([30.0, 36.0, 0.5, 0.5, 0.25, 50.0], np.float32),
    )
    r = o.run(cols)
    p, j = r["points"], r["journeys"]
    step = R * math.radians(0.001)
    assert abs(p["d"][1] - step) < 1e-6 and abs(p["d"][2] - step) < 1e-6
    assert p["d"][0] == 0 and p["d"][3] == 0 and p["d"][4] == 0 and p["d"][5] == 0
    assert abs(p["vhat"][1] - step / 0.5 * 3.6) < 1e-6
    assert abs(p["accel"][1] - (6.0 / 3.6) / 0.5) < 1e-9
    assert abs(p["accel"][2] - ((0.5 - 36.0) / 3.6) / 0.5) < 1e-9
    assert p["accel"][3] == 0 and p["vhat"][3] == 0  # duplicate: dt = 0
    assert abs(p["accel"][4] - ((0.25 - 0.5) / 3.6) / 2.0) < 1e-9
    assert abs(p["accel"][5] - ((50.0 - 0.25) / 3.6) / 0.001) < 1e-6
    assert list(p["flags"]) == [1, 0, 0, 2 | 8, 8, 0]
    assert list(p["dwell"]) == [0, 0, 0, 0, 2000, 0]
    assert j["n"][0] == 6 and j["duration_ms"][0] == 3001 and j["dwell_ms"][0] == 2000
    assert abs(j["distance_m"][0] - 2 * step) < 1e-6
    assert j["start_lat"][0] == 37.0 and j["end_lat"][0] == 37.002
    # a -0.0 speed is +0.0 in the aggregates
    cols2 = dict(jid=np.array([1], np.int64), ts=np.array([t], np.int64), lat=np.array([37.5]),
                 lon=np.array([-92.5]), speed=np.array([-0.0], np.float32))
    r2 = o.run(cols2)
    assert r2["cells"]["min"][0] == 0 and not np.signbit(r2["cells"]["min"][0])


def pin_invalid_records(o):
    t = 1620532122000
    cols = dict(
        jid=np.array([1, 1, 1, 1, 1, 1], np.int64),
        ts=np.array([t, t + 1, t + 2, t + 3, t + 4, t + 5], np.int64),
        lat=np.array([37.0, np.nan, 91.0, 37.0, 37.0, 35.0], np.float64),
        lon=np.array([-92.0, -92.0, -92.0, np.inf, -181.0, -92.0], np.float64),
        speed=np.array([1, 2, 3, 4, 5, np.nan], np.float32),
    )
    r = o.run(cols)
    assert r["counters"]["n_malformed"] == 5 and r["counters"]["n_valid"] == 1
    assert list(r["points"]["perm"]) == [0]
    cols["speed"][5] = 6.0
    r = o.run(cols)
    assert r["counters"]["n_valid"] == 2 and r["counters"]["n_out_of_grid"] == 1  # lat 35.0


# ---- lattice (8 channels: mean speed and unique journeys in four directions) ----------
T0 = 1620518400000


def pin_direction_sectors(o):
    """Cardinal reading: within 45 deg of north is N (0), then E, S, W clockwise; the printed
    heading // 90 (quadrant reading) starts each sector at a multiple of 90 deg."""
    card = {0.0: 0, 44.9: 0, 45.0: 1, 90.0: 1, 134.9: 1, 135.0: 2, 180.0: 2, 224.9: 2, 225.0: 3,
            270.0: 3, 314.9: 3, 315.0: 0, 359.9: 0, 360.0: 0, -10.0: 0, -45.0: 0, -45.1: 3, 405.0: 1}
    for h, d in card.items():
        assert o.direction(h, 0) == d, ("cardinal", h, o.direction(h, 0), d)
    quad = {0.0: 0, 89.9: 0, 90.0: 1, 179.9: 1, 180.0: 2, 270.0: 3, 359.9: 3, -0.5: 3, 360.0: 0}
    for h, d in quad.items():
        assert o.direction(h, 1) == d, ("quadrant", h, o.direction(h, 1), d)
    assert o.direction(float("nan"), 0) == -1 and o.direction(float("inf"), 1) == -1


def _lattice_case(seed=7):
    """Points at cell centres with known (bin, direction, row, col): several journeys share
    cells, journeys re-enter a cell within a bin, some points have no heading or fall outside
    the bins. Returns the columns and the expected groups built from the construction."""
    rng = np.random.default_rng(seed)
    rows, cols_, bins = 460, 670, 288
    heads = [0.0, 90.0, 180.0, 270.0]  # sector centres: directions 0..3
    recs, expect = [], {}
    idx = 0
    for j in range(40):
        jid = int(rng.integers(0, 2 ** 31))
        for _ in range(int(rng.integers(1, 30))):
            b, d = int(rng.integers(0, 3)), int(rng.integers(0, 4))
            r, c = int(rng.integers(100, 103)), int(rng.integers(200, 202))
            ts = T0 + b * 300000 + int(rng.integers(0, 300000))
            lat, lon = 36.0 + 0.01 * r + 0.005, -95.8 + 0.01 * c + 0.005
            spd = float(np.float32(rng.uniform(0, 120)))
            kind = rng.random()
            h = heads[d] if kind > 0.1 else float("nan")
            if kind < 0.05:
                ts = T0 + bins * 300000 + 1  # after the lattice's last bin
            recs.append((jid, ts, lat, lon, spd, h))
            if kind > 0.1:
                key = ((b * 4 + d) * rows + r) * cols_ + c
                expect.setdefault(key, []).append((jid, idx, spd))
            idx += 1
    order = rng.permutation(len(recs))
    recs = [recs[i] for i in order]
    pos = {int(old): new for new, old in enumerate(order)}
    for key in expect:
        expect[key] = [(jid, pos[i], spd) for jid, i, spd in expect[key]]
    cols = {"jid": np.array([r[0] for r in recs], np.int64), "ts": np.array([r[1] for r in recs], np.int64),
            "lat": np.array([r[2] for r in recs]), "lon": np.array([r[3] for r in recs]),
            "speed": np.array([r[4] for r in recs], np.float32), "heading": np.array([r[5] for r in recs], np.float32)}
    return cols, expect


def pin_lattice_bruteforce(o):
    """Per (bin, direction, cell): point count, speed sum (in journey, input order), mean,
    unique journeys; per channel min-max normalisation over the occupied cells."""
    cols, expect = _lattice_case()
    L = o.lattice(cols)
    c = L["cells"]
    keys = sorted(expect)
    assert list(c["key"]) == keys
    n_kept = sum(len(v) for v in expect.values())
    assert int(c["count"].sum()) == n_kept and L["n_dropped"] == len(cols["jid"]) - n_kept
    mean, vol = [], []
    for q, key in enumerate(keys):
        pts = sorted(expect[key], key=lambda t: (t[0], t[1]))
        s = 0.0
        for _, _, spd in pts:
            s += spd
        assert c["count"][q] == len(pts) and c["sum"][q] == s
        assert c["volume"][q] == len({t[0] for t in pts})
        assert c["mean"][q] == np.float32(s / len(pts))
        assert c["dxn"][q] == (key // (460 * 670)) % 4
        mean.append(np.float32(s / len(pts)))
        vol.append(np.float32(len({t[0] for t in pts})))
    assert max(vol) > 1  # journeys share cells
    for ch in range(8):
        sel = [q for q, key in enumerate(keys) if (key // (460 * 670)) % 4 == ch // 2]
        v = [(mean if ch % 2 == 0 else vol)[q] for q in sel]
        mn, mx = (min(v), max(v)) if v else (np.float32(0), np.float32(0))
        assert L["ch_min"][ch] == mn and L["ch_max"][ch] == mx, (ch, L["ch_min"][ch], mn, L["ch_max"][ch], mx)
        out = c["mean_norm" if ch % 2 == 0 else "volume_norm"]
        for q, x in zip(sel, v):
            want = np.float32((x - mn) / (mx - mn)) if mx > mn else np.float32(0)
            assert out[q] == want


def pin_lattice_invariants(o):
    """On a generated day: conservation, volume <= count, means inside [min, max] of the
    speeds, normalised channels inside [0, 1] and reaching both ends."""
    import cvgen

    cols = cvgen.generate(cvgen.params("small_day", seed=5, n_journeys=400))
    L = o.lattice(cols)
    c = L["cells"]
    kept = int((np.isfinite(cols["lat"]) & (np.abs(cols["lat"]) <= 90)).sum())
    assert int(c["count"].sum()) + L["n_dropped"] == kept
    assert (c["volume"] <= c["count"]).all() and (c["volume"] >= 1).all()
    assert (c["mean_norm"] >= 0).all() and (c["mean_norm"] <= 1).all()
    for d in range(4):
        sel = c["dxn"] == d
        if sel.sum() > 1 and L["ch_max"][2 * d] > L["ch_min"][2 * d]:
            assert c["mean_norm"][sel].min() == 0 and c["mean_norm"][sel].max() == 1


def pin_run_length_dwell_and_speed_acceleration(o):
    """Time since a stop began (dwell summed over consecutive stop steps, reset at a moving step
    and at a journey start) and acceleration from implied speeds on a meridian (closed form)."""
    t = 1620532122000
    deg = lambda m: math.degrees(m / R)  # metres along a meridian
    lat = [37.0]
    for v in (10.0, 12.0, 14.0):  # 1 s steps at 10, 12, 14 m/s
        lat.append(lat[-1] + deg(v))
    lat += [lat[-1]] * 2  # a duplicate, then a 1 s step at rest
    n1 = len(lat)
    cols = dict(jid=np.array([7] * n1 + [8] * 7 + [9] * 2, np.int64),
                ts=np.array([t + 1000 * i for i in range(4)] + [t + 3000, t + 4000] +
                            [t + 1000 * i for i in range(7)] + [t, t + 1000], np.int64),
                lat=np.array(lat + [38.0] * 7 + [38.5] * 2),
                lon=np.full(n1 + 9, -92.5),
                speed=np.array([30, 30, 30, 30, 30, 30] + [5, 0, 0, 0, 5, 0, 0] + [0, 0], np.float32))
    p = o.run(cols)["points"]
    a = p["accel_v"]
    assert a[0] == 0 and a[1] == 0  # no previous implied speed
    assert abs(a[2] - 2.0) < 1e-6 and abs(a[3] - 2.0) < 1e-6
    assert a[4] == 0 and a[5] == 0  # a zero-dt step breaks the chain on both sides
    assert list(p["stop_ms"][n1:n1 + 7]) == [0, 0, 1000, 2000, 0, 0, 1000]
    assert list(p["stop_ms"][n1 + 7:]) == [0, 1000]  # a new journey starts a new run
    assert (p["stop_ms"][:n1] == 0).all()


CPU_PINS = [pin_haversine_closed_forms, pin_grid_index, pin_time_bin, pin_parse_fields, pin_table1,
            pin_bruteforce_orders, pin_kinematics_hand, pin_invalid_records, pin_direction_sectors,
            pin_run_length_dwell_and_speed_acceleration,
            pin_lattice_bruteforce, pin_lattice_invariants]
DATA_PINS = [pin_invariants, pin_library_cross_check, pin_csv_roundtrip]
