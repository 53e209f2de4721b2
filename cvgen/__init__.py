"""Seeded synthetic connected-vehicle records (ctypes binding of ``cvgen.c``).

The records stand in for the Missouri DOT connected-vehicle data of arXiv 2305.07454
(Methods, "Connected Vehicle Dataset"; Table 1), which is not available: shuffled rows of
(journey id, timestamp ms, latitude, longitude, speed km/h, heading deg) with lognormal or
Zipf journey lengths, 0.3-1.0 s sampling plus jitter, a diurnal start-time curve and random
walks inside the 36.0-40.6 N, 95.8-89.1 W box.

This module draws inputs only; it holds none of the ETL method's arithmetic. The CPU oracle
and the CUDA library both consume the arrays it returns.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libcvgen.so")
_SRC = os.path.join(_HERE, "cvgen.c")


class Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_journeys", ctypes.c_int64),
        ("len_dist", ctypes.c_int32),
        ("median_len", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("zipf_s", ctypes.c_double),
        ("min_len", ctypes.c_int64),
        ("max_len", ctypes.c_int64),
        ("day_start_ms", ctypes.c_int64),
        ("n_days", ctypes.c_int32),
        ("lat_lo", ctypes.c_double),
        ("lat_hi", ctypes.c_double),
        ("lon_lo", ctypes.c_double),
        ("lon_hi", ctypes.c_double),
        ("dup_frac", ctypes.c_double),
        ("outlier_frac", ctypes.c_double),
        ("stop_prob", ctypes.c_double),
        ("negzero_frac", ctypes.c_double),
        ("jid_mode", ctypes.c_int32),
        ("shuffle", ctypes.c_int32),
        ("threads", ctypes.c_int32),
    ]


# Named workloads, by what they are.
WORKLOADS = {
    # 1,000 journeys, lognormal lengths with median 150 (mean ~200): ~200k records.
    "small_day": dict(n_journeys=1000, median_len=150.0),
    # 60,000 journeys over one day, ~150M records: the median is raised to 1,875 points so
    # that the stated journey and record totals hold together (mean ~2,500 points).
    "full_day": dict(n_journeys=60000, median_len=1875.0),
    # A tenth of the full day (6,000 journeys, ~15M records): still larger than L2, small
    # enough for detailed profiler captures.
    "tenth_day": dict(n_journeys=6000, median_len=1875.0),
}

DAY_START_MS = 1620518400000  # 2021-05-09 00:00:00 UTC
COLUMNS = ("jid", "ts", "lat", "lon", "speed", "heading")
DTYPES = {"jid": np.int64, "ts": np.int64, "lat": np.float64, "lon": np.float64,
          "speed": np.float32, "heading": np.float32}


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-pthread", "-shared", "-fPIC", "-o", _SO, _SRC, "-lm"])
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.cvgen_default.argtypes = [ctypes.POINTER(Params)]
        lib.cvgen_count.argtypes = [ctypes.POINTER(Params)]
        lib.cvgen_count.restype = ctypes.c_int64
        vp = ctypes.c_void_p
        lib.cvgen_fill.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, vp, vp, vp, vp, vp, vp]
        lib.cvgen_fill.restype = ctypes.c_int
        lib.cvgen_csv.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_int32, vp, ctypes.c_int64,
                                  ctypes.POINTER(ctypes.c_int64)]
        lib.cvgen_csv.restype = ctypes.c_int64
        _lib = lib
    return _lib


def params(workload: str | None = "small_day", seed: int = 1, **overrides) -> Params:
    lib = _load()
    p = Params()
    lib.cvgen_default(ctypes.byref(p))
    p.seed = seed
    if workload is not None:
        for k, v in WORKLOADS[workload].items():
            setattr(p, k, v)
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def count(p: Params) -> int:
    n = _load().cvgen_count(ctypes.byref(p))
    if n < 0:
        raise ValueError("bad generator parameters")
    return int(n)


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def generate(p: Params | str = "small_day", seed: int = 1, out: dict | None = None,
             **overrides) -> dict:
    """Returns the six columns as numpy arrays (or fills ``out``, a dict of arrays)."""
    if isinstance(p, str):
        p = params(p, seed=seed, **overrides)
    n = count(p)
    if out is None:
        out = {c: np.empty(n, dtype=DTYPES[c]) for c in COLUMNS}
    for c in COLUMNS:
        a = out[c]
        if a.dtype != DTYPES[c] or a.shape[0] < n:
            raise ValueError(f"output column {c} has the wrong type or length")
    rc = _load().cvgen_fill(ctypes.byref(p), n, *[_ptr(out[c]) for c in COLUMNS])
    if rc != 0:
        raise RuntimeError(f"cvgen_fill failed ({rc})")
    return {c: out[c][:n] for c in COLUMNS}


def to_csv(cols: dict, seed: int = 1, malformed_frac: float = 0.005, threads: int = 0):
    """CSV bytes (numpy uint8) of the columns and the number of rows deliberately corrupted."""
    lib = _load()
    n = int(cols["jid"].shape[0])
    ptrs = [_ptr(np.ascontiguousarray(cols[c])) for c in COLUMNS]
    bad = ctypes.c_int64(0)
    size = lib.cvgen_csv(*ptrs, n, seed, malformed_frac, threads, None, 0, ctypes.byref(bad))
    if size < 0:
        raise RuntimeError("cvgen_csv sizing failed")
    buf = np.empty(max(int(size), 1), dtype=np.uint8)
    got = lib.cvgen_csv(*ptrs, n, seed, malformed_frac, threads, _ptr(buf), int(size), ctypes.byref(bad))
    if got != size:
        raise RuntimeError("cvgen_csv write failed")
    return buf[: int(size)], int(bad.value)


# The batched workload: 7 days x the 4 quadrant boxes of the statewide box, each instance a
# day of one region with its own grid (230 x 335 cells of 0.01 deg) and its own day start.
# Instance sizes are log-uniform in [2M, 150M] records (times `scale`), journey lengths Zipf
# with s = 1.5 on [10, 200,000].
WEEK_BOX = (36.0, 40.6, -95.8, -89.1)
ZIPF_S, ZIPF_MIN, ZIPF_MAX = 1.5, 10, 200_000


def _zipf_mean(s: float, lo: int, hi: int) -> float:
    k = np.arange(lo, hi + 1, dtype=np.float64)
    w = k ** -s
    return float((w * k).sum() / w.sum())


def week_regions(seed: int = 1, scale: float = 1.0, days: int = 7, min_records: float = 2e6,
                 max_records: float = 150e6, zipf_max: int = ZIPF_MAX) -> list:
    """Instance recipes: dicts with the generator parameters (``params``) and the grid
    (lat_min, lon_min, n_rows, n_cols, t0_ms) of each (day, quadrant) instance."""
    rng = np.random.default_rng(seed)
    lat0, lat1, lon0, lon1 = WEEK_BOX
    latm, lonm = (lat0 + lat1) / 2, (lon0 + lon1) / 2
    quads = [(lat0, latm, lon0, lonm), (lat0, latm, lonm, lon1), (latm, lat1, lon0, lonm), (latm, lat1, lonm, lon1)]
    mean_len = _zipf_mean(ZIPF_S, ZIPF_MIN, zipf_max)
    out = []
    for d in range(days):
        for q, (a, b, c, e) in enumerate(quads):
            target = float(np.exp(rng.uniform(np.log(min_records), np.log(max_records)))) * scale
            t0 = DAY_START_MS + d * 86_400_000
            p = params(None, seed=seed * 1000 + d * 4 + q + 1, n_journeys=max(1, int(round(target / mean_len))),
                       len_dist=1, zipf_s=ZIPF_S, min_len=ZIPF_MIN, max_len=zipf_max, day_start_ms=t0,
                       n_days=1, lat_lo=a, lat_hi=b, lon_lo=c, lon_hi=e)
            out.append({"params": p, "lat_min": a, "lon_min": c, "n_rows": int(round((b - a) / 0.01)),
                        "n_cols": int(round((e - c) / 0.01)), "t0_ms": t0})
    return out
