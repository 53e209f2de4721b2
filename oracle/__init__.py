"""ctypes binding of the plain CPU oracle (``cvoracle.c``).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import this package. The CUDA library never calls it and shares no
code with it.

The oracle follows arXiv 2305.07454: CSV extract (Methods, "Connected Vehicle Dataset";
Table 1), the floor-division binning of Algorithm 2 unrolled into one global positional
index (Accelerated ETL section, steps (3)-(4)), and the groupby count / sum / mean of
Table 3, plus per-journey kinematics and summaries whose definitions are readings (the
paper is silent on them); each reading is stated in ``cvoracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cvoracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]

KEY_INVALID = 0xFFFFFFFF
F_START, F_DUP, F_OFFGRID, F_STOP = 0x01, 0x02, 0x04, 0x08
DXN_CARDINAL, DXN_QUADRANT = 0, 1


def build(force: bool = False, src: str = _SRC, out: str = _SO) -> str:
    """Compiles the oracle with gcc (plain C, no FMA contraction, no fast-math)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        subprocess.check_call(["gcc", *CFLAGS, "-o", out, src, "-lm"])
    return out


class Params(ctypes.Structure):
    _fields_ = [
        ("lat_min", ctypes.c_double),
        ("lon_min", ctypes.c_double),
        ("cell_deg", ctypes.c_double),
        ("n_rows", ctypes.c_int32),
        ("n_cols", ctypes.c_int32),
        ("n_bins", ctypes.c_int32),
        ("t0_ms", ctypes.c_int64),
        ("bin_ms", ctypes.c_int64),
        ("v_stop_kmh", ctypes.c_float),
        ("earth_radius_m", ctypes.c_double),
    ]


class LatticeParams(ctypes.Structure):
    _fields_ = [("bin_ms", ctypes.c_int64), ("n_bins", ctypes.c_int32), ("direction", ctypes.c_int32)]


LATTICE_DTYPES = {"key": np.uint32, "bin": np.int32, "dxn": np.int32, "row": np.int32, "col": np.int32,
                  "count": np.uint32, "sum": np.float64, "mean": np.float32, "volume": np.uint32,
                  "mean_norm": np.float32, "volume_norm": np.float32}


class _LatticeCells(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in LATTICE_DTYPES]


def default_params(**kw) -> Params:
    """The statewide grid: 0.01 deg cells over 36.0-40.6 N, 95.8-89.1 W (460 x 670),
    1-minute bins over one day starting 2021-05-09 00:00 UTC, 1 km/h stop speed."""
    p = Params(lat_min=36.0, lon_min=-95.8, cell_deg=0.01, n_rows=460, n_cols=670,
               n_bins=1440, t0_ms=1620518400000, bin_ms=60000, v_stop_kmh=1.0,
               earth_radius_m=6371000.0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


_P = ctypes.c_void_p


class _Points(ctypes.Structure):
    _fields_ = [(n, _P) for n in ("perm", "d", "vhat", "accel", "dwell", "key", "flags", "stop_ms", "accel_v")]


class _Journeys(ctypes.Structure):
    _fields_ = [(n, _P) for n in ("jid", "n", "start_ts", "end_ts", "duration_ms", "distance_m",
                                  "dwell_ms", "start_lat", "start_lon", "end_lat", "end_lon")]


class _Cells(ctypes.Structure):
    _fields_ = [(n, _P) for n in ("key", "row", "col", "bin", "count", "sum", "mean", "min", "max", "volume")]


class _Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_in", "n_malformed", "n_valid", "n_out_of_grid",
                                              "n_dup", "n_journeys", "n_cells")]


POINT_DTYPES = dict(perm=np.uint32, d=np.float64, vhat=np.float64, accel=np.float64,
                    dwell=np.int64, key=np.uint32, flags=np.uint8, stop_ms=np.int64, accel_v=np.float64)
JOURNEY_DTYPES = dict(jid=np.int64, n=np.int64, start_ts=np.int64, end_ts=np.int64,
                      duration_ms=np.int64, distance_m=np.float64, dwell_ms=np.int64,
                      start_lat=np.float64, start_lon=np.float64, end_lat=np.float64,
                      end_lon=np.float64)
CELL_DTYPES = dict(key=np.uint32, row=np.int32, col=np.int32, bin=np.int32, count=np.uint32,
                   sum=np.float64, mean=np.float64, min=np.float32, max=np.float32, volume=np.uint32)


class Oracle:
    def __init__(self, so_path: str | None = None):
        lib = ctypes.CDLL(so_path or build())
        lib.orc_run.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _P, _P, _P, _P, _P,
                                ctypes.POINTER(_Points), ctypes.POINTER(_Journeys),
                                ctypes.POINTER(_Cells), ctypes.POINTER(_Counters)]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_parse_csv.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, _P, _P,
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        lib.orc_parse_csv.restype = ctypes.c_int64
        lib.orc_parse_decimal.argtypes = [ctypes.c_char_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
        lib.orc_parse_decimal.restype = ctypes.c_int
        lib.orc_parse_integer.argtypes = [ctypes.c_char_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        lib.orc_parse_integer.restype = ctypes.c_int
        lib.orc_haversine_m.argtypes = [ctypes.c_double] * 5
        lib.orc_haversine_m.restype = ctypes.c_double
        lib.orc_grid_index.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        lib.orc_grid_index.restype = ctypes.c_int32
        lib.orc_time_bin.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32]
        lib.orc_time_bin.restype = ctypes.c_int32
        lib.orc_direction.argtypes = [ctypes.c_float, ctypes.c_int32]
        lib.orc_direction.restype = ctypes.c_int32
        lib.orc_lattice.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(LatticeParams), ctypes.c_int64,
                                    _P, _P, _P, _P, _P, _P, ctypes.POINTER(_LatticeCells),
                                    ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _P, _P]
        lib.orc_lattice.restype = ctypes.c_int
        self.lib = lib

    # ---- single steps ----
    def haversine_m(self, lat1, lon1, lat2, lon2, radius_m=6371000.0) -> float:
        return self.lib.orc_haversine_m(lat1, lon1, lat2, lon2, radius_m)

    def grid_index(self, x, x_min, step, n) -> int:
        return self.lib.orc_grid_index(x, x_min, step, n)

    def time_bin(self, ts, t0_ms, bin_ms, n_bins) -> int:
        return self.lib.orc_time_bin(ts, t0_ms, bin_ms, n_bins)

    def direction(self, heading: float, mode: int = DXN_CARDINAL) -> int:
        return self.lib.orc_direction(heading, mode)

    def lattice(self, cols: dict, params: Params | None = None, bin_ms: int = 300000, n_bins: int = 288,
                direction: int = DXN_CARDINAL) -> dict:
        """The 8-channel lattice of the kept rows (needs a heading column)."""
        p = params or default_params()
        lp = LatticeParams(bin_ms=bin_ms, n_bins=n_bins, direction=direction)
        a = {k: np.ascontiguousarray(cols[k], dtype=dt) for k, dt in
             (("jid", np.int64), ("ts", np.int64), ("lat", np.float64), ("lon", np.float64),
              ("speed", np.float32), ("heading", np.float32))}
        n = int(a["jid"].shape[0])
        out = {k: np.empty(max(n, 1), dt) for k, dt in LATTICE_DTYPES.items()}
        sc = _LatticeCells(**{k: v.ctypes.data for k, v in out.items()})
        nc, nd = ctypes.c_int64(), ctypes.c_int64()
        mn, mx = np.zeros(8, np.float32), np.zeros(8, np.float32)
        rc = self.lib.orc_lattice(ctypes.byref(p), ctypes.byref(lp), n, *[a[k].ctypes.data for k in
                                  ("jid", "ts", "lat", "lon", "speed", "heading")], ctypes.byref(sc),
                                  ctypes.byref(nc), ctypes.byref(nd), mn.ctypes.data, mx.ctypes.data)
        if rc != 0:
            raise RuntimeError(f"orc_lattice failed ({rc})")
        return {"cells": {k: v[:nc.value] for k, v in out.items()}, "n_dropped": int(nd.value),
                "ch_min": mn, "ch_max": mx}

    def parse_decimal(self, s: str):
        b = s.encode()
        out = ctypes.c_double()
        ok = self.lib.orc_parse_decimal(b, len(b), ctypes.byref(out))
        return out.value if ok else None

    def parse_integer(self, s: str):
        b = s.encode()
        out = ctypes.c_int64()
        ok = self.lib.orc_parse_integer(b, len(b), ctypes.byref(out))
        return out.value if ok else None

    # ---- extract ----
    def parse_csv(self, buf: np.ndarray | bytes):
        """Returns (columns dict, n_lines, n_malformed): one row per line, malformed lines as
        rows (0, 0, NaN, NaN, NaN, NaN) that the extract drops."""
        if isinstance(buf, (bytes, bytearray)):
            buf = np.frombuffer(bytes(buf), dtype=np.uint8)
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        cap = int(np.count_nonzero(buf == ord("\n"))) + 1
        cols = dict(jid=np.empty(cap, np.int64), ts=np.empty(cap, np.int64),
                    lat=np.empty(cap, np.float64), lon=np.empty(cap, np.float64),
                    speed=np.empty(cap, np.float32), heading=np.empty(cap, np.float32))
        nl, nm = ctypes.c_int64(), ctypes.c_int64()
        rows = self.lib.orc_parse_csv(buf.ctypes.data, buf.shape[0], cap,
                                      *[cols[c].ctypes.data for c in
                                        ("jid", "ts", "lat", "lon", "speed", "heading")],
                                      ctypes.byref(nl), ctypes.byref(nm))
        if rows < 0:
            raise RuntimeError("orc_parse_csv: capacity too small")
        return {k: v[:rows].copy() for k, v in cols.items()}, int(nl.value), int(nm.value)

    # ---- whole path ----
    def run(self, cols: dict, params: Params | None = None) -> dict:
        p = params or default_params()
        jid = np.ascontiguousarray(cols["jid"], dtype=np.int64)
        ts = np.ascontiguousarray(cols["ts"], dtype=np.int64)
        lat = np.ascontiguousarray(cols["lat"], dtype=np.float64)
        lon = np.ascontiguousarray(cols["lon"], dtype=np.float64)
        speed = np.ascontiguousarray(cols["speed"], dtype=np.float32)
        n = int(jid.shape[0])
        cap = max(n, 1)
        pts = {k: np.empty(cap, dt) for k, dt in POINT_DTYPES.items()}
        jr = {k: np.empty(cap, dt) for k, dt in JOURNEY_DTYPES.items()}
        cl = {k: np.empty(cap, dt) for k, dt in CELL_DTYPES.items()}
        sp = _Points(**{k: v.ctypes.data for k, v in pts.items()})
        sj = _Journeys(**{k: v.ctypes.data for k, v in jr.items()})
        sc = _Cells(**{k: v.ctypes.data for k, v in cl.items()})
        cnt = _Counters()
        rc = self.lib.orc_run(ctypes.byref(p), n, jid.ctypes.data, ts.ctypes.data, lat.ctypes.data,
                              lon.ctypes.data, speed.ctypes.data, ctypes.byref(sp), ctypes.byref(sj),
                              ctypes.byref(sc), ctypes.byref(cnt))
        if rc != 0:
            raise RuntimeError(f"orc_run failed ({rc})")
        c = {k: int(getattr(cnt, k)) for k, _ in _Counters._fields_}
        nv, nj, nc = c["n_valid"], c["n_journeys"], c["n_cells"]
        return dict(points={k: v[:nv] for k, v in pts.items()},
                    journeys={k: v[:nj] for k, v in jr.items()},
                    cells={k: v[:nc] for k, v in cl.items()},
                    counters=c)


_default = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default
