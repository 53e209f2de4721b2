"""Element-by-element comparison of the CUDA path's outputs with the oracle's.

Tolerances (FP64 form): bit-exact for the order, keys, counts, flags, integer times, dwell,
min and max; |x - y| <= 1e-6 * max(|x|, |y|) + 1e-9 for floating-point sums, distances,
implied speeds and accelerations. The GPU stores implied speed and acceleration as float32,
so those compare the oracle's binary64 value with the float32 result (6e-8 relative rounding,
well inside the bound).
"""
from __future__ import annotations

import numpy as np

REL = 1e-6
ABS = 1e-9


def close(name, got, want, rel=REL, abs_=ABS):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape, (name, got.shape, want.shape)
    if got.size == 0:
        return
    both_nan = np.isnan(got) & np.isnan(want)
    err = np.abs(got - want)
    bound = rel * np.maximum(np.abs(got), np.abs(want)) + abs_
    bad = ~(both_nan | (err <= bound))
    assert not bad.any(), (f"{name}: {int(bad.sum())} of {got.size} outside tolerance; first at "
                           f"{int(np.flatnonzero(bad)[0])}: got {got[bad][0]!r} want {want[bad][0]!r}")


def exact(name, got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    assert got.shape == want.shape, (name, got.shape, want.shape)
    if got.size == 0:
        return
    if got.dtype.kind == "f":
        ok = (got == want) | (np.isnan(got) & np.isnan(want))
    else:
        ok = got == want.astype(got.dtype)
    assert ok.all(), (f"{name}: {int((~ok).sum())} of {got.size} differ; first at "
                      f"{int(np.flatnonzero(~ok)[0])}: got {got[~ok][0]!r} want {want[~ok][0]!r}")


def compare(gpu: dict, orc: dict, points: bool = True, rel: float = REL, counters: bool = True):
    if counters:
        gc, oc = gpu["counters"], orc["counters"]
        for k in ("n_in", "n_malformed", "n_valid", "n_out_of_grid", "n_dup", "n_journeys", "n_cells"):
            assert gc[k] == oc[k], (k, gc[k], oc[k])
    gj, oj = gpu["journeys"], orc["journeys"]
    exact("journey id", gj["id"], oj["jid"])
    exact("journey n", gj["n"], oj["n"])
    offs = np.concatenate([[0], np.cumsum(oj["n"])[:-1]]) if oj["n"].size else oj["n"]
    exact("journey offset", gj["offset"], offs)
    for k in ("start_ts", "end_ts", "duration_ms", "dwell_ms", "start_lat", "start_lon", "end_lat", "end_lon"):
        exact("journey " + k, gj[k], oj[k])
    close("journey distance", gj["distance_m"], oj["distance_m"], rel)
    g, o = gpu["cells"], orc["cells"]
    for k in ("key", "row", "col", "bin", "count", "min", "max"):
        exact("cell " + k, g[k], o[k])
    if g.get("volume") is not None and g["volume"].shape == g["key"].shape:  # batch mode
        exact("cell volume", g["volume"], o["volume"])
    close("cell sum", g["sum"], o["sum"], rel)
    close("cell mean", g["mean"], o["mean"], rel)
    if points:
        gp, op = gpu["points"], orc["points"]
        for k in ("perm", "key", "flags", "dwell", "stop_ms"):
            exact("point " + k, gp[k], op[k])
        close("point d", gp["d"], op["d"], rel)
        close("point vhat", gp["vhat"], op["vhat"], rel)
        close("point accel", gp["accel"], op["accel"], rel)
        # a difference of two close implied speeds over dt: the float32 form's distances
        # (2^-24 relative, speeds <= 36 m/s, steps >= 0.25 s) bound its error by ~1e-4 m/s^2
        close("point accel_v", gp["accel_v"], op["accel_v"], rel, ABS if rel <= REL else 1e-4)
