"""The float32 form against the binary64 oracle: order, keys, counts, flags, integer times,
min and max bit-exact; floating-point outputs within 1e-4 relative (with the 1e-9 absolute
floor). The largest and the 99.9th-percentile relative error of each output are reported."""
import numpy as np
import pytest

from parity import compare

pytestmark = pytest.mark.gpu

REL32 = 1e-4


def rel_err(got, want):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    den = np.maximum(np.maximum(np.abs(got), np.abs(want)), 1e-300)
    e = np.abs(got - want) / den
    e[(np.abs(got - want) <= 1e-9)] = 0.0
    return e


def run32(cols):
    import torch

    import paper_2305_07454_b300 as P

    t = {k: torch.from_numpy(np.ascontiguousarray(cols[k])).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
    with P.Pipeline(materialize_points=1, precision=P.FP32) as p:
        return p.run(t)


def report(g, o):
    """Largest and 99.9th-percentile relative error of every floating-point output."""
    out = {}
    for part, k in (("points", "d"), ("points", "vhat"), ("points", "accel"), ("points", "accel_v"),
                    ("journeys", "distance_m"), ("cells", "sum"), ("cells", "mean")):
        e = rel_err(g[part][k], o[part][k])
        out[f"{part}.{k}"] = (float(e.max()) if e.size else 0.0, float(np.quantile(e, 0.999)) if e.size else 0.0)
    # the acceleration from implied speeds differences two close speeds over a sub-second step,
    # so its float32 error is bounded in absolute terms (about 1e-4 m/s^2): reported too
    d = np.abs(np.asarray(g["points"]["accel_v"], np.float64) - o["points"]["accel_v"])
    out["points.accel_v.abs_m_s2"] = (float(d.max()) if d.size else 0.0,
                                      float(np.quantile(d, 0.999)) if d.size else 0.0)
    return out


def test_fp32_small_day(orc, small_day):
    g, o = run32(small_day), orc.run(small_day)
    errs = report(g, o)
    print("float32 form, max / p99.9 relative error per output:", errs)
    for k, (mx, _) in errs.items():
        if k.startswith("points.accel_v"):
            continue
        assert mx <= REL32, (k, mx)
    a_g = np.asarray(g["points"]["accel_v"], np.float64)
    a_o = o["points"]["accel_v"]
    assert np.all(np.abs(a_g - a_o) <= REL32 * np.maximum(np.abs(a_g), np.abs(a_o)) + 1e-4)
    # everything that is not floating point is identical to the binary64 form
    import parity

    for k in ("perm", "key", "flags", "dwell", "stop_ms"):
        parity.exact("point " + k, g["points"][k], o["points"][k])
    for k in ("id", "n", "offset", "start_ts", "end_ts", "duration_ms", "dwell_ms"):
        parity.exact("journey " + k, g["journeys"][k], o["journeys"]["jid" if k == "id" else k]
                     if k != "offset" else np.concatenate([[0], np.cumsum(o["journeys"]["n"])[:-1]]))
    for k in ("key", "row", "col", "bin", "count", "min", "max"):
        parity.exact("cell " + k, g["cells"][k], o["cells"][k])


def test_fp32_within_tolerance_everywhere(orc, small_day):
    """The generic comparison with the float32 tolerance."""
    g, o = run32(small_day), orc.run(small_day)
    compare(g, o, rel=REL32)
