"""The FP64 form's distance over the whole domain its fast path can meet, against the oracle.

The journey kernel evaluates the haversine of steps below 0.0229 degrees on both axes with a
series whose terms above 2^-22 relative are binary64 (cosines from a 0.01-degree table by angle
addition, a float32 reciprocal square root refined in binary64), and larger steps with the
general formula. Each case here aims at a place where that scheme could go wrong: latitudes
from pole to pole (the cosine's relative correction divides by a cosine that vanishes at the
poles), steps just either side of the switch, points on the table's knots and half-way between
them (where the table index rounds), and steps across the antimeridian. Per-point distances
must stay within 1e-13 relative of the oracle's libm evaluation, journey sums within 1e-12, and
every other output within the usual parity bounds (keys, order and counts exact), also on grids
placed far from the default box.
"""
import numpy as np
import pytest

from parity import close, compare

pytestmark = pytest.mark.gpu

T0 = 1620518400000


def run_gpu(cols, **cfg):
    import torch

    import paper_2305_07454_b300 as P

    t = {k: torch.from_numpy(np.ascontiguousarray(cols[k])).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
    with P.Pipeline(materialize_points=1, **cfg) as p:
        return p.run(t)


def _journeys(paths, seed):
    """Shuffled columns from explicit (lat, lon) paths, one journey each (test-local inputs)."""
    rng = np.random.default_rng(seed)
    parts = []
    for j, (lat, lon) in enumerate(paths):
        m = lat.shape[0]
        dt = rng.integers(300, 1000, m)
        dt[0] = 0
        ts = T0 + 3_600_000 + int(rng.integers(0, 3_600_000)) + np.cumsum(dt)
        spd = np.abs(rng.normal(40, 30, m)).astype(np.float32)
        parts.append(dict(jid=np.full(m, 1000 + j, np.int64), ts=ts.astype(np.int64), lat=lat.astype(np.float64),
                          lon=lon.astype(np.float64), speed=spd))
    cols = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    perm = rng.permutation(cols["jid"].shape[0])
    return {k: np.ascontiguousarray(v[perm]) for k, v in cols.items()}


def _walk(rng, lat0, lon0, m, step):
    lat = np.clip(lat0 + np.cumsum(rng.normal(0, step, m)), -90.0, 90.0)
    lon = lon0 + np.cumsum(rng.normal(0, step, m))
    lon = (lon + 180.0) % 360.0 - 180.0
    return lat, lon


def _check(cols, **cfg):
    import oracle

    o = oracle.get().run(cols, oracle.default_params(**cfg))
    g = run_gpu(cols, **cfg)
    compare(g, o)
    close("point d", g["points"]["d"], o["points"]["d"], rel=1e-13, abs_=1e-12)
    close("journey distance", g["journeys"]["distance_m"], o["journeys"]["distance_m"], rel=1e-12, abs_=1e-9)
    d_g, d_o = g["points"]["d"], o["points"]["d"]
    nz = d_o > 0
    return float(np.max(np.abs(d_g[nz] - d_o[nz]) / d_o[nz])) if nz.any() else 0.0


def test_latitudes_pole_to_pole():
    """Random walks at 75 base latitudes in [-89.9, 89.9] (and both poles), steps from 1e-6 to
    0.01 degrees, longitudes all round the globe."""
    rng = np.random.default_rng(5)
    paths = []
    bases = np.concatenate([np.linspace(-89.9, 89.9, 73), [-90.0, 90.0]])
    for i, b in enumerate(bases):
        step = [1e-6, 2e-5, 1e-3, 0.01][i % 4]
        m = [40, 300, 700][i % 3]
        paths.append(_walk(rng, b, rng.uniform(-180, 180), m, step))
    err = _check(_journeys(paths, seed=6))
    print("max relative error of d:", err)


@pytest.mark.parametrize("lat0", [-89.95, -60.0, -0.01, 0.0, 37.0, 75.5, 89.95])
def test_steps_either_side_of_the_series_switch(lat0):
    """Steps of 0.0228, 0.0229 and 0.0230 degrees (and near-zero) in every sign combination on
    both axes: the series below 0.0229, the general formula above."""
    steps = [0.0, 1e-9, 0.0228, 0.02289999, 0.0229, 0.02290001, 0.0230]
    dl, dn = [], []
    for a in steps:
        for b in steps:
            for sa in (1, -1):
                for sb in (1, -1):
                    dl.append(sa * a)
                    dn.append(sb * b)
    dl, dn = np.array(dl), np.array(dn)
    # alternate forward and back so the walk stays near lat0
    sign = np.where(np.arange(dl.shape[0]) % 2 == 0, 1.0, -1.0)
    lat = np.clip(lat0 + np.concatenate([[0.0], np.cumsum(dl * sign)]), -90, 90)
    lon = -92.0 + np.concatenate([[0.0], np.cumsum(dn * sign)])
    # steps from an exactly representable origin too (the coordinate difference is then exact)
    lat2 = np.concatenate([[0.0], np.abs(dl)]) * np.where(np.arange(dl.shape[0] + 1) % 2 == 0, 0.0, 1.0)
    lon2 = np.concatenate([[0.0], np.abs(dn)]) * np.where(np.arange(dn.shape[0] + 1) % 2 == 0, 0.0, 1.0)
    err = _check(_journeys([(lat, lon), (lat2, lon2)], seed=7))
    print("max relative error of d:", err)


def test_points_on_and_between_the_cosine_table_knots():
    """Latitudes on the 0.01-degree knots, half-way between them (where the table index rounds
    either way) and a hair either side of half-way, hopping between neighbours."""
    rng = np.random.default_rng(8)
    paths = []
    for k0 in (-8999, -8000, -4567, -1, 0, 1, 3700, 3701, 6543, 8999):
        base = k0 * 0.01
        offs = np.array([0.0, 0.005, -0.005, 0.005 + 1e-12, 0.005 - 1e-12, -0.005 + 1e-12, -0.005 - 1e-12,
                         0.01, 0.015, -0.015, 0.0049999, 0.0050001])
        lat = np.clip(base + rng.choice(offs, 400), -90.0, 90.0)
        lon = -92.0 + np.cumsum(rng.normal(0, 3e-3, 400))
        paths.append((lat, lon))
    err = _check(_journeys(paths, seed=9))
    print("max relative error of d:", err)


def test_antimeridian_crossings():
    """Steps across +-180 degrees of longitude (differenced in degrees first: 359.9998 degrees,
    the general formula) and along it, at several latitudes."""
    paths = []
    for lat0 in (-75.0, -10.0, 0.0, 37.2, 89.0):
        lon = np.array([179.9999, -179.9999, 179.99995, -180.0, 180.0, -179.9, 179.9, 179.9999, -179.99995] * 20)
        lat = lat0 + np.arange(lon.shape[0]) * 1e-5
        paths.append((lat, lon))
    err = _check(_journeys(paths, seed=10))
    print("max relative error of d:", err)


@pytest.mark.parametrize("grid", [
    dict(lat_min=-45.0, lon_min=100.0, n_rows=300, n_cols=300),
    dict(lat_min=-89.9, lon_min=-180.0, cell_deg=0.5, n_rows=359, n_cols=720),
    dict(lat_min=59.99, lon_min=170.0, n_rows=500, n_cols=999),
])
def test_grids_far_from_the_default_box(grid):
    """Keys on other grids, with journeys that walk over them (and off their edges)."""
    rng = np.random.default_rng(11)
    cd = grid.get("cell_deg", 0.01)
    paths = []
    for i in range(30):
        lat0 = grid["lat_min"] + rng.uniform(0, grid["n_rows"] * cd)
        lon0 = grid["lon_min"] + rng.uniform(0, grid["n_cols"] * cd)
        paths.append(_walk(rng, lat0, lon0, [50, 600, 1500][i % 3], [2e-5, 1e-3, 0.02][i % 3]))
    cols = _journeys(paths, seed=12)
    err = _check(cols, **grid)
    print("max relative error of d:", err)
