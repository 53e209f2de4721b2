"""The 8-channel lattice against the oracle: occupied cells bit-exact (keys, counts, unique
journeys, speed sums in the same order, means, normalised channels), channel extremes and
dropped rows equal; the dense tensor holds each occupied cell's two channels and zeros
elsewhere."""
import numpy as np
import pytest

import cvgen
from oracle_pins import _lattice_case
from parity import exact

pytestmark = pytest.mark.gpu

COLS = ("jid", "ts", "lat", "lon", "speed", "heading")
SMALL = dict(bin_ms=3600000, n_bins=24)  # hour bins keep the dense tensor small here


def gpu_lattice(cols, device=True, **cfg):
    import torch

    import paper_2305_07454_b300 as P

    t = {k: torch.from_numpy(np.ascontiguousarray(cols[k])) for k in COLS}
    if device:
        t = {k: v.cuda() for k, v in t.items()}
    with P.Pipeline() as p:
        p.run(t, to_host=False)
        L = p.lattice(**cfg)
        dense = L["dense"]
        if dense is not None:
            L["dense_checks"] = dense_checks(L, dense, cfg.get("normalize", 0))
        L["dense"] = None
    return L


def dense_checks(L, dense, normalized):
    """The dense tensor at every occupied cell, its total and its non-zero count, on the device."""
    import torch

    c = {k: torch.from_numpy(v).cuda() for k, v in L["cells"].items()}
    b, d, r, col = (c[k].long() for k in ("bin", "dxn", "row", "col"))
    a = dense[b, 2 * d, r, col]
    v = dense[b, 2 * d + 1, r, col]
    want_a = c["mean_norm"] if normalized else c["mean"]
    want_v = c["volume_norm"] if normalized else c["volume"].float()
    assert torch.equal(a, want_a) and torch.equal(v, want_v)
    total = float(dense.double().sum())
    assert abs(total - float(want_a.double().sum() + want_v.double().sum())) <= 1e-6 * max(1.0, abs(total))
    assert int((dense != 0).sum()) == int((want_a != 0).sum() + (want_v != 0).sum())
    return True


def check(g, o):
    assert g["n_dropped"] == o["n_dropped"]
    exact("ch_min", g["ch_min"], o["ch_min"])
    exact("ch_max", g["ch_max"], o["ch_max"])
    for k in ("key", "bin", "dxn", "row", "col", "count", "sum", "mean", "volume", "mean_norm", "volume_norm"):
        exact("lattice " + k, g["cells"][k], o["cells"][k])


def test_small_day(orc, small_day):
    g = gpu_lattice(small_day, **SMALL, dense=1)
    o = orc.lattice(small_day, **SMALL)
    check(g, o)
    assert g["dense_checks"]


def test_overlapping_journeys_and_normalised_dense(orc):
    cols, _ = _lattice_case(seed=11)
    g = gpu_lattice(cols, bin_ms=300000, n_bins=288, dense=1, normalize=1)
    o = orc.lattice(cols)
    check(g, o)
    assert g["cells"]["volume"].max() > 1 and g["dense_checks"]


def test_quadrant_directions_and_host_input(orc):
    cols = cvgen.generate(cvgen.params("small_day", seed=12, n_journeys=500))
    g = gpu_lattice(cols, device=False, **SMALL, direction=1, dense=0)
    o = orc.lattice(cols, **SMALL, direction=1)
    check(g, o)


def test_many_journeys_sharing_cells(orc):
    """3,000 journeys of a few hundred points over one day: many share a cell and bin."""
    p = cvgen.params("small_day", seed=13, n_journeys=3000, median_len=300.0)
    cols = cvgen.generate(p)
    g = gpu_lattice(cols, dense=0)
    o = orc.lattice(cols)
    check(g, o)


def test_csv_input(orc):
    import torch

    import paper_2305_07454_b300 as P

    cols = cvgen.generate(cvgen.params("small_day", seed=14, n_journeys=300))
    text, _ = cvgen.to_csv(cols, seed=14, malformed_frac=0.01)
    parsed, _, _ = orc.parse_csv(text)
    with P.Pipeline() as p:
        p.extract_csv(torch.from_numpy(text).cuda())
        p.transform()
        p.load()
        g = p.lattice(**SMALL, dense=0)
    check(g, orc.lattice(parsed, **SMALL))


def test_lattice_errors(small_day):
    import torch

    import paper_2305_07454_b300 as P

    t = {k: torch.from_numpy(np.ascontiguousarray(small_day[k])).cuda() for k in COLS}
    with P.Pipeline() as p:
        p.extract(t)
        with pytest.raises(P.CvetlError) as e:
            p.lattice()
        assert e.value.status == P.ESTATE
        p.transform()
        p.load()
        with pytest.raises(P.CvetlError) as e:
            p.lattice(n_bins=0)
        assert e.value.status == P.EINVAL
        no_heading = {k: v for k, v in t.items() if k != "heading"}
        p.run(no_heading, to_host=False)
        with pytest.raises(P.CvetlError) as e:
            p.lattice()
        assert e.value.status == P.EINVAL


@pytest.mark.parametrize("direction", [0, 1])
def test_headings_at_sector_edges(orc, direction):
    """Headings on and next to every sector edge, far outside [0, 360), tiny, signed zero,
    infinite and NaN: the float32 fast path and the out-of-line binary64 path against the
    oracle's definition."""
    edges = [-405.0, -360.0, -315.0, -270.0, -225.0, -180.0, -135.0, -90.0, -45.0, 0.0, 45.0, 90.0,
             135.0, 180.0, 225.0, 270.0, 315.0, 360.0, 405.0, 720.0]
    h = []
    for e in edges:
        f = np.float32(e)
        h += [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    h += [np.float32(v) for v in (-0.0, 1e-30, -1e-30, 1e-45, -1e-45, 1e30, -1e30, 3.4e38, -3.4e38)]
    h += [np.float32(np.inf), np.float32(-np.inf), np.float32(np.nan)]
    h = np.array(h, np.float32)
    n = h.shape[0]
    rng = np.random.default_rng(21)
    cols = dict(jid=rng.integers(0, 5, n).astype(np.int64),
                ts=(1620518400000 + rng.integers(0, 86_400_000, n)).astype(np.int64),
                lat=38.0 + rng.uniform(0, 0.05, n), lon=-92.0 + rng.uniform(0, 0.05, n),
                speed=rng.uniform(0, 100, n).astype(np.float32), heading=h)
    g = gpu_lattice(cols, **SMALL, direction=direction, dense=0)
    o = orc.lattice(cols, **SMALL, direction=direction)
    check(g, o)
    assert g["n_dropped"] == 3  # the non-finite headings
