"""Batches of instances (days x regions, each with its own grid and day) in one pass: every
instance's slice of the tables equals the oracle run on that instance alone with its grid."""
import numpy as np
import pytest

import cvgen
import oracle
from parity import compare, exact

pytestmark = pytest.mark.gpu

COLS = ("jid", "ts", "lat", "lon", "speed")


def make(seed=3, days=2, lo=5e3, hi=5e4, zipf_max=5000):
    recipes = cvgen.week_regions(seed=seed, days=days, min_records=lo, max_records=hi, zipf_max=zipf_max)
    insts = []
    for r in recipes:
        cols = cvgen.generate(r["params"])
        inst = {k: cols[k] for k in COLS}
        inst.update({k: r[k] for k in ("lat_min", "lon_min", "n_rows", "n_cols", "t0_ms")})
        insts.append(inst)
    return insts


def on_device(insts):
    import torch

    return [{k: (torch.from_numpy(v).cuda() if k in COLS else v) for k, v in q.items()} for q in insts]


def oracle_params(q):
    return oracle.default_params(lat_min=q["lat_min"], lon_min=q["lon_min"], n_rows=q["n_rows"],
                                 n_cols=q["n_cols"], t0_ms=q["t0_ms"])


def check_instances(orc, insts, res, rel=1e-6, points=True):
    for q, g in zip(insts, res):
        o = orc.run({k: q[k] for k in COLS}, oracle_params(q))
        if points:
            rg = g["ranges"]
            p = dict(g["points"])
            valid = p["key"] != 0xFFFFFFFF
            p["key"] = np.where(valid, p["key"] - np.uint32(rg["key_begin"]), p["key"]).astype(np.uint32)
            p["perm"] = (p["perm"] - np.uint32(rg["row_begin"])).astype(np.uint32)
            g = dict(g, points=p)
        # journey offsets are positions in the batch's sorted points
        j = dict(g["journeys"])
        if j["offset"].size:
            j["offset"] = j["offset"] - j["offset"][0]
        g = dict(g, journeys=j)
        compare(g, o, points=points, rel=rel, counters=False)


@pytest.mark.parametrize("precision,rel", [(0, 1e-6), (1, 1e-4)], ids=["fp64", "fp32"])
def test_each_instance_matches_the_oracle(orc, precision, rel):
    import paper_2305_07454_b300 as P

    insts = make()
    assert len(insts) == 8 and len({q["t0_ms"] for q in insts}) == 2
    with P.Pipeline(materialize_points=1, precision=precision) as p:
        res = p.run_batch(on_device(insts))
        tot = res[0]["batch_counters"]
    check_instances(orc, insts, res, rel=rel)
    assert tot["n_in"] == sum(q["jid"].shape[0] for q in insts)


def test_device_instances_read_in_place_aligned_or_not(orc):
    """Device instances are read in place: with every column aligned, the scatter takes 16-row
    groups per instance (32-byte column loads; an instance's last group may be partial and its
    first row need not be a multiple of 4); with one column 8 bytes off a 32-byte boundary (a
    view one element into a larger tensor), the one-row scatter. Both give each instance the
    oracle's results."""
    import torch

    import paper_2305_07454_b300 as P

    insts = make(seed=6, days=1)
    dev = on_device(insts)
    with P.Pipeline(materialize_points=1) as p:
        check_instances(orc, insts, p.run_batch(dev))
    shifted = []
    for q in dev:
        r = dict(q)
        big = torch.empty(q["lat"].shape[0] + 1, dtype=q["lat"].dtype, device=q["lat"].device)
        big[1:] = q["lat"]
        r["lat"] = big[1:]  # 8 bytes past the allocation's start
        assert r["lat"].data_ptr() % 32 != 0
        shifted.append(r)
    with P.Pipeline(materialize_points=1) as p:
        check_instances(orc, insts, p.run_batch(shifted))


def test_host_instances_and_one_instance_batch(orc):
    import torch

    import paper_2305_07454_b300 as P

    insts = make(seed=4, days=1)
    with P.Pipeline(materialize_points=1) as p:
        res = p.run_batch(insts)  # host columns
    check_instances(orc, insts, res)
    # a batch of one instance on the context's own grid gives the plain batch's bits
    q = dict(insts[0], lat_min=36.0, lon_min=-95.8, n_rows=460, n_cols=670, t0_ms=cvgen.DAY_START_MS)
    with P.Pipeline(materialize_points=1) as p:
        one = p.run_batch([q])[0]
        plain = p.run({k: torch.from_numpy(q[k]).cuda() for k in COLS})
    for part in ("cells", "journeys", "points"):
        for k in plain[part]:
            exact(f"{part} {k}", one[part][k], plain[part][k])


def test_empty_malformed_and_single_row_instances(orc):
    """Degenerate instances between ordinary ones: no rows, only malformed rows (NaN latitude)
    and a single row; every instance's slice equals the oracle on that instance alone."""
    import paper_2305_07454_b300 as P

    base = make(seed=9, days=1)
    a, b, c, d = base[:4]
    empty = dict(a, **{k: a[k][:0].copy() for k in COLS})
    bad = dict(b, lat=np.full_like(b["lat"], np.nan))
    one = dict(c, **{k: c[k][:1].copy() for k in COLS})
    insts = [a, empty, bad, one, d]
    with P.Pipeline(materialize_points=1) as p:
        res = p.run_batch(on_device(insts))
        tot = res[0]["batch_counters"]
    check_instances(orc, insts, res)
    assert tot["n_malformed"] == sum(orc.run({k: q[k] for k in COLS}, oracle_params(q))["counters"]["n_malformed"]
                                     for q in insts) >= b["jid"].shape[0]
    assert [r["journeys"]["n"].shape[0] for r in res[1:4]] == [0, 0, 1]


def test_same_ids_in_two_instances_are_two_journeys(orc):
    import paper_2305_07454_b300 as P

    insts = make(seed=5, days=1)[:2]
    insts[1] = dict(insts[1], jid=insts[1]["jid"] % 7 + insts[0]["jid"][0])  # ids shared with instance 0
    with P.Pipeline(materialize_points=1) as p:
        res = p.run_batch(on_device(insts))
    check_instances(orc, insts, res)


def test_batch_errors():
    import paper_2305_07454_b300 as P

    insts = make(seed=6, days=1)[:2]
    with P.Pipeline() as p:
        with pytest.raises(P.CvetlError) as e:
            p.extract_batch([])
        assert e.value.status == P.EINVAL
        bad = dict(insts[0], jid=insts[0]["jid"] + (1 << 60))
        p.extract_batch(on_device([bad, insts[1]]))
        with pytest.raises(P.CvetlError) as e:
            p.transform()
        assert e.value.status == P.EINVAL
        with pytest.raises(P.CvetlError) as e:
            p.extract_batch(on_device([dict(insts[0], n_rows=60000, n_cols=60000)]))
        assert e.value.status == P.EINVAL
