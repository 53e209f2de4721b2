"""The batch path as a CUDA graph (config.graph = 1): the first run of a shape runs eagerly and is
captured, later runs of the shape replay the graph. Every run gives the eager path's bits, and a
replay recomputes from whatever the input buffers hold."""
import numpy as np
import pytest

from parity import exact
from test_gpu_batch import make, on_device

pytestmark = pytest.mark.gpu

COLS = ("jid", "ts", "lat", "lon", "speed")


def same(a, b, parts=("cells", "journeys", "points")):
    assert a["counters"] == b["counters"]
    for part in parts:
        for k in a[part]:
            exact(f"{part} {k}", b[part][k], a[part][k])


def test_replays_match_the_eager_path(small_day):
    import torch

    import paper_2305_07454_b300 as P

    t = {k: torch.from_numpy(np.ascontiguousarray(small_day[k])).cuda() for k in COLS}
    with P.Pipeline(materialize_points=1) as p:
        ref = p.run(t)
    with P.Pipeline(materialize_points=1, graph=1, profile=1) as p:
        runs = [p.run(t) for _ in range(3)]
        st = p.stats()
    for r in runs:
        same(ref, r)
    assert st["stages"]["journey_sort"]["launches"] == 3 * 4 and st["stages"]["journeys"]["launches"] == 3
    assert st["graph_replays"] == 2  # the first run of the shape is eager and captured


def test_a_replay_recomputes_from_the_buffers(orc, small_day):
    import torch

    import paper_2305_07454_b300 as P

    t = {k: torch.from_numpy(np.ascontiguousarray(small_day[k])).cuda() for k in COLS}
    slow = dict(small_day, speed=(small_day["speed"] * np.float32(0.5)).astype(np.float32))
    with P.Pipeline(materialize_points=1, graph=1) as p:
        p.run(t)
        p.run(t)  # captured shape
        t["speed"].copy_(torch.from_numpy(slow["speed"]))  # same buffers, same shape, new values
        got = p.run(t)
        assert p.stats()["graph_replays"] == 2
    with P.Pipeline(materialize_points=1) as p:
        want = p.run({k: torch.from_numpy(np.ascontiguousarray(slow[k])).cuda() for k in COLS})
    same(want, got)
    assert np.array_equal(got["cells"]["max"], np.asarray(orc.run(slow)["cells"]["max"]))


def test_batches_in_graph_mode():
    import paper_2305_07454_b300 as P

    insts = on_device(make(seed=9, days=1))
    with P.Pipeline(materialize_points=1) as p:
        ref = p.run_batch(insts)
    with P.Pipeline(materialize_points=1, graph=1) as p:
        for _ in range(3):
            got = p.run_batch(insts)
            for a, b in zip(ref, got):
                for part in ("cells", "journeys", "points"):
                    for k in a[part]:
                        exact(f"{part} {k}", b[part][k], a[part][k])
        assert p.stats()["graph_replays"] == 2
