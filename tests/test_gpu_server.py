"""Serving runtime: journey-hash feeds of a day, replayed as arrival windows through the server
with several slots. Each feed's tables are bit-identical to the same feed run alone through a
stream-mode context; the feeds merged equal the oracle's batch tables over the whole day;
two requests run together only when their reservations fit the memory budget together."""
import pytest

from parity import close, exact
from streams import LATE, arrivals, concat, merge_cells, merge_journeys, shard, windows

pytestmark = pytest.mark.gpu

COLS = ("jid", "ts", "lat", "lon", "speed")


def pinned(wins):
    import torch

    return [({k: torch.from_numpy(c[k]).pin_memory() for k in COLS}, end) for c, end in wins]


def alone(wins, precision):
    import torch

    import paper_2305_07454_b300 as P

    with P.Pipeline(mode=P.STREAM, lateness_ms=LATE, precision=precision) as p:
        for cols, end in wins:
            p.push_window({k: torch.from_numpy(cols[k]).cuda() for k in COLS}, end)
        p.flush()
        return p.results()


def serve(feed_wins, n_slots, budget=0, precision=0):
    """Submits every window of every feed in order of window end, then each feed's flush."""
    import paper_2305_07454_b300 as P

    host = [pinned(w) for w in feed_wins]
    order = sorted((end, f, i) for f, w in enumerate(host) for i, (_, end) in enumerate(w))
    with P.Server(n_slots=n_slots, mem_budget_bytes=budget) as srv:
        ids = [srv.add_feed(lateness_ms=LATE, precision=precision) for _ in host]
        tickets = [srv.submit(ids[f], host[f][i][0], end) for end, f, i in order]
        tickets += [srv.submit_flush(f) for f in ids]
        infos = [srv.wait(t) for t in tickets]
        res = [srv.feed(f).results() for f in ids]
    return res, infos


@pytest.fixture(scope="module")
def feeds(small_day):
    parts = shard(small_day, 3)
    return [windows(p, arrivals(p, 20 + i)) for i, p in enumerate(parts)]


def check_same(a, b):
    assert a["counters"] == b["counters"]
    for part in ("cells", "journeys"):
        for k in a[part]:
            exact(f"{part} {k}", b[part][k], a[part][k])


def check_merged(res, orc, feed_wins, rel):
    o = orc.run(concat([w for fw in feed_wins for w in fw]))
    cells = merge_cells([r["cells"] for r in res])
    for k in ("key", "row", "col", "bin", "count", "min", "max"):
        exact("cell " + k, cells[k], o["cells"][k])
    close("cell sum", cells["sum"], o["cells"]["sum"], rel)
    close("cell mean", cells["mean"], o["cells"]["mean"], rel)
    j = merge_journeys([r["journeys"] for r in res])
    exact("journey id", j["id"], o["journeys"]["jid"])
    for k in ("n", "start_ts", "end_ts", "duration_ms", "dwell_ms", "start_lat", "start_lon", "end_lat", "end_lon"):
        exact("journey " + k, j[k], o["journeys"][k])
    close("journey distance", j["distance_m"], o["journeys"]["distance_m"], rel)


@pytest.mark.parametrize("precision,rel", [(0, 1e-6), (1, 1e-4)], ids=["fp64", "fp32"])
def test_each_feed_is_the_same_alone_and_in_the_mix(orc, feeds, precision, rel):
    res, infos = serve(feeds, n_slots=3, precision=precision)
    assert all(i["status"] == 0 for i in infos)
    assert max(i["peak_in_flight"] for i in infos) >= 2  # feeds overlapped on the GPU
    for w, r in zip(feeds, res):
        check_same(alone(w, precision), r)
    check_merged(res, orc, feeds, rel)


def overlapping(infos):
    spans = sorted(((i["start_ns"], i["done_ns"], i) for i in infos), key=lambda t: t[0])
    for a in range(len(spans)):
        for b in range(a + 1, len(spans)):
            if spans[b][0] >= spans[a][1]:
                break
            yield spans[a][2], spans[b][2]


def test_feed_order_and_admission_by_memory(feeds):
    """Requests of one feed never overlap and run in submission order; two requests that ran
    at the same time had reservations that fit the budget together."""
    import paper_2305_07454_b300 as P

    sizes = sorted(c["ts"].shape[0] for w in feeds for c, _ in w)
    budget = sizes[-1] * P.SERVE_BYTES_PER_ROW
    assert sizes[-1] + sizes[-2] > sizes[-1]  # some pairs cannot run together
    res, infos = serve(feeds, n_slots=3, budget=budget)
    assert all(i["status"] == 0 for i in infos)
    for f in range(len(feeds)):
        mine = [i for i in infos if i["feed"] == f]  # submission order
        assert all(b["start_ns"] >= a["done_ns"] for a, b in zip(mine, mine[1:]))
    for a, b in overlapping(infos):
        assert (a["n"] + b["n"]) * P.SERVE_BYTES_PER_ROW <= budget, (a, b)
    ref, _ = serve(feeds, n_slots=1)
    for x, y in zip(ref, res):
        check_same(x, y)


def test_server_errors(feeds):
    import torch

    import paper_2305_07454_b300 as P

    w = pinned(feeds[0][:3])
    with P.Server(n_slots=2, mem_budget_bytes=1 << 20) as srv:
        f = srv.add_feed(lateness_ms=LATE)
        big = {k: torch.zeros(5000, dtype=v.dtype).pin_memory() for k, v in w[0][0].items()}
        with pytest.raises(P.CvetlError) as e:
            srv.submit(f, big, w[0][1])  # 5000 rows x 320 B > 1 MiB
        assert e.value.status == P.EFULL
        with pytest.raises(P.CvetlError) as e:
            srv.submit(7, w[0][0], w[0][1])
        assert e.value.status == P.EINVAL
        t1 = srv.submit(f, w[1][0], w[1][1])
        t0 = srv.submit(f, w[0][0], w[0][1])  # window ends must not go back
        assert srv.wait(t1)["status"] == P.OK
        info = srv.wait(t0, check=False)
        assert info["status"] == P.EINVAL and "order" in info["message"]
        with pytest.raises(P.CvetlError) as e:
            srv.wait(t0)  # released
        assert e.value.status == P.EINVAL
        srv.wait(srv.submit_flush(f))
        with pytest.raises(P.CvetlError) as e:
            srv.submit(f, w[2][0], w[2][1])
        assert e.value.status == P.ESTATE
        r = srv.feed(f).results()
        assert r["counters"]["n_in"] == w[1][0]["ts"].shape[0]
