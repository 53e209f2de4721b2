"""Stream mode: windows of records by arrival time. After the last window and cvetl_flush the
tables equal the batch tables of the oracle over the same records (integers, min and max
exactly, sums within the tolerance); records older than the previous watermark when they arrive
are dropped and counted; a stream gives the same bits alone and interleaved with others."""
import numpy as np
import pytest

import cvgen
from parity import compare, exact
from streams import LATE, arrivals, windows

pytestmark = pytest.mark.gpu

def stream_run(wins, precision=0, stream=None, lateness=LATE, tuning=None):
    import torch

    import paper_2305_07454_b300 as P

    with P.Pipeline(stream=stream, mode=P.STREAM, lateness_ms=lateness, precision=precision) as p:
        if tuning:
            p.tuning = tuning
        for cols, end in wins:
            t = {k: torch.from_numpy(cols[k]).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
            p.push_window(t, end)
        p.flush()
        return p.results()


def expected_drops(wins, lateness=LATE):
    """The watermark rule applied on the host: a record is too late when its timestamp is below
    the watermark left by the previous window."""
    keep = []
    wprev = None
    for cols, end in wins:
        ok = np.ones(cols["ts"].shape[0], bool) if wprev is None else cols["ts"] >= wprev
        keep.append({k: v[ok] for k, v in cols.items()})
        wprev = end - lateness
    return {k: np.concatenate([c[k] for c in keep]) for k in keep[0]}


@pytest.mark.parametrize("split", [0, 512])
def test_stream_equals_batch(orc, small_day, split):
    """Each window's journey fragments are short: with split 512 nearly all of them take the
    64-thread journey kernel, continuing their journeys' state across windows."""
    wins = windows(small_day, arrivals(small_day, 1))
    assert len(wins) > 100
    g = stream_run(wins, tuning=dict(small_journey_max=split))
    o = orc.run({k: np.concatenate([c[k] for c, _ in wins]) for k in small_day})
    assert g["counters"]["n_too_late"] == 0
    compare(g, o, points=False)


def test_stream_with_ids_over_the_full_int64_range(orc, small_day):
    """Journey ids at the ends of int64, -1 (the hash table's empty pattern) and random full-range
    values: each window's id sort covers all the bits the ids span."""
    rng = np.random.default_rng(31)
    ids = np.unique(small_day["jid"])
    extremes = np.array([np.iinfo(np.int64).min, np.iinfo(np.int64).min + 1, -1, 0, 1,
                         np.iinfo(np.int64).max - 1, np.iinfo(np.int64).max], np.int64)
    new = np.concatenate([extremes, rng.integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, ids.shape[0],
                                                 dtype=np.int64)])[: ids.shape[0]]
    assert np.unique(new).shape[0] == ids.shape[0]
    cols = dict(small_day, jid=new[np.searchsorted(ids, small_day["jid"])])
    wins = windows(cols, arrivals(cols, 3))
    g = stream_run(wins)
    o = orc.run({k: np.concatenate([c[k] for c, _ in wins]) for k in cols})
    compare(g, o, points=False)


def test_stream_drops_records_beyond_the_lateness(orc, small_day):
    wins = windows(small_day, arrivals(small_day, 2, late_frac=0.05, max_delay=120000))
    kept = expected_drops(wins)
    g = stream_run(wins)
    n_late = sum(c["ts"].shape[0] for c, _ in wins) - kept["ts"].shape[0]
    assert n_late > 0 and g["counters"]["n_too_late"] == n_late
    o = orc.run(kept)
    g["counters"]["n_in"] -= n_late
    compare(g, o, points=False)


def test_stream_empty_and_late_only_windows(orc, small_day):
    """Windows with no rows (one repeating the previous window's end, one taking the next
    window's end early, which makes part of that window late) and a window whose rows are all
    below the watermark: the tables equal the oracle over the kept rows; drops are counted."""
    wins = windows(small_day, arrivals(small_day, 4))
    empty = {k: v[:0].copy() for k, v in wins[0][0].items()}
    late = {k: v[:40].copy() for k, v in wins[5][0].items()}
    seq = []
    for i, (cols, end) in enumerate(wins):
        seq.append((cols, end))
        if i == 10:
            seq.append((empty, end))
        if i == 20:
            seq.append((late, end))
        if i == 30:
            seq.append((empty, wins[i + 1][1]))
    kept = expected_drops(seq)
    n_late = sum(c["ts"].shape[0] for c, _ in seq) - kept["ts"].shape[0]
    g = stream_run(seq)
    assert n_late > 40 and g["counters"]["n_too_late"] == n_late
    o = orc.run(kept)
    g["counters"]["n_in"] -= n_late
    compare(g, o, points=False)


def test_stream_float32_form(orc, small_day):
    import paper_2305_07454_b300 as P

    wins = windows(small_day, arrivals(small_day, 3))
    g = stream_run(wins, precision=P.FP32)
    o = orc.run({k: np.concatenate([c[k] for c, _ in wins]) for k in small_day})
    compare(g, o, points=False, rel=1e-4)


def test_each_stream_is_the_same_alone_and_in_the_mix():
    import torch

    import paper_2305_07454_b300 as P

    days = [cvgen.generate(cvgen.params("small_day", seed=s, n_journeys=300)) for s in (11, 12, 13)]
    wins = [windows(d, arrivals(d, s)) for s, d in zip((11, 12, 13), days)]
    alone = [stream_run(w) for w in wins]
    # interleaved: three contexts on three CUDA streams, windows pushed round-robin
    streams = [torch.cuda.Stream() for _ in wins]
    pipes = [P.Pipeline(stream=s, mode=P.STREAM, lateness_ms=LATE) for s in streams]
    pos = [0, 0, 0]
    while any(pos[i] < len(wins[i]) for i in range(3)):
        for i in range(3):
            if pos[i] < len(wins[i]):
                cols, end = wins[i][pos[i]]
                with torch.cuda.stream(streams[i]):
                    t = {k: torch.from_numpy(cols[k]).cuda(non_blocking=False) for k in ("jid", "ts", "lat", "lon", "speed")}
                streams[i].synchronize()
                pipes[i].push_window(t, end)
                pos[i] += 1
    mixed = []
    for p in pipes:
        p.flush()
        mixed.append(p.results())
        p.close()
    for a, m in zip(alone, mixed):
        assert a["counters"] == m["counters"]
        for part in ("cells", "journeys"):
            for k in a[part]:
                exact(f"{part} {k}", m[part][k], a[part][k])


def test_stream_call_order_and_errors(small_day):
    import torch

    import paper_2305_07454_b300 as P

    wins = windows(small_day, arrivals(small_day, 4))[:3]
    with P.Pipeline(mode=P.STREAM) as p:
        t = {k: torch.from_numpy(wins[1][0][k]).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
        p.push_window(t, wins[1][1])
        t0 = {k: torch.from_numpy(wins[0][0][k]).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
        with pytest.raises(P.CvetlError) as e:
            p.extract(t0, wins[0][1])  # out of order
        assert e.value.status == P.EINVAL
        p.flush()
        with pytest.raises(P.CvetlError) as e:
            p.extract(t, wins[2][1])
        assert e.value.status == P.ESTATE
    with P.Pipeline() as p:
        with pytest.raises(P.CvetlError) as e:
            p.flush()
        assert e.value.status == P.ESTATE


def test_stream_memory_admission(small_day):
    import torch

    import paper_2305_07454_b300 as P

    wins = windows(small_day, arrivals(small_day, 5))
    big = {k: np.concatenate([c[k] for c, _ in wins]) for k in small_day}
    with P.Pipeline(mode=P.STREAM, mem_budget_bytes=4 << 20) as p:
        t = {k: torch.from_numpy(big[k]).cuda() for k in ("jid", "ts", "lat", "lon", "speed")}
        with pytest.raises(P.CvetlError) as e:
            p.extract(t, wins[-1][1])
        assert e.value.status == P.EFULL
