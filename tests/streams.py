"""Replaying a day of records as arrival windows, for the stream-mode and server tests: each
record arrives at its timestamp, a fraction of them later by a uniform delay; windows are the
60 s arrival intervals, records inside a window in input order (the day is shuffled)."""
import numpy as np

T0 = 1620518400000
LATE = 30000


def arrivals(cols, seed, late_frac=0.02, max_delay=30000):
    rng = np.random.default_rng(seed)
    n = cols["jid"].shape[0]
    delay = np.zeros(n, np.int64)
    k = rng.random(n) < late_frac
    delay[k] = rng.integers(1, max_delay + 1, int(k.sum()))
    return cols["ts"] + delay


def windows(cols, arrival, width=60000):
    """[(columns of the window, window end ms)] in arrival order."""
    w = (arrival - T0) // width
    order = np.argsort(w, kind="stable")
    bounds = np.flatnonzero(np.diff(w[order])) + 1
    out = []
    for idx in np.split(order, bounds):
        if idx.size == 0:
            continue
        wid = int(w[idx[0]])
        out.append(({k: np.ascontiguousarray(v[idx]) for k, v in cols.items()}, T0 + (wid + 1) * width))
    return out


def concat(wins):
    return {k: np.concatenate([c[k] for c, _ in wins]) for k in wins[0][0]}


def shard(cols, n_feeds):
    """Journey-hash partition of a day (each journey in exactly one feed)."""
    h = (cols["jid"].astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(40)
    s = (h % np.uint64(n_feeds)).astype(np.int64)
    return [{k: v[s == i] for k, v in cols.items()} for i in range(n_feeds)]


def merge_cells(parts):
    """Cell tables of disjoint journey sets merged by key: counts and sums add, min / max."""
    key = np.concatenate([p["key"] for p in parts])
    order = np.argsort(key, kind="stable")
    key = key[order]
    cat = {k: np.concatenate([p[k] for p in parts])[order] for k in ("row", "col", "bin", "count", "sum", "min", "max")}
    head = np.concatenate([[True], key[1:] != key[:-1]]) if key.size else np.zeros(0, bool)
    seg = np.cumsum(head) - 1
    m = int(head.sum())
    out = {"key": key[head], "row": cat["row"][head], "col": cat["col"][head], "bin": cat["bin"][head]}
    out["count"] = np.bincount(seg, weights=cat["count"], minlength=m).astype(np.uint32)
    out["sum"] = np.bincount(seg, weights=cat["sum"], minlength=m)
    mn = np.full(m, np.inf, np.float32)
    mx = np.full(m, -np.inf, np.float32)
    np.minimum.at(mn, seg, cat["min"])
    np.maximum.at(mx, seg, cat["max"])
    out["min"], out["max"] = mn, mx
    out["mean"] = out["sum"] / out["count"]
    return out


def merge_journeys(parts):
    j = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    order = np.argsort(j["id"], kind="stable")
    j = {k: v[order] for k, v in j.items()}
    j["offset"] = np.concatenate([[0], np.cumsum(j["n"])[:-1]]).astype(np.int64) if j["n"].size else j["n"]
    return j
