"""Benchmark of the full-day connected-vehicle ETL on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload full_day] [--impl ours|reference]

One step = extract -> transform -> load -> results over one day of synthetic, fully shuffled
records (60k journeys, ~150M records; the statewide-shaped generator stands in for the
Missouri DOT data, which is not available). The device-resident number (`value`) times
steps whose inputs are already in HBM; `e2e` times the same calls with pinned host inputs,
the host->device copy and the read-back of the result tables inside the timed region.
Prints one JSON line (rank 0).

The serving leg (`serving` in the line; --serve-feeds 0 skips it) replays the same day as
one-minute arrival windows (2% of records up to 30 s late, so none is too late for the 30 s
lateness) through the library's server: the day is split into journey-hash feeds, each window
into one request per feed, FP32 form. "paced" submits a minute's requests only after the
previous minute has completed (the GPU is idle when a window arrives, as under real-time
60 s pacing; every latency is far below 60 s); "max_rate" submits the whole day at once.
Window latency = the last request's completion - the first request's submission. The served
tables are compared with the batch tables of the same day.

--impl reference times the plain CPU oracle (the reference of this build) on the host, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CV records/s & % HBM roofline, full-day ETL; p50/p99 window latency"
UNIT = "records/s"
COLS = ("jid", "ts", "lat", "lon", "speed")
BYTES = {"jid": 8, "ts": 8, "lat": 8, "lon": 8, "speed": 4}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def over_ranks(maxes, sums, world: int, device="cpu"):
    """The job's figures over the ranks of a replica run: the largest of each value in `maxes`
    (times: the slowest rank decides) and the total of each value in `sums` (records). One
    process per GPU; the process group (NCCL on GPUs, gloo on CPU) is already initialised."""
    maxes, sums = [float(v) for v in maxes], [int(v) for v in sums]
    if world == 1:
        return maxes, sums
    import torch
    import torch.distributed as dist

    tm = torch.tensor(maxes, dtype=torch.float64, device=device)
    ts = torch.tensor(sums, dtype=torch.int64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return [float(v) for v in tm.tolist()], [int(v) for v in ts.tolist()]


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_workload(name: str, seed: int, pinned: bool):
    import torch

    import cvgen

    p = cvgen.params(name, seed=seed)
    n = cvgen.count(p)
    dt = {"jid": torch.int64, "ts": torch.int64, "lat": torch.float64, "lon": torch.float64,
          "speed": torch.float32, "heading": torch.float32}
    host = {k: torch.empty(n, dtype=v, pin_memory=pinned) for k, v in dt.items()}
    cvgen.generate(p, out={k: v.numpy() for k, v in host.items()})
    return host, n, int(p.n_journeys)


def algorithmic_bytes(stage: str, c: dict) -> float:
    """Bytes a stage must move per launch, from the counters."""
    nin, nv, J, R = c["n_in"], c["n_valid"], c["n_journeys"], c["n_runs"]
    return {
        "hash_count": 28.0 * nin + 4.0 * nin,           # jid, lat, lon, speed read; row slot written
        "scatter": 32.0 * nin + 32.0 * nv,              # ts, lat, lon, speed, slot read; records written
        "journeys": 32.0 * nv + 28.0 * R + 96.0 * J,    # records read; runs and journey rows written
        "cell_write": 28.0 * R + 44.0 * c["n_cells"],
        "csv_count": float(c.get("csv_bytes", 0)),                  # the text read
        "csv_parse": float(c.get("csv_bytes", 0)) + 40.0 * nin,    # the text read; six columns written
    }.get(stage, 0.0)


# binary64 operations per point of the journey kernel: the cosine of the latitude (2: offset from
# the table point, one fma), the distance (10: two differences, two squares, the cosine product,
# one fma, the scaled square root and its residual, the scaling, the final fma), the journey
# distance sum (1) and the implied speed's rounding to float32 (1)
FP64_OPS_PER_POINT = 14.0
SMS, FP64_PER_CLK_PER_SM = 148, 2.0


def fp64_peak_gops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", 2032.0))
    except Exception:
        mhz = 2032.0
    return SMS * FP64_PER_CLK_PER_SM * mhz / 1e3, mhz


# Per-pass DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per record of a stage,
# from one ncu capture of the tenth-day workload (14,637,283 records) with the kernels as they
# stand, scaled by records to the workload's pass (the full day is too large to capture under
# the profiler's size rule); FP64 form, column or CSV input. The journeys entry adds its two
# kernel shapes (256- and 64-thread CTAs). Empty a stage's entry when its kernels change, until
# they are captured again.
TRAFFIC_PER_RECORD = {
    "journeys": (827.050496e6 + 68.221696e6 + 3.345408e6 + 0.0) / 14637283,
    "scatter": (468.913152e6 + 428.840448e6) / 14637283,
    "hash_count": (410.996736e6 + 48.926464e6) / 14637283,
    "csv_parse": (856.018944e6 + 549.557760e6) / 14637283,
}


def unit_launches(stage, launches, steps):
    """Number of passes over the stage's algorithmic work in `launches`. Every stage's launch is
    one pass, except the journeys stage: its two kernel shapes (journeys of up to 512 points in
    64-thread CTAs, the rest in 256-thread CTAs) share one pass over all points per step, so its
    time per pass is the sum of both launches."""
    if stage == "journeys":
        return max(1, steps)
    return max(1, launches)


def run_ours(args):
    import torch

    import paper_2305_07454_b300 as P

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    host, n, J = make_workload(args.workload, seed=1 + rank, pinned=True)
    csv_host = None
    if args.input == "csv":
        import cvgen

        text, _ = cvgen.to_csv({k: host[k].numpy() for k in host}, seed=1 + rank, malformed_frac=0.005)
        csv_host = torch.from_numpy(text).pin_memory()
        d_csv = csv_host.to(dev, non_blocking=True)
    d_in = {k: host[k].to(dev, non_blocking=True) for k in COLS + ("heading",)}
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def extract_dev(p):
        if csv_host is None:
            p.extract(d_in)
        else:
            p.extract_csv(d_csv)

    def run_dev(p):
        extract_dev(p)
        p.transform()
        p.load()
        return p.results(to_host=False)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident steps ------------------------------------------------------------
    prec = P.FP32 if args.precision == "fp32" else P.FP64
    pipe = P.Pipeline(stream=stream, precision=prec)
    # launch shapes from the library's autotuner on this workload (outside the timed region)
    extract_dev(pipe)
    t_tune = time.perf_counter()
    tuning = pipe.autotune(reps=2) if args.autotune else {**pipe.tuning, "ms": None}
    tuning["seconds"] = time.perf_counter() - t_tune
    for _ in range(args.warmup):
        run_dev(pipe)
    pipe.stats_reset()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            extract_dev(pipe)
            pipe.transform()
            pipe.load()
            pipe.tables()  # reads the sizes and counters back (synchronises the stream)
        ev1.record(stream)
        barrier()
    ms_total = ev0.elapsed_time(ev1)
    # per-kernel times from CUDA events around every launch, taken on a second pipeline with the
    # same launch shapes over as many steps (the events' own cost stays out of the timed steps)
    prof = P.Pipeline(stream=stream, profile=1, precision=prec)
    prof.tuning = {k: v for k, v in tuning.items() if k not in ("ms", "seconds")}
    run_dev(prof)  # first use of the shapes
    prof.stats_reset()
    for _ in range(args.steps):
        extract_dev(prof)
        prof.transform()
        prof.load()
        prof.tables()
    stats = prof.stats()
    prof.close()
    t = pipe.tables()
    counters = {k: int(getattr(t, k)) for k in ("n_in", "n_malformed", "n_valid", "n_out_of_grid",
                                                 "n_dup", "n_runs")}
    counters.update(n_journeys=int(t.n_journeys), n_cells=int(t.n_cells))
    if csv_host is not None:
        counters["csv_bytes"] = int(csv_host.numel())
    (ms_total,), (n_job,) = over_ranks([ms_total], [n], world, dev)
    ms_step = ms_total / args.steps
    value = n_job * args.steps / (ms_total / 1e3)

    # ---- end to end through the C ABI with host inputs ------------------------------------
    # Two pipelines, each on its own stream and host thread (the library calls release the
    # GIL), take alternate steps: one step's host->device copy of its pinned inputs overlaps
    # the other's kernels and result read-back. Every step copies its inputs and reads its
    # tables back into pinned host buffers inside the timed region.
    import threading

    e2e_per_pipe = max(1, min(args.steps, 3))
    pipes_h = [P.Pipeline(stream=torch.cuda.Stream(device=dev), precision=prec) for _ in range(2)]
    host_outs = [ph.host_tables(cells=counters["n_cells"], journeys=counters["n_journeys"]) for ph in pipes_h]
    last = [None, None]

    def run_host(i):
        ph = pipes_h[i]
        if csv_host is None:
            ph.extract({k: host[k] for k in COLS})
        else:
            ph.extract_csv(csv_host)
        ph.transform()
        ph.load()
        last[i] = ph.results(to_host=True, out=host_outs[i])

    for i in range(2):
        run_host(i)
    barrier()
    errors = []

    def worker(i):
        try:
            for _ in range(e2e_per_pipe):
                run_host(i)
        except Exception as exc:  # reported after the join
            errors.append(exc)

    t0 = time.perf_counter()
    threads = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    barrier()
    e2e_s = (time.perf_counter() - t0) / (2 * e2e_per_pipe)
    if errors:
        raise errors[0]
    (e2e_s,), _ = over_ranks([e2e_s], [], world, dev)
    out = last[0]
    h2d = sum(BYTES[k] for k in COLS) * n if csv_host is None else int(csv_host.numel())
    d2h = sum(v.nbytes for part in ("cells", "journeys") for v in out[part].values()) + 8 * 6
    for ph in pipes_h:
        ph.close()

    # the 8-channel lattice of the day (5-minute bins, dense [288, 8, 460, 670] float32 tensor)
    lat_ms = []
    for i in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L = pipe.lattice(to_host=False, dense=1, normalize=1)
        e1.record(stream)
        torch.cuda.synchronize()
        if i:
            lat_ms.append(e0.elapsed_time(e1))
    lattice = {"ms": statistics.median(lat_ms), "cells": int(L["cells"]["key"].shape[0]),
               "dense_shape": list(L["dense"].shape), "dropped": L["n_dropped"],
               "records_per_s": counters["n_valid"] / (statistics.median(lat_ms) / 1e3),
               "what": "after load: 5-minute bins x 4 cardinal directions x cells; mean speed and unique journeys, "
                       "min-max normalised, dense tensor written"}
    del L
    # ---- roofline of the dominant kernel ---------------------------------------------------
    stages = stats["stages"]
    top = max(stages, key=lambda s: stages[s]["ms"])
    avg_ms = stages[top]["ms"] / unit_launches(top, stages[top]["launches"], args.steps)
    hbm_peak, peak_src = load_peaks()
    tpr = TRAFFIC_PER_RECORD.get(top) if args.precision != "fp32" else None
    traffic = tpr * counters["n_valid"] if tpr else None
    if top == "journeys" and args.precision == "fp64":
        gops_peak, mhz = fp64_peak_gops()
        ops = FP64_OPS_PER_POINT * counters["n_valid"]
        achieved = ops / (avg_ms / 1e3) / 1e9
        roofline = {"bound": "alu", "kernel": top, "achieved": achieved, "peak": gops_peak,
                    "unit": "G binary64 ops/s",
                    "peak_source": f"derived: {SMS} SMs x {FP64_PER_CLK_PER_SM:g} binary64 ops/clk x {mhz:g} MHz",
                    "frac": achieved / gops_peak, "ops_per_launch": ops, "avg_launch_ms": avg_ms,
                    "traffic": traffic,
                    "hbm_achieved_gbs": algorithmic_bytes(top, counters) / (avg_ms / 1e3) / 1e9}
    else:
        ab = algorithmic_bytes(top, counters)
        achieved = ab / (avg_ms / 1e3) / 1e9 if ab else None
        roofline = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": hbm_peak,
                    "peak_source": peak_src, "unit": "GB/s",
                    "frac": (achieved / hbm_peak) if achieved else None,
                    "algorithmic_bytes_per_launch": ab, "avg_launch_ms": avg_ms, "traffic": traffic}
    step_bytes = sum(algorithmic_bytes(s, counters) * unit_launches(s, v["launches"], args.steps) / args.steps
                     for s, v in stages.items() if v["launches"])
    hbm_step = {"algorithmic_bytes_per_step": step_bytes,
                "achieved": step_bytes / (ms_step / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": step_bytes / (ms_step / 1e3) / 1e9 / hbm_peak}
    shares = {s: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps}
              for s, v in stages.items() if v["launches"]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32 (binary64 coordinate differences)",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {J} journeys, {n} records, one day, "
                               + ("binary columns" if csv_host is None else
                                  f"CSV text ({int(csv_host.numel())} bytes, 0.5% malformed rows)")
                               + ", fully shuffled", "records": n, "journeys": J, "input": args.input, "precision": args.precision,
                   "l2": "inputs larger than L2 (no flush needed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   **({"records_all_ranks": n_job} if world > 1 else {})},
        "e2e": {"value": n_job / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "pipelines": 2},
        "gpu_launches": stats["total_launches"],
        "tuning": tuning,
        "roofline": roofline,
        "hbm_step": hbm_step,
        "stages": shares,
        "counters": counters,
        "lattice": lattice,
        "clocks": clk.summary(),
    }
    if args.serve_feeds > 0:
        batch_cells = pipe.results(to_host=True)["cells"]
        line["serving"] = serving(host, n, args, batch_cells, ms_step)
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(host, n, budget_s=args.cpu_budget)
        print(json.dumps(line), flush=True)
    pipe.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _window_order(host, n, feeds, t0, seed=7):
    """Row order of the replay: by arrival minute, then feed (journey hash), input order inside."""
    ts = host["ts"].numpy()
    rng = np.random.default_rng(seed)
    late = rng.random(n) < 0.02
    arrival = ts.copy()
    arrival[late] += rng.integers(1, 30001, int(late.sum()))
    w = (arrival - t0) // 60000
    del arrival, late
    h = (host["jid"].numpy().astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(40)
    key = w * feeds + (h % np.uint64(feeds)).astype(np.int64)
    # 16-bit keys take numpy's radix sort
    key = key.astype(np.int16 if int(key.max()) < 32767 else np.int32)
    order = np.argsort(key, kind="stable")
    n_win = int(w.max()) + 1
    bounds = np.searchsorted(key[order], np.arange(n_win * feeds + 1))
    return order, bounds, n_win


def _replay(P, cols, bounds, n_win, feeds, t0, slots, budget, paced, upto=None):
    """One replay through a fresh server; returns (per-window latency ms, per-request service ms,
    seconds from the first submission to the last completion, feed results)."""
    upto = n_win if upto is None else upto
    with P.Server(n_slots=slots, mem_budget_bytes=budget) as srv:
        ids = [srv.add_feed(precision=P.FP32, lateness_ms=30000) for _ in range(feeds)]

        def submit(m):
            out = []
            for f in range(feeds):
                a, b = int(bounds[m * feeds + f]), int(bounds[m * feeds + f + 1])
                out.append(srv.submit(ids[f], {k: cols[k][a:b] for k in COLS}, t0 + (m + 1) * 60000))
            return out

        win = []
        if paced:
            for m in range(upto):
                win.append([srv.wait(t) for t in submit(m)])
        else:
            tickets = [submit(m) for m in range(upto)]
            win = [[srv.wait(t) for t in ts] for ts in tickets]
        fl = [srv.wait(srv.submit_flush(f)) for f in ids]
        first = min(i["submit_ns"] for w in win for i in w)
        last = max(i["done_ns"] for i in fl)
        lat = [(max(i["done_ns"] for i in w) - min(i["submit_ns"] for i in w)) / 1e6 for w in win]
        svc = [(i["done_ns"] - i["start_ns"]) / 1e6 for w in win for i in w]  # per request
        res = [srv.feed(f).results(to_host=True) for f in ids]
        peak = max(i["peak_in_flight"] for i in fl)
    return lat, svc, (last - first) / 1e9, res, peak


def _merged_cells(res):
    parts = [r["cells"] for r in res]
    key = np.concatenate([p["key"] for p in parts])
    order = np.argsort(key, kind="stable")
    key = key[order]
    head = np.flatnonzero(np.concatenate([[True], key[1:] != key[:-1]])) if key.size else np.zeros(0, np.int64)
    cat = lambda k: np.concatenate([p[k] for p in parts])[order]
    return {"key": key[head],
            "count": np.add.reduceat(cat("count").astype(np.int64), head) if key.size else np.zeros(0, np.int64),
            "sum": np.add.reduceat(cat("sum"), head) if key.size else np.zeros(0),
            "min": np.minimum.reduceat(cat("min"), head) if key.size else np.zeros(0, np.float32),
            "max": np.maximum.reduceat(cat("max"), head) if key.size else np.zeros(0, np.float32)}


def serving(host, n, args, batch_cells, batch_ms):
    """The serving leg: the day replayed through the server, paced and at maximum rate."""
    import torch

    import paper_2305_07454_b300 as P

    t0 = int(P.default_config().t0_ms)
    feeds, slots = args.serve_feeds, args.serve_slots or args.serve_feeds
    budget = int(args.serve_budget_gb * (1 << 30))
    order, bounds, n_win = _window_order(host, n, feeds, t0)
    cols = {k: torch.empty(n, dtype=host[k].dtype, pin_memory=True) for k in COLS}
    for k in COLS:
        np.take(host[k].numpy(), order, out=cols[k].numpy())
    del order
    _replay(P, cols, bounds, n_win, feeds, t0, slots, budget, paced=True, upto=90)  # loads the kernels
    pct = lambda v, q: float(np.percentile(np.asarray(v), q))
    out = {"workload": f"the batch day replayed as {n_win} one-minute arrival windows, 2% of records "
                       f"up to 30 s late, {feeds} journey-hash feeds, FP32 form",
           "windows": n_win, "feeds": feeds, "slots": slots, "mem_budget_bytes": budget,
           "records": n, "batch_fp64_ms_per_day": batch_ms}
    sizes = np.diff(bounds[::feeds][: n_win + 1]) if feeds else []
    out["window_records"] = {"min": int(np.min(sizes)), "p50": int(np.median(sizes)), "max": int(np.max(sizes))}
    for mode, paced in (("paced", True), ("max_rate", False)):
        lat, svc, secs, res, peak = _replay(P, cols, bounds, n_win, feeds, t0, slots, budget, paced)
        out[mode] = {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "max_ms": max(lat),
                     "service_p50_ms": pct(svc, 50), "service_p99_ms": pct(svc, 99),
                     "records_per_s": n / secs, "seconds": secs, "peak_in_flight": peak}
        if paced:
            c = {k: sum(r["counters"][k] for r in res) for k in ("n_in", "n_too_late", "n_valid")}
            m = _merged_cells(res)
            b = batch_cells
            same = (m["key"].shape == b["key"].shape and np.array_equal(m["key"], b["key"])
                    and np.array_equal(m["count"], b["count"].astype(np.int64))
                    and np.array_equal(m["min"], b["min"]) and np.array_equal(m["max"], b["max"]))
            rel = float(np.max(np.abs(m["sum"] - b["sum"]) / np.maximum(np.abs(b["sum"]), 1e-300))) if same and b["sum"].size else None
            out["vs_batch"] = {"counters": c, "keys_counts_min_max_equal": bool(same),
                               "cell_sum_max_rel_err": rel}
    return out


def _roofline(stages, counters, precision, n_steps_div=1.0):
    """Roofline entry of the dominant kernel from per-stage CUDA-event times (per step)."""
    top = max(stages, key=lambda k: stages[k]["ms"])
    avg_ms = stages[top]["ms"] / unit_launches(top, stages[top]["launches"], 1)
    hbm_peak, peak_src = load_peaks()
    if top == "journeys" and precision == "fp64":
        gops_peak, mhz = fp64_peak_gops()
        ops = FP64_OPS_PER_POINT * counters["n_valid"]
        achieved = ops / (avg_ms / 1e3) / 1e9
        return {"bound": "alu", "kernel": top, "achieved": achieved, "peak": gops_peak,
                "unit": "G binary64 ops/s",
                "peak_source": f"derived: {SMS} SMs x {FP64_PER_CLK_PER_SM:g} binary64 ops/clk x {mhz:g} MHz",
                "frac": achieved / gops_peak, "ops_per_launch": ops, "avg_launch_ms": avg_ms, "traffic": None}
    ab = algorithmic_bytes(top, counters)
    achieved = ab / (avg_ms / 1e3) / 1e9 if ab else None
    return {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": hbm_peak, "peak_source": peak_src,
            "unit": "GB/s", "frac": (achieved / hbm_peak) if achieved else None,
            "algorithmic_bytes_per_launch": ab, "avg_launch_ms": avg_ms, "traffic": None}


def _max_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size == 0:
        return 0.0
    d = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    d[(a == 0) & (b == 0)] = 0.0
    return float(d.max())


def run_week(args):
    """The batched workload: 7 days x 4 regional boxes in one batch (one pass of every kernel,
    launch shapes from the autotuner, the post-sizing sequence replayed as a CUDA graph)."""
    import torch

    import cvgen
    import paper_2305_07454_b300 as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = args.precision or "fp32"
    recipes = cvgen.week_regions(seed=1 + rank, scale=args.scale)
    t_gen = time.perf_counter()
    host, grids = [], []
    dt = {"jid": torch.int64, "ts": torch.int64, "lat": torch.float64, "lon": torch.float64,
          "speed": torch.float32, "heading": torch.float32}
    for r in recipes:
        n_i = cvgen.count(r["params"])
        h = {k: torch.empty(n_i, dtype=v, pin_memory=True) for k, v in dt.items()}
        cvgen.generate(r["params"], out={k: v.numpy() for k, v in h.items()})
        host.append(h)
        grids.append({k: r[k] for k in P.GRID_KEYS})
    t_gen = time.perf_counter() - t_gen
    n = sum(h["jid"].shape[0] for h in host)
    d_insts = [dict(g, **{k: h[k].to(dev, non_blocking=True) for k in COLS}) for g, h in zip(grids, host)]
    h_insts = [dict(g, **{k: h[k] for k in COLS}) for g, h in zip(grids, host)]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    pc = P.FP32 if prec == "fp32" else P.FP64

    # per-stage times of one eager run (profiled), and the FP64 form for the error report
    with P.Pipeline(stream=stream, precision=pc, profile=1) as pe:
        pe.extract_batch(d_insts)
        tune_t = time.perf_counter()
        tuning = pe.autotune(reps=2)
        tune_t = time.perf_counter() - tune_t
        pe.transform()
        pe.load()
        pe.stats_reset()
        pe.extract_batch(d_insts)
        pe.transform()
        pe.load()
        stats = pe.stats()
        res = pe.results(to_host=True)
        t = pe.tables()
    counters = {k: int(getattr(t, k)) for k in ("n_in", "n_malformed", "n_valid", "n_out_of_grid", "n_dup", "n_runs")}
    counters.update(n_journeys=int(t.n_journeys), n_cells=int(t.n_cells))
    errors = None
    if pc == P.FP32:
        with P.Pipeline(stream=stream, precision=P.FP64) as p64:
            p64.extract_batch(d_insts)
            p64.transform()
            p64.load()
            ref = p64.results(to_host=True)
        same_int = all(np.array_equal(res["cells"][k], ref["cells"][k]) for k in ("key", "count", "min", "max")) and \
            all(np.array_equal(res["journeys"][k], ref["journeys"][k]) for k in ("id", "n", "start_ts", "end_ts", "dwell_ms"))
        errors = {"integers_keys_counts_min_max_equal": bool(same_int),
                  "journey_distance_max_rel": _max_rel(res["journeys"]["distance_m"], ref["journeys"]["distance_m"]),
                  "cell_sum_max_rel": _max_rel(res["cells"]["sum"], ref["cells"]["sum"]),
                  "cell_mean_max_rel": _max_rel(res["cells"]["mean"], ref["cells"]["mean"])}
        del ref
    del res

    # timed: graph replays of the tuned shapes
    pipe = P.Pipeline(stream=stream, precision=pc, graph=1)
    pipe.tuning = {k: v for k, v in tuning.items() if k != "ms"}

    def step(insts):
        pipe.extract_batch(insts)
        pipe.transform()
        pipe.load()
        pipe.tables()

    for _ in range(max(args.warmup, 2)):
        step(d_insts)
    pipe.stats_reset()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step(d_insts)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    gst = pipe.stats()
    ms_step = ms_total / args.steps
    value = n / (ms_step / 1e3)
    # end to end from pinned host columns
    e2e_steps = max(1, min(args.steps, 2))
    step(h_insts)
    t = pipe.tables()
    host_out = pipe.host_tables(cells=int(t.n_cells), journeys=int(t.n_journeys))
    pipe.results(to_host=True, out=host_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(h_insts)
        out = pipe.results(to_host=True, out=host_out)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    d2h = sum(v.nbytes for part in ("cells", "journeys") for v in out[part].values())
    pipe.close()
    stages = stats["stages"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 2), "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "f32 (binary64 coordinate differences)",
        "data": "synthetic",
        "config": {"workload": f"week_regions x{args.scale:g}: {len(recipes)} instances (7 days x 4 regional "
                               f"boxes), {n} records, {counters['n_journeys']} journeys, Zipf(1.5) journey "
                               "lengths on [10, 200000], one batch",
                   "records": n, "instances": len(recipes), "precision": prec, "scale": args.scale,
                   "instance_records": [int(h["jid"].shape[0]) for h in host],
                   "l2": "inputs larger than L2 (no flush needed)", "parallelism": "1 GPU"},
        "tuning": {**tuning, "seconds": tune_t},
        "graph": {"replays_in_timed_steps": gst["graph_replays"], "launches_per_step": gst["total_launches"] / args.steps},
        "e2e": {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": n * sum(BYTES[k] for k in COLS),
                "d2h_bytes_per_step": d2h},
        "gpu_launches": gst["total_launches"],
        "roofline": _roofline(stages, counters, prec),
        "stages": {k: {"ms_per_step": v["ms"], "launches_per_step": v["launches"]} for k, v in stages.items() if v["launches"]},
        "errors_vs_fp64_form": errors,
        "counters": counters,
        "generation_s": t_gen,
        "clocks": clk.summary(),
    }
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline({k: host[0][k] for k in COLS}, int(host[0]["jid"].shape[0]), budget_s=args.cpu_budget)
        print(json.dumps(line), flush=True)


def _sample_journeys(host, frac_den: int):
    """Whole journeys: the records whose journey id falls in 1 of frac_den hash classes."""
    jid = host["jid"].numpy() if hasattr(host["jid"], "numpy") else host["jid"]
    h = (jid.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(40)
    sel = np.flatnonzero((h % np.uint64(frac_den)) == 0)
    return {k: (host[k].numpy() if hasattr(host[k], "numpy") else host[k])[sel] for k in COLS}


def cpu_baseline(host, n, budget_s=15.0):
    import oracle

    o = oracle.get()
    den = 64
    sample = _sample_journeys(host, den)
    t0 = time.perf_counter()
    o.run(sample)
    dt = time.perf_counter() - t0
    # grow the sample toward the budget (about 10-30 s of CPU work)
    while dt < budget_s / 4 and den > 4:
        den //= 2
        sample = _sample_journeys(host, den)
        t0 = time.perf_counter()
        o.run(sample)
        dt = time.perf_counter() - t0
    m = sample["jid"].shape[0]
    return {"value": m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"whole journeys with id hash in 1 of {den} classes: {m} records, "
                      f"{len(np.unique(sample['jid']))} journeys, {dt:.1f} s single-threaded",
            "cpu": _cpu_model()}


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip() + f" ({os.cpu_count()} threads online)"
    except Exception:
        pass
    return None


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import cvgen
    import oracle

    o = oracle.get()
    p = cvgen.params(args.workload, seed=1)
    n = cvgen.count(p)
    host = cvgen.generate(p)
    den = 32 if n > 10_000_000 else 1
    sample = _sample_journeys(host, den)
    m = sample["jid"].shape[0]
    for _ in range(args.warmup):
        o.run(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.run(sample)
    dt = (time.perf_counter() - t0) / args.steps
    value = m / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {int(p.n_journeys)} journeys, {n} records, one day, "
                               "binary columns, fully shuffled", "records": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"whole journeys with id hash in 1 of {den} classes: {m} records per step",
                         "cpu": _cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="full_day")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--input", default="columns", choices=["columns", "csv"])
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"],
                    help="fp64 for the day workloads, fp32 for week_regions unless given")
    ap.add_argument("--scale", type=float, default=0.25, help="week_regions: instance size factor")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--serve-feeds", type=int, default=4, help="0 skips the serving leg")
    ap.add_argument("--autotune", type=int, default=1,
                    help="0 keeps the library's default launch shapes (a fixed launch order for ncu)")
    ap.add_argument("--serve-slots", type=int, default=0, help="server slots (default: one per feed)")
    ap.add_argument("--serve-budget-gb", type=float, default=8.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "week_regions":
        run_week(args)
    else:
        args.precision = args.precision or "fp64"
        run_ours(args)


if __name__ == "__main__":
    main()
