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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CV records/s & % HBM roofline, full-day ETL; p50/p99 window latency"
UNIT = "records/s"
COLS = ("jid", "ts", "lat", "lon", "speed")
L2_BYTES = 126 * 2**20
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
        fd, self.path = tempfile.mkstemp(prefix="cvetl_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
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
        if getattr(self, "_summary", None) is not None:
            return self._summary
        try:
            rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.strip()]
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        self._summary = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                         "reasons": reasons, "samples": len(rows)}
        return self._summary


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


FUSED_MIN_POINTS = 8193  # journeys of this many points and more take the fused journey kernel


def algorithmic_bytes(stage: str, c: dict) -> float:
    """Bytes a stage must move per launch, from the counters. The journey stage splits by size:
    journeys above 8192 points (n_fused points, j_fused journeys) in the fused kernel, the
    others (n_walk points) ordered by the class sort and walked."""
    nin, nv, J, R = c["n_in"], c["n_valid"], c["n_journeys"], c["n_runs"]
    nf, jf = c.get("n_fused", 0), c.get("j_fused", 0)
    nw = nv - nf
    return {
        "hash_count": 28.0 * nin + 4.0 * nin,           # jid, lat, lon, speed read; row slot written
        "scatter": 32.0 * nin + 32.0 * nv,              # ts, lat, lon, speed, slot read; records written
        "journeys": 32.0 * nf + 96.0 * jf,              # records read; journey rows written (its runs: below)
        "journey_sort": 10.0 * nw,                      # timestamps read, u16 ordered positions written
        "journey_walk": 34.0 * nw + 28.0 * R + 96.0 * (J - jf),  # records and positions read; runs, journeys written
        "cell_write": 28.0 * R + 44.0 * c["n_cells"],
        "csv_count": float(c.get("csv_bytes", 0)),                  # the text read
        "csv_parse": float(c.get("csv_bytes", 0)) + 40.0 * nin,    # the text read; six columns written
    }.get(stage, 0.0)


# binary64 operations per point of the journey kernels: the cosine of the latitude (2: offset from
# the table point, one fma) and the distance (3: two coordinate differences and the final sum of
# a float32 pair; the squares, products, square root and scaling run on float32 pairs); the
# journey distance is summed in integer fixed point and the implied speed is the float32
# rounding of the pair, off the binary64 pipe
FP64_OPS_PER_POINT = 5.0
SMS = 148

# Bytes per record the method must move (the algorithmic floor: read the needed input once,
# reorder it once, keep kinematics and keys in registers), binary columns; CSV text adds its
# bytes read and the columns written
CONTRACT_BYTES_PER_RECORD = 108.0
CONTRACT_CSV_EXTRA_PER_RECORD = 100.0


def fp64_probe(stream, reps=3):
    """The measured binary64 roof: the library's issue-rate probe (8 independent chains per
    thread, 1,184 CTAs of 256 threads, about 20 ms per launch) timed with CUDA events on the
    stream, best of `reps` per kind. Returns G ops/s per kind, and ops per clock per SM at the
    SM clock sampled while the probes ran."""
    import torch

    import paper_2305_07454_b300 as P

    blocks, threads = SMS * 8, 256
    sink = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    kinds = {"fma": P.PROBE_FMA, "add": P.PROBE_ADD, "mul": P.PROBE_MUL, "mix": P.PROBE_MIX}
    out = {}
    with Clocks(torch.cuda.current_device()) as clk:
        for name, kind in kinds.items():
            iters = 600 if kind == P.PROBE_MIX else 6000
            P.probe_fp64(kind, blocks, threads, 10, sink, stream)  # load
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ops = P.probe_fp64(kind, blocks, threads, iters, sink, stream)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[name] = ops / (best / 1e3) / 1e9
    cs = clk.summary() or {}
    mhz = cs.get("sm_mhz")
    return {"gops": out, "sm_mhz": mhz,
            "ops_per_clk_per_sm": {k: v * 1e9 / (SMS * mhz * 1e6) for k, v in out.items()} if mhz else None,
            "peak_gops": max(out[k] for k in ("fma", "add", "mul")),
            "how": f"{blocks} CTAs x {threads} threads x 8 independent chains, CUDA events, best of {reps}; "
                   "peak = the fastest single operation kind"}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per step and per kept record of
# every stage, from one ncu capture of the tenth-day workload (14,637,283 records) with the
# kernels as they stand: one warm step of each path (binary64 form, float32 form, CSV input),
# scaled by records to the workload (the full day is too large to capture under the profiler's
# size rule). A stage's entry is only valid while its kernels are the ones captured.
TRAFFIC_PER_RECORD = {
    "hash_count": 31.183, "collect_slots": 0.144, "radix_histogram": 0.224, "radix_onesweep": 2.563,
    "journey_sizes": 0.044, "scan": 0.22, "journey_cursors": 0.003, "scatter": 60.987, "journey_sort": 30.096,
    "journeys": 5.048, "journey_walk": 86.278, "cell_heads": 0.214, "cell_write": 1.073,
    # CSV input adds (per kept record of the CSV day)
    "csv_count": 58.654, "csv_parse": 97.572,
}
TRAFFIC_PER_RECORD_FP32 = {
    "hash_count": 31.181, "collect_slots": 0.144, "radix_histogram": 0.224, "radix_onesweep": 2.565,
    "journey_sizes": 0.044, "scan": 0.22, "journey_cursors": 0.003, "scatter": 60.985, "journey_sort": 30.119,
    "journeys": 5.043, "journey_walk": 86.737, "cell_heads": 0.214, "cell_write": 1.073,
}


# The kernel sources the traffic figures above were captured with: sha256 over the files of
# paper_2305_07454_b300/csrc (name and bytes, in name order). When the sources differ, the
# figures describe other kernels: the line then reports no traffic and no gate figure.
TRAFFIC_SOURCES_SHA256 = "6131ae99dabbc1197068a5aac2eb1df811f4306e6b125ea26ea9e21fd3f996a2"


def kernel_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2305_07454_b300", "csrc")
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".cpp", ".h")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def traffic_table(precision: str) -> dict:
    """The ncu DRAM bytes per record of the form's stages, or {} when the kernels have changed
    since they were captured."""
    if kernel_sources_sha256() != TRAFFIC_SOURCES_SHA256:
        return {}
    return TRAFFIC_PER_RECORD if precision == "fp64" else TRAFFIC_PER_RECORD_FP32


def unit_launches(stage, launches, steps):
    """Number of passes over the stage's algorithmic work in `launches`. Every stage's launch is
    one pass, except the journey sort (the class bounds and one launch per size class share one
    pass over the classes' points per step) and the fused journey kernel of stream windows (its
    two shapes share one pass), whose time per pass is the sum of their launches."""
    if stage in ("journeys", "journey_sort"):
        return max(1, steps)
    return max(1, launches)


def _day_steps(P, pipe, extract_dev, steps, warmup, barrier, local):
    """W warm-up steps, then K timed steps (CUDA events on the launching stream, a barrier and a
    device synchronisation on both sides). Returns (ms for the K steps, clock summary)."""
    import torch

    stream = pipe.stream
    for _ in range(warmup):
        extract_dev(pipe)
        pipe.transform()
        pipe.load()
        pipe.tables()
    pipe.stats_reset()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(steps):
            extract_dev(pipe)
            pipe.transform()
            pipe.load()
            pipe.tables()  # reads the sizes and counters back (synchronises the stream)
        ev1.record(stream)
        barrier()
    return ev0.elapsed_time(ev1), clk.summary()


def _stage_stats(P, stream, prec, tuning, extract_dev, steps):
    """Per-kernel times from CUDA events around every launch, taken on a second pipeline with the
    same launch shapes over as many steps (the events' own cost stays out of the timed steps)."""
    prof = P.Pipeline(stream=stream, profile=1, precision=prec)
    prof.tuning = {k: v for k, v in tuning.items() if k not in ("ms", "seconds")}
    extract_dev(prof)
    prof.transform()
    prof.load()
    prof.tables()  # first use of the shapes
    prof.stats_reset()
    for _ in range(steps):
        extract_dev(prof)
        prof.transform()
        prof.load()
        prof.tables()
    stats = prof.stats()
    prof.close()
    return stats


def _hbm_step(stages, counters, ms_step, steps, csv, traffic=None):
    """The step's bytes against the measured copy bandwidth: the method's algorithmic floor
    (CONTRACT_BYTES_PER_RECORD per record; CSV adds its text and columns) and the kernels' own
    byte model (algorithmic_bytes per stage: the passes this implementation makes), and, from the
    ncu DRAM traffic per record of every stage, the gate figure (sum of DRAM bytes over the sum
    of kernel times)."""
    hbm_peak, peak_src = load_peaks()
    n = counters["n_in"]
    contract = n * (CONTRACT_BYTES_PER_RECORD + (CONTRACT_CSV_EXTRA_PER_RECORD if csv else 0.0))
    impl = sum(algorithmic_bytes(s, counters) * unit_launches(s, v["launches"], steps) / steps
               for s, v in stages.items() if v["launches"])
    gbs = lambda b: b / (ms_step / 1e3) / 1e9
    out = {"peak": hbm_peak, "peak_source": peak_src, "unit": "GB/s",
           "contract_bytes_per_step": contract, "contract_bytes_per_record": contract / n if n else None,
           "achieved": gbs(contract), "frac": gbs(contract) / hbm_peak,
           "implementation_bytes_per_step": impl, "implementation_achieved": gbs(impl),
           "implementation_frac": gbs(impl) / hbm_peak}
    timed = {s: v for s, v in stages.items() if v["launches"] and v["ms"] > 0}
    traffic = traffic or {}
    missing = sorted(s for s in timed if s not in traffic)
    if not traffic:
        out["gate"] = None
        out["gate_missing_traffic"] = "no ncu traffic for these kernels (sources changed since the capture)"
    elif missing:
        out["gate"] = None
        out["gate_missing_traffic"] = missing
    else:
        dram = sum(traffic[s] * counters["n_valid"] for s in timed)
        kms = sum(v["ms"] for v in timed.values()) / steps
        out["gate"] = {"dram_bytes_per_step": dram, "kernel_ms_per_step": kms,
                       "achieved": dram / (kms / 1e3) / 1e9, "frac": dram / (kms / 1e3) / 1e9 / hbm_peak,
                       "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per step and record of every "
                                 "stage (tenth-day capture), scaled by records; CUDA-event kernel times"}
    return out


def _roofline_entry(top, stages, counters, steps, precision, probe):
    """Roofline of the dominant stage: the FP64 journey kernel against the measured binary64
    issue rate, any other stage against the measured HBM copy bandwidth."""
    avg_ms = stages[top]["ms"] / unit_launches(top, stages[top]["launches"], steps)
    hbm_peak, peak_src = load_peaks()
    tpr = traffic_table(precision).get(top)
    # per launch (a pass over the stage's work): the step's traffic over the passes per step
    traffic = tpr * counters["n_valid"] / (unit_launches(top, stages[top]["launches"], steps) / steps) if tpr else None
    if top in ("journeys", "journey_walk") and precision == "fp64" and probe:
        nf = counters.get("n_fused", 0)  # the points of the kernel's own journeys
        ops = FP64_OPS_PER_POINT * (nf if top == "journeys" else counters["n_valid"] - nf)
        achieved = ops / (avg_ms / 1e3) / 1e9
        return {"bound": "alu", "kernel": top, "achieved": achieved, "peak": probe["peak_gops"],
                "unit": "G binary64 ops/s",
                "peak_source": "measured: binary64 issue-rate probe, fastest kind (" + probe["how"] + ")",
                "frac": achieved / probe["peak_gops"], "ops_per_launch": ops, "avg_launch_ms": avg_ms,
                "traffic": traffic,
                "hbm_achieved_gbs": algorithmic_bytes(top, counters) / (avg_ms / 1e3) / 1e9,
                "hbm_frac": algorithmic_bytes(top, counters) / (avg_ms / 1e3) / 1e9 / hbm_peak}
    ab = algorithmic_bytes(top, counters)
    achieved = ab / (avg_ms / 1e3) / 1e9 if ab else None
    return {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": hbm_peak,
            "peak_source": peak_src, "unit": "GB/s",
            "frac": (achieved / hbm_peak) if achieved else None,
            "algorithmic_bytes_per_launch": ab, "avg_launch_ms": avg_ms, "traffic": traffic}


def _counters(t, csv_host=None, pipe=None):
    c = {k: int(getattr(t, k)) for k in ("n_in", "n_malformed", "n_valid", "n_out_of_grid", "n_dup", "n_runs")}
    c.update(n_journeys=int(t.n_journeys), n_cells=int(t.n_cells))
    if csv_host is not None:
        c["csv_bytes"] = int(csv_host.numel())
    if pipe is not None:  # the journey stage's split by size (from the journey table)
        jn = pipe.results(to_host=True)["journeys"]["n"]
        big = jn >= FUSED_MIN_POINTS
        c.update(n_fused=int(jn[big].sum()), j_fused=int(big.sum()))
    return c


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
    ms_total, clocks = _day_steps(P, pipe, extract_dev, args.steps, args.warmup, barrier, local)
    stats = _stage_stats(P, stream, prec, tuning, extract_dev, args.steps)
    counters = _counters(pipe.tables(), csv_host, pipe)
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
    probe = fp64_probe(stream) if args.precision == "fp64" else None
    stages = stats["stages"]
    top = max(stages, key=lambda s: stages[s]["ms"])
    roofline = _roofline_entry(top, stages, counters, args.steps, args.precision, probe)
    hbm_step = _hbm_step(stages, counters, ms_step, args.steps, csv_host is not None,
                         traffic_table(args.precision))
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
                   "l2": ("inputs larger than L2 (no flush needed)" if h2d > L2_BYTES else
                          "inputs smaller than L2, steps back to back without a flush (a parity-size case)"),
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
        "fp64_probe": probe,
        "clocks": clocks,
    }
    batch_res = pipe.results(to_host=True)
    pipe.close()
    # ---- the same day in the float32 form (its own tuned shapes, same protocol) -----------
    if args.fp32_leg and args.precision == "fp64":
        line["fp32_day"] = _leg(lambda: _fp32_day(P, stream, extract_dev, args, barrier, local, world, dev, n_job,
                                                  csv_host, batch_res))
    # ---- the same day extracted from CSV text (binary64 form) ------------------------------
    if args.csv_leg and csv_host is None:
        line["csv_day"] = _leg(lambda: _csv_day(P, host, stream, args, barrier, local, world, dev, rank))
    if args.serve_feeds > 0:
        line["serving"] = serving(host, n, args, batch_res["cells"], ms_step)
    if args.week_scale > 0 and csv_host is None:
        del d_in
        torch.cuda.empty_cache()
        line["week"] = _leg(lambda: week_leg(args, args.week_scale, local, rank))
        line["week"].pop("_host0", None)
    if rank == 0:
        line["cpu_baseline"], line["parity"] = cpu_baseline(host, n, budget_s=args.cpu_budget,
                                                            batch=batch_res if csv_host is None else None)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _leg(fn):
    """Runs an extra leg of the bench; a failure is reported in its entry instead of ending the
    run (the headline figures above it stand on their own)."""
    try:
        return fn()
    except Exception as exc:  # noqa: BLE001 - reported in the line
        import torch

        torch.cuda.synchronize()
        return {"error": f"{type(exc).__name__}: {exc}"}


def _fp32_day(P, stream, extract_dev, args, barrier, local, world, dev, n_job, csv_host, batch_res):
    p32 = P.Pipeline(stream=stream, precision=P.FP32)
    extract_dev(p32)
    tune32 = p32.autotune(reps=2) if args.autotune else {**p32.tuning, "ms": None}
    ms32, clk32 = _day_steps(P, p32, extract_dev, args.steps, args.warmup, barrier, local)
    st32 = _stage_stats(P, stream, P.FP32, tune32, extract_dev, args.steps)["stages"]
    c32 = _counters(p32.tables(), csv_host, p32)
    r32 = p32.results(to_host=True)
    p32.close()
    (ms32,), _ = over_ranks([ms32], [0], world, dev)
    top32 = max(st32, key=lambda s: st32[s]["ms"])
    return {"ms_per_step": ms32 / args.steps, "records_per_s": n_job * args.steps / (ms32 / 1e3),
            "hbm_step": _hbm_step(st32, c32, ms32 / args.steps, args.steps, csv_host is not None,
                                  traffic_table("fp32")),
            "roofline": _roofline_entry(top32, st32, c32, args.steps, "fp32", None),
            "stages": {s: {"ms_per_step": v["ms"] / args.steps} for s, v in st32.items() if v["launches"]},
            "errors_vs_fp64_form": _form_errors(r32, batch_res), "tuning": tune32, "clocks": clk32}


def _csv_day(P, host, stream, args, barrier, local, world, dev, rank):
    """The day's records as CSV text (0.5% malformed rows), parsed and processed on the device:
    device-resident timed steps (extract from the text, transform, load), stage times from a
    profiled run, the step's bytes against the measured copy bandwidth."""
    import torch

    import cvgen

    t_gen = time.perf_counter()
    text, n_bad = cvgen.to_csv({k: host[k].numpy() for k in host}, seed=1 + rank, malformed_frac=0.005)
    t_gen = time.perf_counter() - t_gen
    d_csv = torch.from_numpy(text).to(dev)
    del text
    torch.cuda.synchronize()
    extract = lambda p: p.extract_csv(d_csv)
    pc = P.Pipeline(stream=stream, precision=P.FP64)
    extract(pc)
    tune = pc.autotune(reps=2) if args.autotune else {**pc.tuning, "ms": None}
    ms, clk = _day_steps(P, pc, extract, args.steps, args.warmup, barrier, local)
    st = _stage_stats(P, stream, P.FP64, tune, extract, args.steps)["stages"]
    c = _counters(pc.tables(), None, pc)
    c["csv_bytes"] = int(d_csv.numel())
    pc.close()
    del d_csv
    torch.cuda.empty_cache()
    (ms,), (nj,) = over_ranks([ms], [c["n_in"]], world, dev)
    top = max(st, key=lambda k: st[k]["ms"])
    return {"workload": f"the day as CSV text ({c['csv_bytes']} bytes, {n_bad} malformed rows)",
            "ms_per_step": ms / args.steps, "records_per_s": nj * args.steps / (ms / 1e3),
            "hbm_step": _hbm_step(st, c, ms / args.steps, args.steps, True, traffic_table("fp64")),
            "roofline": _roofline_entry(top, st, c, args.steps, "fp64", None),
            "stages": {k: {"ms_per_step": v["ms"] / args.steps} for k, v in st.items() if v["launches"]},
            "counters": c, "generation_s": t_gen, "tuning": tune, "clocks": clk}


def _host_available_bytes():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except Exception:
        pass
    return None


def _form_errors(res, ref):
    """Float32 form against the binary64 form of the same input: integer outputs identical,
    largest relative error of each floating-point output."""
    same_int = all(np.array_equal(res["cells"][k], ref["cells"][k]) for k in ("key", "count", "min", "max")) and \
        all(np.array_equal(res["journeys"][k], ref["journeys"][k]) for k in ("id", "n", "start_ts", "end_ts", "dwell_ms"))
    return {"integers_keys_counts_min_max_equal": bool(same_int),
            "journey_distance_max_rel": _max_rel(res["journeys"]["distance_m"], ref["journeys"]["distance_m"]),
            "cell_sum_max_rel": _max_rel(res["cells"]["sum"], ref["cells"]["sum"]),
            "cell_mean_max_rel": _max_rel(res["cells"]["mean"], ref["cells"]["mean"])}


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


def _max_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size == 0:
        return 0.0
    d = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    d[(a == 0) & (b == 0)] = 0.0
    return float(d.max())


def week_leg(args, scale, local, rank, steps=None, warmup=None):
    """The batched workload: 7 days x 4 regional boxes in one batch (one pass of every kernel,
    launch shapes from the autotuner, the post-sizing sequence replayed as a CUDA graph), float32
    form unless --precision says otherwise; the binary64 form runs once first (results kept on
    the host) for the per-output error report."""
    import torch

    import cvgen
    import paper_2305_07454_b300 as P

    steps = args.steps if steps is None else steps
    warmup = max(args.warmup, 2) if warmup is None else warmup
    dev = torch.device("cuda", local)
    prec = args.precision if args.workload == "week_regions" and args.precision else "fp32"
    recipes = cvgen.week_regions(seed=1 + rank, scale=scale)
    n_all = sum(cvgen.count(r["params"]) for r in recipes)
    avail = _host_available_bytes()
    need = n_all * (sum(BYTES[k] for k in COLS) + 4) * 2  # pinned columns, heading scratch, headroom
    if avail is not None and avail < need:
        return {"skipped": f"host memory: {avail / 2**30:.0f} GiB available, {need / 2**30:.0f} GiB wanted "
                           f"for {n_all} records"}
    t_gen = time.perf_counter()
    host, grids = [], []
    dt = {"jid": torch.int64, "ts": torch.int64, "lat": torch.float64, "lon": torch.float64,
          "speed": torch.float32}
    for r in recipes:
        n_i = cvgen.count(r["params"])
        h = {k: torch.empty(n_i, dtype=v, pin_memory=True) for k, v in dt.items()}
        cvgen.generate(r["params"], out={**{k: v.numpy() for k, v in h.items()},
                                         "heading": np.empty(n_i, np.float32)})
        host.append(h)
        grids.append({k: r[k] for k in P.GRID_KEYS})
    t_gen = time.perf_counter() - t_gen
    n = sum(h["jid"].shape[0] for h in host)
    d_insts = [dict(g, **{k: h[k].to(dev, non_blocking=True) for k in COLS}) for g, h in zip(grids, host)]
    h_insts = [dict(g, **{k: h[k] for k in COLS}) for g, h in zip(grids, host)]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    pc = P.FP32 if prec == "fp32" else P.FP64

    ref = None
    if pc == P.FP32:  # the binary64 form of the same batch, for the error report
        with P.Pipeline(stream=stream, precision=P.FP64) as p64:
            p64.extract_batch(d_insts)
            p64.transform()
            p64.load()
            ref = p64.results(to_host=True)
        torch.cuda.empty_cache()
    # per-stage times of one eager run (profiled)
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
        counters = _counters(pe.tables(), None, pe)
    errors = _form_errors(res, ref) if ref is not None else None
    del res, ref
    torch.cuda.empty_cache()

    # timed: graph replays of the tuned shapes
    pipe = P.Pipeline(stream=stream, precision=pc, graph=1)
    pipe.tuning = {k: v for k, v in tuning.items() if k != "ms"}

    def step(insts):
        pipe.extract_batch(insts)
        pipe.transform()
        pipe.load()
        pipe.tables()

    for _ in range(warmup):
        step(d_insts)
    pipe.stats_reset()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(steps):
            step(d_insts)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    gst = pipe.stats()
    ms_step = ms_total / steps
    # end to end from pinned host columns
    e2e_steps = max(1, min(steps, 2))
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
    del d_insts
    torch.cuda.empty_cache()
    stages = stats["stages"]
    top = max(stages, key=lambda s: stages[s]["ms"])
    return {
        "workload": f"week_regions x{scale:g}: {len(recipes)} instances (7 days x 4 regional boxes), {n} records, "
                    f"{counters['n_journeys']} journeys, Zipf(1.5) journey lengths on [10, 200000], one batch",
        "records": n, "instances": len(recipes), "precision": prec, "scale": scale,
        "instance_records": [int(h["jid"].shape[0]) for h in host],
        "steps": steps, "warmup": warmup, "ms_per_step": ms_step, "records_per_s": n / (ms_step / 1e3),
        "tuning": {**tuning, "seconds": tune_t},
        "graph": {"replays_in_timed_steps": gst["graph_replays"], "launches_per_step": gst["total_launches"] / steps},
        "e2e": {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": n * sum(BYTES[k] for k in COLS),
                "d2h_bytes_per_step": d2h},
        "gpu_launches": gst["total_launches"],
        "roofline": _roofline_entry(top, stages, counters, 1, prec, None),
        "hbm_step": _hbm_step(stages, counters, ms_step, 1, False),
        "stages": {k: {"ms_per_step": v["ms"], "launches_per_step": v["launches"]} for k, v in stages.items() if v["launches"]},
        "errors_vs_fp64_form": errors,
        "counters": counters,
        "generation_s": t_gen,
        "clocks": clk.summary(),
        "_host0": {k: host[0][k] for k in COLS},
    }


def run_week(args):
    """--workload week_regions: the batched workload as the line's headline."""
    rank, world, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    w = week_leg(args, args.scale, local, rank)
    host0 = w.pop("_host0")
    line = {
        "metric": METRIC, "value": w["records_per_s"], "unit": UNIT, "n_gpus": world, "steps": w["steps"],
        "warmup": w["warmup"], "ms_per_step": w["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if w["precision"] == "fp64" else "f32 (binary64 coordinate differences)",
        "data": "synthetic",
        "config": {"workload": w["workload"], "records": w["records"], "instances": w["instances"],
                   "precision": w["precision"], "scale": w["scale"], "instance_records": w["instance_records"],
                   "l2": "inputs larger than L2 (no flush needed)", "parallelism": "1 GPU"},
        **{k: w[k] for k in ("tuning", "graph", "e2e", "gpu_launches", "roofline", "hbm_step", "stages",
                             "errors_vs_fp64_form", "counters", "generation_s", "clocks")},
    }
    if rank == 0:
        line["cpu_baseline"], _ = cpu_baseline(host0, int(host0["jid"].shape[0]), budget_s=args.cpu_budget)
        print(json.dumps(line), flush=True)


def _sample_journeys(host, frac_den: int):
    """Whole journeys: the records whose journey id falls in 1 of frac_den hash classes."""
    jid = host["jid"].numpy() if hasattr(host["jid"], "numpy") else host["jid"]
    h = (jid.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(40)
    sel = np.flatnonzero((h % np.uint64(frac_den)) == 0)
    return {k: (host[k].numpy() if hasattr(host[k], "numpy") else host[k])[sel] for k in COLS}


def _agree(name, got, want, bad, rel=None, abs_=1e-9):
    """Records in `bad` the first element where got and want differ (exactly, or beyond
    rel * max(|got|, |want|) + abs_ when rel is given)."""
    got, want = np.asarray(got), np.asarray(want)
    if got.shape != want.shape:
        bad.append(f"{name}: shape {got.shape} vs {want.shape}")
        return
    if rel is None:
        ok = (got == want.astype(got.dtype)) | (np.isnan(got) & np.isnan(want)) if got.dtype.kind == "f" \
            else got == want.astype(got.dtype)
    else:
        g, w = got.astype(np.float64), want.astype(np.float64)
        ok = (np.abs(g - w) <= rel * np.maximum(np.abs(g), np.abs(w)) + abs_) | (np.isnan(g) & np.isnan(w))
    if not ok.all():
        i = int(np.flatnonzero(~ok)[0])
        bad.append(f"{name}: {int((~ok).sum())} of {ok.size} differ, first at {i}: {got.flat[i]!r} vs {want.flat[i]!r}")


def _parity(sample, o, batch):
    """The CUDA path against the oracle at the benchmarked size. (1) The full day's journey rows
    of the sampled journeys (whole journeys, so their rows depend on nothing else) against the
    oracle's: counts, times, dwell and positions exactly, distance within 1e-6 relative.
    (2) The pipeline run on the sample alone against the oracle on the sample: every table and
    per-point column (order, keys, flags, counts, min and max exactly; floats within 1e-6).
    (3) Properties of the full day's tables that hold at any size: conservation of records,
    cell keys strictly increasing, min <= mean <= max."""
    import torch

    import paper_2305_07454_b300 as P

    bad = []
    bj, oj = batch["journeys"], o["journeys"]
    at = np.searchsorted(bj["id"], oj["jid"])
    at = np.minimum(at, max(bj["id"].shape[0] - 1, 0))
    if not np.array_equal(bj["id"][at], oj["jid"]):
        bad.append("full-day journey ids: sampled ids missing")
    else:
        for k in ("n", "start_ts", "end_ts", "duration_ms", "dwell_ms", "start_lat", "start_lon", "end_lat", "end_lon"):
            _agree("full-day journey " + k, bj[k][at], oj[k], bad)
        _agree("full-day journey distance_m", bj["distance_m"][at], oj["distance_m"], bad, rel=1e-6)
    t = {k: torch.from_numpy(np.ascontiguousarray(sample[k])).cuda() for k in COLS}
    with P.Pipeline(materialize_points=1) as p:
        g = p.run(t)
    for k in ("n_in", "n_malformed", "n_valid", "n_out_of_grid", "n_dup", "n_journeys", "n_cells"):
        if g["counters"][k] != o["counters"][k]:
            bad.append(f"sample counter {k}: {g['counters'][k]} vs {o['counters'][k]}")
    _agree("sample journey id", g["journeys"]["id"], oj["jid"], bad)
    for k in ("n", "start_ts", "end_ts", "duration_ms", "dwell_ms", "start_lat", "start_lon", "end_lat", "end_lon"):
        _agree("sample journey " + k, g["journeys"][k], oj[k], bad)
    _agree("sample journey distance_m", g["journeys"]["distance_m"], oj["distance_m"], bad, rel=1e-6)
    for k in ("key", "row", "col", "bin", "count", "min", "max"):
        _agree("sample cell " + k, g["cells"][k], o["cells"][k], bad)
    for k in ("sum", "mean"):
        _agree("sample cell " + k, g["cells"][k], o["cells"][k], bad, rel=1e-6)
    for k in ("perm", "key", "flags", "dwell", "stop_ms"):
        _agree("sample point " + k, g["points"][k], o["points"][k], bad)
    for k in ("d", "vhat", "accel", "accel_v"):
        _agree("sample point " + k, g["points"][k], o["points"][k], bad, rel=1e-6)
    bc, cc = batch["cells"], batch["counters"]
    if int(bc["count"].astype(np.int64).sum()) + cc["n_out_of_grid"] != cc["n_valid"]:
        bad.append("full day: cell counts + off-grid points != kept records")
    if int(batch["journeys"]["n"].sum()) != cc["n_valid"]:
        bad.append("full day: journey sizes do not add up to the kept records")
    if bc["key"].size and not np.all(np.diff(bc["key"].astype(np.int64)) > 0):
        bad.append("full day: cell keys not strictly increasing")
    if not (np.all(bc["min"] <= bc["mean"] + 1e-9) and np.all(bc["mean"] <= bc["max"] + 1e-9)):
        bad.append("full day: a cell mean outside [min, max]")
    return {"journeys_checked": int(oj["jid"].shape[0]), "records_checked": int(o["counters"]["n_in"]),
            "ok": not bad, "failures": bad[:8],
            "what": "full-day journey rows of the sampled journeys vs the oracle (exact; distance 1e-6); "
                    "the pipeline on the sample vs the oracle, every table and point column; "
                    "full-day conservation and ordering"}


def cpu_baseline(host, n, budget_s=15.0, batch=None):
    """The oracle, single-threaded, timed on a bounded sample of whole journeys; with the day's
    batch results, the parity check of the CUDA path on that sample (returned second)."""
    import oracle

    o = oracle.get()
    den = 64
    sample = _sample_journeys(host, den)
    t0 = time.perf_counter()
    out = o.run(sample)
    dt = time.perf_counter() - t0
    # grow the sample toward the budget (about 10-30 s of CPU work)
    while dt < budget_s / 4 and den > 4:
        den //= 2
        sample = _sample_journeys(host, den)
        t0 = time.perf_counter()
        out = o.run(sample)
        dt = time.perf_counter() - t0
    m = sample["jid"].shape[0]
    base = {"value": m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"whole journeys with id hash in 1 of {den} classes: {m} records, "
                      f"{len(np.unique(sample['jid']))} journeys, {dt:.1f} s single-threaded",
            "cpu": _cpu_model()}
    return base, (_leg(lambda: _parity(sample, out, batch)) if batch is not None else None)


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
    ap.add_argument("--fp32-leg", type=int, default=1, help="0 skips the float32 form of the day")
    ap.add_argument("--csv-leg", type=int, default=1, help="0 skips the day extracted from CSV text")
    ap.add_argument("--week-scale", type=float, default=1.0,
                    help="instance size factor of the week_regions leg of the day run (0 skips it)")
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
