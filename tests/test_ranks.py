"""The replica path of bench.py on CPU: two gloo ranks combine their figures the way the GPU
ranks do (the slowest rank's time, the records of all ranks), and the reference arm does its
work on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    maxes, sums = bench.over_ranks([10.0 + 5 * rank, 0.5 - 0.1 * rank], [1000 + rank, 7], w)
    out.put((rank, r, w, local, maxes, sums))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_over_ranks_with_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, local, maxes, sums in got:
        assert (r, w, local) == (rank, world, rank)
        assert maxes == [10.0 + 5 * (world - 1), 0.5]
        assert sums == [sum(1000 + k for k in range(world)), 7 * world]


def test_one_rank_needs_no_group():
    assert bench.over_ranks([3.5], [12], 1) == ([3.5], [12])


def test_reference_arm_works_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, steps, warmup = "small_day", 1, 1

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""


def test_journey_stage_is_one_pass_per_step():
    """The journey sort launches its class bounds and one kernel per size class per step over one
    pass of the classes' points: its time per pass is the stage time per step, and its
    algorithmic bytes count once per step; every other stage's launch is a pass of its own. The
    journey stage's bytes split by size between the fused kernel (journeys above 8192 points)
    and the sort and walk of the others."""
    assert bench.unit_launches("journey_sort", 20, 10) == 10
    assert bench.unit_launches("journey_sort", 10, 10) == 10
    assert bench.unit_launches("journeys", 20, 10) == 10
    assert bench.unit_launches("journey_walk", 10, 10) == 10
    assert bench.unit_launches("radix_onesweep", 160, 10) == 160
    assert bench.unit_launches("scatter", 0, 10) == 1
    c = {"n_in": 100, "n_valid": 90, "n_journeys": 3, "n_runs": 7, "n_cells": 5, "n_fused": 40, "j_fused": 1}
    assert bench.algorithmic_bytes("journeys", c) == 32.0 * 40 + 96.0 * 1
    assert bench.algorithmic_bytes("journey_sort", c) == 10.0 * 50
    assert bench.algorithmic_bytes("journey_walk", c) == 34.0 * 50 + 28.0 * 7 + 96.0 * 2
    # without the split every journey is counted as walked
    c0 = {k: v for k, v in c.items() if k not in ("n_fused", "j_fused")}
    assert bench.algorithmic_bytes("journey_walk", c0) == 34.0 * 90 + 28.0 * 7 + 96.0 * 3


def test_traffic_figures_follow_the_kernel_sources(monkeypatch):
    """The ncu traffic per record is used only while the kernel sources are the ones it was
    captured with (their hash); with other sources the line has no traffic and no gate figure."""
    stages = {"scatter": {"launches": 1, "ms": 4.0}}
    c = {"n_in": 100, "n_valid": 100, "n_journeys": 1, "n_runs": 1, "n_cells": 1}
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_SHA256", bench.kernel_sources_sha256())
    assert bench.traffic_table("fp64") is bench.TRAFFIC_PER_RECORD
    assert bench._hbm_step(stages, c, 4.0, 1, False, bench.traffic_table("fp64"))["gate"] is not None
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_SHA256", "0" * 64)
    assert bench.traffic_table("fp64") == {} and bench.traffic_table("fp32") == {}
    out = bench._hbm_step(stages, c, 4.0, 1, False, bench.traffic_table("fp64"))
    assert out["gate"] is None and "sources changed" in out["gate_missing_traffic"]
