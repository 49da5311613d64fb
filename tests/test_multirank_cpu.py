"""World-size-2 checks of the benchmark's multi-rank host logic on CPU (gloo).

Under torchrun every rank solves its own independent graph (weak scaling, no
data-path collective); the job's time is the max over ranks and its work the
sum over ranks.  These tests run that host logic with two gloo ranks.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    bench.dist_init(w, "gloo")
    try:
        bench.barrier(w)
        t_max = bench.reduce_max(1.0 + rank, w)       # rank 1 is the slow one
        work = bench.reduce_sum(10.0 * (rank + 1), w)  # each rank's own relaxations
        # every rank draws its own graph (seed + rank): the problems differ
        import graphgen
        g = graphgen.dense_graph_torch(16, 0.5, bench.SEED + rank)
        digest = torch.tensor([float(torch.nan_to_num(g, posinf=0).sum())])
        gathered = [torch.zeros(1) for _ in range(w)]
        dist.all_gather(gathered, digest)
        out.put((rank, t_max, work, [float(x) for x in gathered]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_summed_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, work, digests in res:
        assert t_max == 2.0          # max over ranks
        assert work == 30.0          # sum over ranks
        assert digests[0] != digests[1]  # independent graphs per rank


def test_single_rank_helpers_are_identity():
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.reduce_sum(3.5, 1) == 3.5
    bench.barrier(1)


def test_workload_config_matches_between_arms():
    """Both arms (GPU and the CPU reference) print the same config for a workload."""
    assert bench.workload_config(32768, 1) == bench.workload_config(32768, 1, "f32")
    assert "FP64" in bench.workload_config(32768, 2, "f64")["workload"]


def test_phase3_relaxation_count_is_the_algorithmic_work():
    """Sum over the rounds of the phase-4 relaxations equals n^3 minus phases 1-3."""
    n, T = 1000, 128
    R = (n + T - 1) // T
    per_round = bench.phase3_relax_per_round(n, T)
    phase4 = per_round * R
    phase123 = 0
    for r in range(R):
        m = min(T, n - r * T)
        phase123 += m ** 3 + 2 * m * m * (n - m)
    assert phase4 + phase123 == pytest.approx(n ** 3)


def _reference_worker(rank, world, port, path):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import argparse
    import contextlib
    args = argparse.Namespace(n=192, steps=2, warmup=1, dtype="f32", ref_step_seconds=0.2)
    with open(f"{path}.{rank}", "w") as f, contextlib.redirect_stdout(f):
        bench.run_reference(args)


def test_reference_arm_under_two_ranks_prints_one_line_from_rank_0(tmp_path):
    """The CPU reference arm as torchrun launches it for N > 1: rank 0 alone
    times the oracle and prints the one JSON line; the other rank exits 0
    without work or output."""
    import json
    ctx = mp.get_context("spawn")
    port = _free_port()
    path = str(tmp_path / "out")
    procs = [ctx.Process(target=_reference_worker, args=(r, 2, port, path)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    lines0 = open(f"{path}.0").read().strip().splitlines()
    assert open(f"{path}.1").read() == ""
    assert len(lines0) == 1
    line = json.loads(lines0[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 2
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC and line["higher_is_better"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"] > 0
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"] == bench.workload_config(192, 2)
