#!/usr/bin/env python
"""Benchmark of the GB300 blocked Floyd-Warshall library.

Default (``--impl ours``): one step = one blocked FW solve of a synthetic
n = 32768 dense directed graph (edge probability 0.5, integer weights uniform on
[1, 100], FP32 distances + int32 path matrix) through ``apsp_fw_f32``, with the
input restored from a resident copy first (the restore copy, 4 GiB, is inside
the timed region and also flushes L2).  ``value`` = n^3 / t summed over ranks
(min-plus relaxations per second, the metric of the paper's Eq. 1 divided by 2).

The same JSON line also carries:
  * ``roofline``: phase-4 kernel (the dominant one) timed live with CUDA events
    around each of its launches inside the timed region;
  * ``e2e``: the same solve as one C-ABI call on pinned HOST buffers
    (``apsp_fw_f32_host``: host-to-device copy of W, the solve, device-to-host
    copies of D and P, all inside the timed region);
  * ``cpu_baseline``: the CPU oracle (classic FW, Algorithm 1) on a bounded
    prefix of the outer k loop of the same graph, on the host cores;
  * ``fp64``, ``batched``, ``fwd_bwd``: the other measurements the headline
    metric names (FP64 solve, 4096-graph batched launch in a CUDA graph vs
    per-graph launches, forward + backward of 256 graphs of n = 256).

``--impl reference``: the CPU oracle timed on the host cores, each step a
bounded sample (a prefix of the outer k loop) of the same workload.
Multi-GPU (torchrun): every rank solves its own graph (independent problems,
weak scaling, no data-path collective); timing is the max over ranks.  The
4096-graph batch is also split over the ranks (LPT by n^3, no collective) and
timed as one job (max over ranks).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "min-plus relaxations/s (n^3/t) FP32 & FP64 at n=32768; batched graphs/s; fwd+bwd ms"
UNIT = "relax/s"
SEED = 20210517


# ----------------------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, gpu_index=None):
        self.proc = None
        self.path = None
        self.gpu_index = gpu_index

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_index is not None:
                cmd += ["-i", str(self.gpu_index)]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, val in zip(names[1:], r[3][1:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows),
                "power_w_mean": statistics.mean(r[2] for r in loaded),
                "samples": len(rows), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- helpers
def device_facts(torch):
    p = torch.cuda.get_device_properties(0)
    return {"name": p.name, "sms": p.multi_processor_count}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def alu_peak_relax_per_s(sms: int, mhz: float) -> float:
    """add+min peak from unit counts: 128 relaxations / clock / SM (the FMA pipe
    adds 128 lanes per clock, as one packed FP32x2 add per two relaxations, and
    the ALU pipe compares 128 lanes per clock, as one three-input min per two
    relaxations) x SMs x clock.  The measured rate of the instruction pair is
    reported beside it (apsp_measure_peak); it is lower (~89 on GB300)."""
    return 128.0 * sms * mhz * 1e6


def eq1_gflops(relax_per_s: float) -> float:
    """The paper's Eq. 1 rate, GFLOPS = 2 N^3 / (t 10^9): two floating-point
    operations (the add and the compare) per relaxation."""
    return 2.0 * relax_per_s / 1e9


def gflops_per_watt(gflops: float, watts: float) -> float:
    """Energy efficiency as the paper's Tables 2 and 3 give it (§4.3): Eq. 1
    GFLOPS over the platform's power in watts."""
    return gflops / watts


def kernel_source_hash() -> str:
    """Hash of the sources the phase-4 kernel is built from: the shared headers,
    its constants and shared-memory layout (namespace k3 of phases_f32.cuh) and
    the kernel in fw_single.cu, so that changes elsewhere keep a capture valid."""
    d = os.path.join(ROOT, "paper_2105_07298_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("minplus_f32.cuh", "common.cuh", "bulk.cuh"):
        h.update(open(os.path.join(d, f)).read().encode())
    txt = open(os.path.join(d, "phases_f32.cuh")).read()
    h.update(txt[txt.index("namespace k3 {"):txt.index("}  // namespace k3")].encode())
    txt = open(os.path.join(d, "fw_single.cu")).read()
    h.update(txt[txt.index("template <bool EAGER>\n__global__"):txt.index("// Phase timing state")].encode())
    return h.hexdigest()[:16]


def profiled_traffic(n: int):
    """DRAM bytes of phase 4 per round (its one or two launches) at size n, from
    the committed ncu summary: measured on a small case (sampled rounds of an
    n = 16384 solve) and scaled to n by the per-round byte model written there
    (bytes per round proportional to n^2).  Only while the summary was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "phase3_minplus_f32_traffic.txt")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*(\w+)", txt)
    m_bpl = re.search(r"dram_bytes_per_round_n%d:\s*([0-9.eE+]+)" % n, txt)
    if not m_hash or not m_bpl or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_bpl.group(1))


def phase3_relax_per_round(n: int, T: int) -> float:
    """Algorithmic phase-4 relaxations of one round, averaged over the rounds:
    round r updates every (i, j) outside block row/column r with every k of block r."""
    R = (n + T - 1) // T
    tot = 0
    for r in range(R):
        m = min(T, n - r * T)
        tot += (n - m) * (n - m) * m
    return tot / R


def workload_config(n: int, world: int, dtype: str = "f32") -> dict:
    prec = "FP64" if dtype == "f64" else "FP32"
    return {"workload": f"blocked FW, dense directed graph n={n}, p=0.5, int weights U[1,100], "
                        f"{prec} D + int32 P",
            "n": n, "edge_prob": 0.5, "path_matrix": True,
            "l2": "inputs > L2, D restored each step",
            "parallelism": f"{world} independent graph(s), one per GPU"}


def time_events(torch, fn, reps=1):
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / 1e3


# ----------------------------------------------------------------------------- CPU oracle timing
def oracle_partial_rate(W_host, budget_s: float, probe_k: int = 8):
    """Classic FW (the oracle as it is) on a prefix of the outer k loop of W_host.
    Returns (relax/s, k iterations, threads, seconds).  The fixed cost of one call
    (copy of W, P := -1) is measured with k_end = 0 and subtracted; a probe of
    ``probe_k`` iterations sizes the sample to about ``budget_s`` seconds."""
    import oracle
    n = W_host.shape[0]
    t0 = time.perf_counter()
    oracle.fw(W_host, with_path=True, k_end=0)
    fixed = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.fw(W_host, with_path=True, k_end=probe_k)
    per_k = max((time.perf_counter() - t0 - fixed) / probe_k, 1e-3)
    k = int(max(probe_k, min(n, budget_s / per_k)))
    t0 = time.perf_counter()
    oracle.fw(W_host, with_path=True, k_end=k)
    t = max(time.perf_counter() - t0 - fixed, 1e-9)
    return k * float(n) * n / t, k, oracle.num_threads(), t


def run_reference(args):
    """--impl reference: the CPU oracle on bounded samples of the same workload."""
    rank, world, _ = dist_env()
    if world > 1:
        dist_init(world, "gloo")
        if rank != 0:
            barrier(world)
            return
    import numpy as np  # noqa: F401
    import graphgen
    import oracle
    oracle.build()
    n = args.n
    import torch
    W = graphgen.dense_graph_torch(n, 0.5, SEED, dtype=torch.float64 if args.dtype == "f64"
                                   else torch.float32).numpy()
    per_step = args.ref_step_seconds
    for _ in range(args.warmup):
        oracle_partial_rate(W, per_step / 4)
    rates, ks, secs = [], [], []
    for _ in range(args.steps):
        r, k, thr, t = oracle_partial_rate(W, per_step)
        rates.append(r)
        ks.append(k)
        secs.append(t)
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
            "data": "synthetic",
            "config": workload_config(n, world, args.dtype),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": f"outer k iterations 0..{min(ks) - 1} (at least) of classic FW "
                                       f"(Algorithm 1) on the n={n} graph per step (fixed per-call cost excluded)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if world > 1:
        barrier(world)


# ----------------------------------------------------------------------------- GPU arm
def bench_main(torch, apsp, graphgen, args, rank, world, dev):
    n = args.n
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    W = graphgen.dense_graph_torch(n, 0.5, SEED + rank, dtype=dt, device=dev)
    D = torch.empty_like(W)
    P = torch.empty((n, n), dtype=torch.int32, device=dev)

    def step():
        D.copy_(W)
        apsp.apsp_fw(D, P)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    apsp.profile_enable(True)
    with ClockSampler(args.gpu_index) as clk:
        t = time_events(torch, step, args.steps)
    torch.cuda.synchronize()
    barrier(world)
    prof = apsp.profile_collect()
    apsp.profile_enable(False)
    return W, D, P, t, prof, clk.summary()


def bench_e2e(torch, apsp, graphgen, W_dev, args):
    """The same solve as one C-ABI call on pinned HOST buffers (apsp_fw_f32_host):
    every step copies W in, solves, and copies D and P out; the device work
    buffers are the caller's, kept across steps (as a serving loop would)."""
    n = args.n
    Wh = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
    Wh.copy_(W_dev)
    Dh = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
    Ph = torch.empty((n, n), dtype=torch.int32, pin_memory=True)
    wd = torch.empty(n * n, dtype=torch.float32, device=W_dev.device)
    wp = torch.empty(n * n, dtype=torch.int32, device=W_dev.device)
    reps = max(1, min(args.steps, 2))

    def step():
        apsp.apsp_fw_f32_host(Wh, Dh, Ph, work_dist=wd, work_path=wp)

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t = time_events(torch, step, reps)
    wall = (time.perf_counter() - t0) / reps
    parts = {"step_ms": 1e3 * t / reps, "host_wall_ms": 1e3 * wall}
    return n ** 3 / (t / reps), n * n * 4, n * n * 8, Wh, parts


def bench_fp64(torch, apsp, graphgen, args, dev):
    n = args.fp64_n
    W = graphgen.dense_graph_torch(n, 0.5, SEED, dtype=torch.float64, device=dev)
    D = torch.empty_like(W)
    P = torch.empty((n, n), dtype=torch.int32, device=dev)

    def step():
        D.copy_(W)
        apsp.apsp_fw_f64(D, P)

    for _ in range(args.fp64_warmup):
        step()
    torch.cuda.synchronize()
    apsp.profile_enable(True)
    t = time_events(torch, step, args.fp64_steps)
    prof = apsp.profile_collect()
    apsp.profile_enable(False)
    del W, D, P
    return n, t / args.fp64_steps, prof


def bench_batched(torch, apsp, graphgen, args, dev):
    import numpy as np
    from paper_2105_07298_gb300 import batched
    from paper_2105_07298_gb300 import autotune
    tuned = ({} if args.no_autotune else
             autotune.autotune(device=dev, graphs_per_class=304, reps=2, save=False))
    sizes = graphgen.batch_sizes(4096, 16, 512, 1)
    off = batched.packed_offsets(sizes)
    total = batched.packed_numel(sizes)
    W = graphgen.batched_graphs_torch(sizes, 0.3, 1, off, total, device=dev)
    D = torch.empty_like(W)
    P = torch.empty(total, dtype=torch.int32, device=dev)
    plan = batched.BatchedPlan(sizes, off)
    # one launch (memset + persistent kernel) captured in a CUDA graph
    D.copy_(W)
    plan.run(D, P)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run(D, P)
    torch.cuda.current_stream().wait_stream(s)

    def step():
        D.copy_(W)
        g.replay()

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    reps = 3
    t = time_events(torch, step, reps) / reps
    t_copy = time_events(torch, lambda: D.copy_(W), reps) / reps
    t_solve = max(t - t_copy, 1e-9)
    # per-graph launches of the single-graph path on the same graphs
    views = [(D[o:o + int(m) * int(m)].view(int(m), int(m)), P[o:o + int(m) * int(m)].view(int(m), int(m)))
             for m, o in zip(sizes, off)]

    def per_graph():
        for dv, pv in views:
            apsp.apsp_fw_f32(dv, pv)

    D.copy_(W)
    per_graph()
    torch.cuda.synchronize()
    D.copy_(W)
    t_pg = time_events(torch, per_graph, 1)
    # the same plan without a path matrix (distances only), plain launches
    def step_np():
        D.copy_(W)
        plan.run(D)

    step_np()
    torch.cuda.synchronize()
    t_np = max(time_events(torch, step_np, reps) / reps - t_copy, 1e-9)
    relax = float(np.sum(sizes.astype(np.float64) ** 3))
    plan.close()
    facts = device_facts(torch)
    peak = alu_peak_relax_per_s(facts["sms"], float(measured_peaks().get("sm_max_mhz", 2070.0)))
    return {"graphs": 4096, "n_range": [16, 512], "edge_prob": 0.3, "cuda_graph": True,
            "graphs_per_s": 4096 / t_solve, "ms": 1e3 * t_solve, "relax_per_s": relax / t_solve,
            "frac_of_unit_peak": relax / t_solve / peak,
            "per_graph_launches": {"graphs_per_s": 4096 / t_pg, "ms": 1e3 * t_pg},
            "without_path": {"ms": 1e3 * t_np, "relax_per_s": relax / t_np,
                             "frac_of_unit_peak": relax / t_np / peak},
            "speedup_vs_per_graph": t_pg / t_solve,
            "autotuned_variants": {str(c): {"variant": r["variant"], "bounds": r["bounds"], "shape": r["shape"],
                                            "ms_per_variant": r["ms"]} for c, r in tuned.items()},
            "variants": [batched.get_variant(c) for c in range(batched.num_classes())],
            "note": "graph restore copy excluded (timed separately and subtracted)"}


def bench_batched_sharded(torch, apsp, graphgen, args, dev, rank, world):
    """The 4096-graph batch split over the ranks (LPT by n^3, no exchange on the
    data path): this rank's share in one batched launch replayed from a CUDA
    graph.  Returns this rank's seconds per launch and its share."""
    import numpy as np
    from paper_2105_07298_gb300 import batched, shard
    sizes = graphgen.batch_sizes(4096, 16, 512, 1)
    sh = shard.shards(sizes, world)[rank]
    W = graphgen.batched_graphs_torch(sh.sizes, 0.3, 1, sh.offsets, sh.numel, graph_ids=sh.ids, device=dev)
    D = torch.empty_like(W)
    P = torch.empty(sh.numel, dtype=torch.int32, device=dev)
    plan = batched.BatchedPlan(sh.sizes, sh.offsets)
    D.copy_(W)
    plan.run(D, P)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run(D, P)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        D.copy_(W)
        g.replay()
    torch.cuda.synchronize()
    reps = 3
    total = 0.0
    for _ in range(reps):
        D.copy_(W)
        total += time_events(torch, g.replay)
    plan.close()
    return total / reps, {"graphs": int(len(sh.ids)), "relax": float(np.sum(sh.sizes.astype(np.float64) ** 3))}


def bench_fwd_bwd(torch, apsp, graphgen, args, dev):
    import numpy as np
    from paper_2105_07298_gb300 import batched
    Bn, n = 256, 256
    sizes = [n] * Bn
    off = [b * n * n for b in range(Bn)]
    W = graphgen.batched_graphs_torch(sizes, 0.4, 5, np.array(off), Bn * n * n, weights="real",
                                      lo=0.5, hi=2.0, device=dev).view(Bn, n, n)
    gD = torch.from_numpy(graphgen.normal((Bn, n, n), 12)).to(dev)
    D = torch.empty_like(W)
    P = torch.empty((Bn, n, n), dtype=torch.int32, device=dev)
    gW = torch.empty_like(W)
    plan = batched.BatchedPlan(sizes, off)

    def fwd():
        D.copy_(W)
        plan.run(D.view(-1), P.view(-1))

    def bwd():
        apsp.apsp_fw_backward_f32(gD, P, D, gW, check=False)

    def fwd_pg():
        D.copy_(W)
        for b in range(Bn):
            apsp.apsp_fw_f32(D[b], P[b])

    def bwd_pg():
        for b in range(Bn):
            apsp.apsp_fw_backward_f32(gD[b], P[b], D[b], gW[b], check=False)

    for f in (fwd, bwd, fwd_pg, bwd_pg):
        f()
    torch.cuda.synchronize()
    reps = 3
    tf = time_events(torch, fwd, reps) / reps
    tb = time_events(torch, bwd, reps) / reps
    tfp = time_events(torch, fwd_pg, 1)
    tbp = time_events(torch, bwd_pg, 1)
    plan.close()
    return {"graphs": Bn, "n": n, "edge_prob": 0.4, "weights": "real U[0.5,2.0]",
            "fwd_ms": 1e3 * tf, "bwd_ms": 1e3 * tb, "fwd_bwd_ms": 1e3 * (tf + tb),
            "per_graph_path": {"fwd_ms": 1e3 * tfp, "bwd_ms": 1e3 * tbp, "fwd_bwd_ms": 1e3 * (tfp + tbp)},
            "note": "fwd includes the 64 MiB input restore copy"}


def bench_sweep(torch, apsp, graphgen, args, dev, pair_rate=None):
    """FP32 blocked FW over the sizes of the n sweep, with and without the path
    matrix: solve time (device events around the call; the input is restored by
    a device copy before each solve, outside the timed region), relax/s, the
    fraction of the add+min peak (unit counts at the maximum SM clock, and the
    measured instruction-pair rate), and the HBM rate of the algorithmic bytes
    (D read + written and P written once per round: R (2s + 4) n^2 bytes) for the
    whole solve and for phases 1-3 alone."""
    facts = device_facts(torch)
    peaks = measured_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", 6777.0))
    T = apsp.block_size(torch.float32)
    peak_unit = alu_peak_relax_per_s(facts["sms"], max_mhz)
    peak_meas = pair_rate * facts["sms"] * max_mhz * 1e6 if pair_rate else None
    out = []
    with ClockSampler(args.gpu_index) as clk:
        for n in args.sweep:
            W = graphgen.dense_graph_torch(n, 0.5, SEED, dtype=torch.float32, device=dev)
            D = torch.empty_like(W)
            P = torch.empty((n, n), dtype=torch.int32, device=dev)
            R = (n + T - 1) // T
            point = {"n": n}
            for with_path in (True, False):
                reps = 3 if n <= 8192 else 1
                D.copy_(W)
                apsp.apsp_fw_f32(D, P if with_path else None)  # warm-up
                total = 0.0
                apsp.profile_enable(True)
                for _ in range(reps):
                    D.copy_(W)
                    total += time_events(torch, lambda: apsp.apsp_fw_f32(D, P if with_path else None))
                prof = apsp.profile_collect()
                apsp.profile_enable(False)
                t = total / reps
                bytes_round = (2 * 4 + (4 if with_path else 0)) * n * n
                m = min(T, n)
                p123_bytes = (2 * 4 + (4 if with_path else 0)) * (m * m + 2 * m * (n - m))  # per round
                p123_ms = (prof["phase1_diag"][0] + prof["phase2_panels"][0]) / reps
                point["with_path" if with_path else "without_path"] = {
                    "ms": 1e3 * t, "relax_per_s": n ** 3 / t,
                    "frac_of_unit_peak": n ** 3 / t / peak_unit,
                    "frac_of_measured_pair_rate": (n ** 3 / t / peak_meas) if peak_meas else None,
                    "phase_ms": {k: v[0] / reps for k, v in prof.items()},
                    "hbm_gbs": R * bytes_round / t / 1e9, "hbm_frac": R * bytes_round / t / 1e9 / hbm,
                    "phase1_3_hbm_gbs": (R * p123_bytes / (p123_ms / 1e3) / 1e9) if p123_ms > 0 else None}
            out.append(point)
            del W, D, P
            torch.cuda.empty_cache()
    return {"points": out, "clocks": clk.summary(), "dtype": "f32",
            "peak_basis": f"{facts['sms']} SMs x 128 relax/clk/SM x {max_mhz:.0f} MHz; HBM {hbm:.0f} GB/s",
            "note": "phases 1-3 run beside phase 4 (look-ahead stream), so their HBM rate is that of "
                    "their own launches; n=4096 fits in L2"}


def bench_sweep_f64(torch, apsp, graphgen, args, dev):
    """FP64 blocked FW at the smaller sweep sizes, with the path matrix: solve
    time (device events; input restored before each solve, outside the timed
    region), relax/s and the fraction of the unit-count add+min peak (the FP64
    main loop runs the FP32 pair on lower bounds)."""
    facts = device_facts(torch)
    max_mhz = float(measured_peaks().get("sm_max_mhz", 2070.0))
    peak_unit = alu_peak_relax_per_s(facts["sms"], max_mhz)
    out = []
    for n in args.sweep_f64:
        W = graphgen.dense_graph_torch(n, 0.5, SEED, dtype=torch.float64, device=dev)
        D = torch.empty_like(W)
        P = torch.empty((n, n), dtype=torch.int32, device=dev)
        D.copy_(W)
        apsp.apsp_fw_f64(D, P)  # warm-up
        reps = 3
        total = 0.0
        for _ in range(reps):
            D.copy_(W)
            total += time_events(torch, lambda: apsp.apsp_fw_f64(D, P))
        t = total / reps
        out.append({"n": n, "ms": 1e3 * t, "relax_per_s": n ** 3 / t, "frac_of_unit_peak": n ** 3 / t / peak_unit})
        del W, D, P
        torch.cuda.empty_cache()
    return {"points": out, "dtype": "f64", "path_matrix": True}


def run_side_workload(args, torch, apsp, graphgen, dev):
    """--workload batched / fwd_bwd: that measurement alone (profiling runs)."""
    if args.workload == "batched":
        r = bench_batched(torch, apsp, graphgen, args, dev)
        line = {"metric": "batched graphs/s", "value": r["graphs_per_s"], "unit": "graphs/s", **r}
    elif args.workload == "sweep":
        r = bench_sweep(torch, apsp, graphgen, args, dev, apsp.measure_peak(4))
        line = {"metric": "min-plus relaxations/s (FP32 n sweep)", "unit": UNIT, **r}
    else:
        r = bench_fwd_bwd(torch, apsp, graphgen, args, dev)
        line = {"metric": "forward+backward ms", "value": r["fwd_bwd_ms"], "unit": "ms",
                "higher_is_better": False, **r}
    line.update({"n_gpus": 1, "data": "synthetic", "workload": args.workload})
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, "nccl")
    import graphgen
    import paper_2105_07298_gb300 as apsp
    apsp.load()
    if args.workload != "single":
        if rank == 0:
            run_side_workload(args, torch, apsp, graphgen, dev)
        barrier(world)
        return
    facts = device_facts(torch)
    peaks = measured_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))

    W, D, P, t, prof, clocks = bench_main(torch, apsp, graphgen, args, rank, world, dev)
    n = args.n
    t_max = reduce_max(t, world, dev)
    total_relax = reduce_sum(float(n) ** 3 * args.steps, world, dev)
    value = total_relax / t_max

    T = apsp.block_size(torch.float64 if args.dtype == "f64" else torch.float32)
    # Phase 4 of a round is one launch, or two (row/column r+1 first, then the
    # rest) when the next round's phases 1-3 run beside it; its device time is
    # summed per round.
    k3_ms, k3_launches = prof["phase3_minplus"]
    rounds = ((n + T - 1) // T) * args.steps
    per_round_s = (k3_ms / 1e3) / max(rounds, 1)
    relax_round = phase3_relax_per_round(n, T)
    achieved = 2 * relax_round / per_round_s / 1e12  # Eq. 1 FLOP/s (add + compare)
    # The FP64 path's main loop runs one FP32 lower-bound relaxation per FP64
    # relaxation (upper bounds and FP64 adds only to confirm improvements):
    # the same add+min bound as FP32.
    per_clk = 128.0
    peak = 2 * alu_peak_relax_per_s(facts["sms"], max_mhz) * per_clk / 128.0 / 1e12
    mhz_meas = clocks["sm_mhz"] if clocks else None
    try:  # the inner-loop instruction pair on registers only, this GPU (relax/clk/SM)
        rate_meas = apsp.measure_peak(8 if args.dtype == "f64" else 4)
    except Exception:
        rate_meas = None
    traffic = profiled_traffic(n)
    launches = sum(c for _, c in prof.values())
    phase_share = {k: {"ms": round(v[0], 2), "launches": v[1]} for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": workload_config(n, world, args.dtype),
        "roofline": {"bound": "alu", "block": T,
                     "kernel": "fw64_product<0> (phase 4)" if args.dtype == "f64" else "fw_phase3_minplus_f32 (phase 4)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "flop_def": "Eq. 1: 2 FLOP (add + compare) per relaxation; "
                                 f"{relax_round:.4e} relaxations per round (average over rounds)",
                     "peak_basis": f"{facts['sms']} SMs x {per_clk:.0f} relax/clk/SM x {max_mhz:.0f} MHz (max SM clock)",
                     "frac_at_measured_clock": (achieved / (2 * alu_peak_relax_per_s(facts['sms'], mhz_meas)
                                                            * per_clk / 128.0 / 1e12) if mhz_meas else None),
                     "avg_round_ms": per_round_s * 1e3, "launches": k3_launches,
                     "measured_pair_rate_relax_per_clk_sm": rate_meas,
                     "frac_of_measured_pair_rate": (achieved / (2 * rate_meas * facts["sms"] * max_mhz * 1e6 / 1e12)
                                                    if rate_meas else None)},
        "phase_time_ms": phase_share,
        "gpu_launches": launches,
        "clocks": ({k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")} if clocks else None),
        # the paper's Table 3 metric: Eq. 1 GFLOPS (2 per relaxation) per watt of
        # board power sampled during the timed region
        "energy": ({"power_w_mean": clocks["power_w_mean"],
                    "eq1_gflops_per_w": gflops_per_watt(eq1_gflops(value / world), clocks["power_w_mean"]),
                    "relax_per_joule": value / world / clocks["power_w_mean"]}
                   if clocks and clocks.get("power_w_mean") else None),
        "device": facts,
    }

    details = {}
    if world > 1 and not args.no_extras and args.dtype == "f32":
        t_shard, share = bench_batched_sharded(torch, apsp, graphgen, args, dev, rank, world)
        t_job = reduce_max(t_shard, world, dev)
        if rank == 0:
            details["batched_sharded"] = {"graphs": 4096, "ranks": world, "split": "LPT by n^3, no collective",
                                          "scaling": "strong", "ms": 1e3 * t_job, "graphs_per_s": 4096 / t_job,
                                          "rank0_share": share}
    if rank == 0 and not args.no_extras and args.dtype == "f32":
        del D
        torch.cuda.empty_cache()
        e2e_value, h2d, d2h, Wh, parts = bench_e2e(torch, apsp, graphgen, W, args)
        line["e2e"] = {"value": e2e_value * world, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "parts_ms": {k: round(v, 2) for k, v in parts.items()}}
        del W, P
        torch.cuda.empty_cache()
        if args.fp64_n > 0:
            n64, t64, prof64 = bench_fp64(torch, apsp, graphgen, args, dev)
            k3 = prof64["phase3_minplus"]
            T64 = apsp.block_size(torch.float64)
            p4_rate = phase3_relax_per_round(n64, T64) * ((n64 + T64 - 1) // T64) / (k3[0] / 1e3 / args.fp64_steps)
            rate64 = apsp.measure_peak(8)  # the lower-bound pair on registers (relax/clk/SM)
            details["fp64"] = {"n": n64, "value": n64 ** 3 / t64, "unit": UNIT, "ms": 1e3 * t64,
                               "path_matrix": True, "steps": args.fp64_steps, "warmup": args.fp64_warmup,
                               "phase_time_ms": {k: {"ms": v[0], "launches": v[1]} for k, v in prof64.items()},
                               "phase3_relax_per_s": p4_rate,
                               "phase3_frac_of_unit_peak": p4_rate / alu_peak_relax_per_s(facts["sms"], max_mhz),
                               "measured_pair_rate_relax_per_clk_sm": rate64,
                               "phase3_frac_of_measured_pair_rate": p4_rate / (rate64 * facts["sms"] * max_mhz * 1e6)}
        torch.cuda.empty_cache()
        details["batched"] = bench_batched(torch, apsp, graphgen, args, dev)
        torch.cuda.empty_cache()
        details["fwd_bwd"] = bench_fwd_bwd(torch, apsp, graphgen, args, dev)
        torch.cuda.empty_cache()
        if args.sweep:
            details["sweep"] = bench_sweep(torch, apsp, graphgen, args, dev, rate_meas)
        if args.sweep_f64:
            details["sweep_f64"] = bench_sweep_f64(torch, apsp, graphgen, args, dev)
        # CPU baseline: the oracle as it stands, bounded prefix of the same graph
        rate, k, thr, tcpu = oracle_partial_rate(Wh.numpy(), args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
                                "sample": f"classic FW (FP32 + P), first {k} of {n} outer k, {tcpu:.1f} s: a prefix "
                                          f"rate (early k write more)"}
        if args.cpu_full:
            details["cpu_full_runs"] = oracle_full_runs(args.cpu_full)
        for key, val in details.items():  # long records first, one line each
            print("# detail " + json.dumps({key: val}), flush=True)
        line["summary"] = summary_of(details, line)
    elif rank != 0:
        del W, D, P
    if rank == 0:
        print("# detail " + json.dumps({"roofline": line["roofline"], "phase_time_ms": line.pop("phase_time_ms"),
                                        "device": line.pop("device"),
                                        "e2e_parts_ms": (line.get("e2e") or {}).get("parts_ms")}), flush=True)
        print(json.dumps(compact_line(line), separators=(",", ":")), flush=True)
    barrier(world)


ROOFLINE_KEYS = ("bound", "achieved", "peak", "unit", "frac", "traffic", "frac_of_measured_pair_rate",
                 "avg_round_ms")


def compact_line(line):
    """The final JSON line: the contract's keys plus short roofline, e2e,
    cpu_baseline and summary objects (the long records are printed before it)."""
    def r4(v):
        return float("%.4g" % v) if isinstance(v, float) else v
    out = dict(line)
    out["roofline"] = {k: r4(line["roofline"][k]) for k in ROOFLINE_KEYS if k in line["roofline"]}
    if out.get("energy"):
        out["energy"] = {k: r4(v) for k, v in out["energy"].items() if k != "relax_per_joule"}
    out["ms_per_step"] = round(out["ms_per_step"], 3)
    if out.get("e2e"):
        out["e2e"] = {k: r4(v) for k, v in out["e2e"].items() if k != "parts_ms"}
    return out


def oracle_full_runs(sizes):
    """Whole classic-FW solves by the CPU oracle (FP32 + path matrix) at small n,
    beside the GPU sweep: relax/s of a complete run, no prefix."""
    import oracle
    import graphgen
    out = []
    for n in sizes:
        W = graphgen.dense_graph(n, 0.5, SEED)
        t0 = time.perf_counter()
        oracle.fw(W, with_path=True)
        t = time.perf_counter() - t0
        out.append({"n": n, "s": t, "relax_per_s": float(n) ** 3 / t, "cores": oracle.num_threads()})
    return out


def summary_of(details, line):
    """The headline numbers of the side measurements, short enough for the final line."""
    out = {}
    f = details.get("fp64")
    if f:
        out["fp64"] = {"value": float("%.4g" % f["value"]), "ms": round(f["ms"], 1),
                       "phase3_frac": round(f["phase3_frac_of_unit_peak"], 4),
                       "phase3_frac_of_pair": round(f["phase3_frac_of_measured_pair_rate"], 4)}
    b = details.get("batched")
    if b:
        out["batched"] = {"graphs_per_s": round(b["graphs_per_s"]), "ms": round(b["ms"], 3),
                          "relax_per_s": float("%.4g" % b["relax_per_s"]), "frac": round(b["frac_of_unit_peak"], 4),
                          "vs_per_graph": round(b["speedup_vs_per_graph"], 1),
                          "no_path_ms": round(b["without_path"]["ms"], 3)}
    bs = details.get("batched_sharded")
    if bs:
        out["batched_sharded"] = {"graphs_per_s": round(bs["graphs_per_s"]), "ranks": bs["ranks"]}
    fb = details.get("fwd_bwd")
    if fb:
        out["fwd_bwd_ms"] = round(fb["fwd_bwd_ms"], 3)
        out["fwd_bwd_per_graph_ms"] = round(fb["per_graph_path"]["fwd_bwd_ms"], 2)
    en = line.get("energy")
    if en:
        out["eq1_gflops_per_w"] = round(en["eq1_gflops_per_w"], 2)
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["single", "batched", "fwd_bwd", "sweep"], default="single",
                    help="single (the headline line) or one side measurement alone")
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32",
                    help="precision of the timed single-graph solve (the headline is f32)")
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--fp64-n", type=int, default=32768)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--fp64-warmup", type=int, default=3)
    ap.add_argument("--cpu-full", type=lambda x: [int(v) for v in x.split(",") if v], default=[4096, 8192],
                    help="sizes at which the CPU oracle runs a whole solve (empty: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--gpu-index", default=None)
    ap.add_argument("--no-extras", action="store_true", help="only the FP32 timed steps")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched: keep the built-in variant table (deterministic launch order for profiling)")
    ap.add_argument("--sweep", type=lambda x: [int(v) for v in x.split(",") if v], default=[4096, 8192, 32768, 65536],
                    help="comma-separated FP32 sizes of the n sweep (empty: skip)")
    ap.add_argument("--no-sweep", dest="sweep", action="store_const", const=[])
    ap.add_argument("--sweep-f64", type=lambda x: [int(v) for v in x.split(",") if v], default=[4096, 8192],
                    help="comma-separated FP64 sizes of the n sweep beside the n=32768 FP64 line (empty: skip)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
