"""Host-side logic of bench.py on CPU: the clock/throttle summary, the gate
that keeps a recorded DRAM traffic figure only for the kernel source it was
measured on, and the per-round work count of phase 4."""
import os

import pytest

import bench


def _clock_line(sm, smax, power, reasons=("Not Active",) * 5):
    return ", ".join(["0", str(sm), str(smax), str(power), *reasons]) + "\n"


def test_clock_summary_median_power_and_reasons(tmp_path):
    p = tmp_path / "clk.csv"
    idle = _clock_line(345, 2070, 90.0)
    busy = [_clock_line(2070, 2070, 500.0 + i) for i in range(5)]
    capped = _clock_line(1980, 2070, 640.0, ("Active", "Not Active", "Not Active", "Not Active", "Active"))
    p.write_text(idle + "".join(busy) + capped + "garbage line\n")
    c = bench.ClockSampler()
    c.proc, c.path = object(), str(p)  # as if the sampler had run
    s = c.summary()
    assert s["sm_mhz"] == 2070.0           # median over loaded samples (power > 200 W)
    assert s["sm_max_mhz"] == 2070.0
    assert s["power_w_max"] == 640.0
    assert s["samples"] == 7
    assert s["reasons"] == ["sw_power_cap"]
    assert 500.0 < s["power_w_mean"] < 640.0


def test_clock_summary_flags_thermal_slowdown(tmp_path):
    p = tmp_path / "clk.csv"
    p.write_text(_clock_line(1500, 2070, 600.0, ("Active", "Not Active", "Active", "Not Active", "Not Active")))
    c = bench.ClockSampler()
    c.proc, c.path = object(), str(p)
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_traffic_kept_only_for_the_measured_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "phase3_minplus_f32_traffic.txt").write_text(
        "# comment\nkernel_source_hash: 0123abcd\ndram_bytes_per_round_n32768: 5.5e9\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0123abcd")
    assert bench.profiled_traffic(32768) == pytest.approx(5.5e9)
    assert bench.profiled_traffic(16384) is None        # no figure for that size
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "ffffffff")
    assert bench.profiled_traffic(32768) is None        # kernel changed since the capture


def test_committed_traffic_record_is_well_formed():
    """The committed record names a hash and a per-round byte count."""
    path = os.path.join(bench.ROOT, "profiles", "phase3_minplus_f32_traffic.txt")
    txt = open(path).read()
    assert "kernel_source_hash:" in txt and "dram_bytes_per_round_n32768:" in txt


def test_phase4_work_per_round_counts_every_k_of_the_round():
    # n a multiple of T: every round relaxes (n - T)^2 outputs with T values of k
    assert bench.phase3_relax_per_round(1024, 128) == pytest.approx((1024 - 128) ** 2 * 128)
    # a single block has no phase 4
    assert bench.phase3_relax_per_round(100, 128) == 0


def test_recorded_profiler_captures_stay_small():
    """Every ncu command recorded under profiles/ that collects more than the
    per-launch duration captures at most three launches (-c), and every one
    names --clock-control none: the full-size workload is only ever listed
    with durations (one pass)."""
    import glob
    import re
    cmds = []
    for path in glob.glob(os.path.join(bench.ROOT, "profiles", "*")):
        txt = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"^[#\s]*(ncu\s(?!-i\b).*)$", txt, flags=re.M):
            cmds.append((os.path.basename(path), m.group(1)))
    assert cmds
    for name, cmd in cmds:
        assert "--clock-control none" in cmd, (name, cmd)
        metrics = re.search(r"--metrics\s+(\S+)", cmd)
        only_duration = metrics is not None and metrics.group(1) == "gpu__time_duration.sum" and "--set" not in cmd
        if not only_duration:
            count = re.search(r"\s-c\s+(\d+)", cmd)
            assert count and int(count.group(1)) <= 3, (name, cmd)


def test_final_line_stays_short_and_carries_every_headline():
    """The last JSON line (the one a log tail keeps) holds the FP32 value, the
    roofline, e2e, the CPU baseline and the summary of the FP64, batched (with
    and without P) and forward+backward numbers in under 1.5 KB; the long
    records (sweeps, per-phase times, e2e parts) go to the detail lines."""
    import json
    details = {
        "fp64": {"value": 1.299e13, "ms": 2708.0, "phase3_frac_of_unit_peak": 0.3209,
                 "phase3_frac_of_measured_pair_rate": 0.4562, "phase_time_ms": {"x": {"ms": 1.0, "launches": 3}}},
        "batched": {"graphs_per_s": 183160.2, "ms": 22.363, "relax_per_s": 6.476e12, "frac_of_unit_peak": 0.1608,
                    "speedup_vs_per_graph": 55.4, "without_path": {"ms": 15.614, "relax_per_s": 9.3e12,
                                                                   "frac_of_unit_peak": 0.23},
                    "autotuned_variants": {str(c): {"ms_per_variant": [1.0, 2.0, 3.0]} for c in range(4)}},
        "fwd_bwd": {"fwd_bwd_ms": 1.198, "per_graph_path": {"fwd_bwd_ms": 72.36}},
        "sweep": {"points": [{"n": n, "with_path": {"relax_per_s": 1e13}} for n in (4096, 8192, 32768, 65536)]},
        "sweep_f64": {"points": [{"n": n, "relax_per_s": 5e12} for n in (4096, 8192)]},
    }
    line = {"metric": bench.METRIC, "value": 1.557e13, "unit": bench.UNIT, "n_gpus": 1, "steps": 3, "warmup": 3,
            "ms_per_step": 2261.3361, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": bench.workload_config(32768, 1, "f32"),
            "roofline": {"bound": "alu", "achieved": 30.95123, "peak": 80.55, "unit": "TFLOP/s", "frac": 0.38421,
                         "traffic": 5.737e9, "frac_of_measured_pair_rate": 0.5481, "avg_round_ms": 8.812,
                         "flop_def": "x" * 200, "peak_basis": "y" * 100},
            "gpu_launches": 3072, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
            "energy": {"power_w_mean": 542.0, "eq1_gflops_per_w": 57.44, "relax_per_joule": 2.9e10},
            "e2e": {"value": 1.27e13, "unit": bench.UNIT, "h2d_bytes_per_step": 1 << 32,
                    "d2h_bytes_per_step": 1 << 33, "parts_ms": {"step_ms": 2765.33, "host_wall_ms": 2765.38}},
            "cpu_baseline": {"value": 2.0e10, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
                             "sample": "classic FW (FP32 + P), first 137 of 32768 outer k, 7.3 s: a prefix rate (early k write more)"}}
    line["summary"] = bench.summary_of(details, line)
    out = json.dumps(bench.compact_line(line), separators=(",", ":"))
    assert len(out) < 1500
    d = json.loads(out)
    assert set(bench.ROOFLINE_KEYS) >= set(d["roofline"]) and "flop_def" not in d["roofline"]
    s = d["summary"]
    assert s["fp64"]["value"] == 1.299e13 and s["batched"]["no_path_ms"] == 15.614
    assert s["fwd_bwd_ms"] == 1.198 and "parts_ms" not in d["e2e"]
    for key in ("e2e", "cpu_baseline", "clocks", "gpu_launches"):
        assert key in d


def test_cpu_baseline_sample_is_a_measured_prefix():
    """The CPU baseline times a prefix of the oracle's outer k loop: k between
    the probe and n, a positive rate n^2 k / t, the oracle's thread count."""
    import graphgen
    import oracle
    W = graphgen.dense_graph(256, 0.5, bench.SEED)
    rate, k, threads, t = bench.oracle_partial_rate(W, 0.05, probe_k=8)
    assert 8 <= k <= 256 and t > 0 and threads == oracle.num_threads() >= 1
    assert rate == pytest.approx(k * 256.0 ** 2 / t)
    runs = bench.oracle_full_runs([128])
    assert runs[0]["n"] == 128 and runs[0]["relax_per_s"] == pytest.approx(128.0 ** 3 / runs[0]["s"])
