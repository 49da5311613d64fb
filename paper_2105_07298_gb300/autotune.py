"""Autotuner for the batched kernel: per size class, time every kernel variant
on synthetic graphs of that class and keep the fastest.

The batched launch solves graphs of several size classes at once; each class
may use a different variant.  The variants differ in block edge, register
blocking and path tracking (``batched.variant_info``): 64 x 64 blocks with
4 x 4 register tiles, path entries recovered after each block product (0,
lazy) or kept in the inner loop (1, eager); 128 x 128 blocks with 8 x 4
register tiles, the single-graph phase kernels run by one CTA with eager
tracking (2).  Choices are cached per device name in a JSON file and applied
with :func:`apply_cached`.

Timing only: every variant computes the same distances (bit-exact on integer
weights), so the choice never changes results on integer inputs.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import batched as _b

def _cache_path() -> str:
    """Per-user cache file (outside the build folder, so a clean build keeps it);
    APSP_AUTOTUNE_CACHE overrides it."""
    env = os.environ.get("APSP_AUTOTUNE_CACHE")
    if env:
        return env
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "apsp_fw_gb300", "autotune.json")


CACHE = _cache_path()


def _class_sizes(cls: int, count: int, seed: int):
    lo, hi = _b.class_bounds(cls)
    hi = min(hi, 512)
    rng = np.random.default_rng(seed + cls)
    return rng.integers(lo, hi + 1, size=count).astype(np.int64)


def _random_batch(torch, sizes, off, total, seed, device):
    """Dense random graphs for timing only (edge probability 0.3, integer
    weights 1..100, +inf non-edges, zero diagonal), packed at ``off``."""
    gen = torch.Generator(device="cpu").manual_seed(seed)
    W = torch.full((total,), float("inf"), dtype=torch.float32)
    for n, o in zip(sizes, off):
        n, o = int(n), int(o)
        w = torch.randint(1, 101, (n, n), generator=gen).float()
        w[torch.rand((n, n), generator=gen) >= 0.3] = float("inf")
        w.fill_diagonal_(0)
        W[o:o + n * n] = w.reshape(-1)
    return W.to(device)


def _time_plan(torch, sizes, W, D, P, reps: int) -> float:
    plan = _b.BatchedPlan(sizes, _b.packed_offsets(sizes))
    D.copy_(W)
    plan.run(D, P)  # warm-up
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        D.copy_(W)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        plan.run(D, P)
        e.record()
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e))
    plan.close()
    return float(np.median(times))


def autotune(device="cuda:0", graphs_per_class: int = 608, reps: int = 3, seed: int = 7,
             save: bool = True, verbose: bool = False) -> dict:
    """Choose a variant per size class; returns {class: {"variant", "ms": [per variant]}}."""
    import torch

    result = {}
    for cls in range(_b.num_classes()):
        sizes = _class_sizes(cls, graphs_per_class, seed)
        off = _b.packed_offsets(sizes)
        total = _b.packed_numel(sizes)
        W = _random_batch(torch, sizes, off, total, seed + cls, device)
        D = torch.empty_like(W)
        P = torch.empty(total, dtype=torch.int32, device=device)
        ms = []
        for v in range(_b.num_variants(cls)):
            _b.set_variant(cls, v)
            ms.append(_time_plan(torch, sizes, W, D, P, reps))
        best = int(np.argmin(ms))
        _b.set_variant(cls, best)
        result[cls] = {"variant": best, "ms": ms, "bounds": list(_b.class_bounds(cls)),
                       "shape": _b.variant_info(best)}
        if verbose:
            print(f"class {cls} {_b.class_bounds(cls)}: variant ms {ms} -> {best}")
        del W, D, P
    # Variant 2 needs the two-CTAs-per-SM kernel, which every class then runs
    # on: time the whole mixed batch with the per-class choices and with each
    # variant-2 class set to its best 64-block variant, and keep the faster.
    if any(r["variant"] == 2 for r in result.values()):
        sizes = np.concatenate([_class_sizes(c, graphs_per_class // 2, seed + 100) for c in result])
        off = _b.packed_offsets(sizes)
        total = _b.packed_numel(sizes)
        W = _random_batch(torch, sizes, off, total, seed + 100, device)
        D = torch.empty_like(W)
        P = torch.empty(total, dtype=torch.int32, device=device)
        t_mixed = _time_plan(torch, sizes, W, D, P, max(reps, 5))
        alt = {c: (r["variant"] if r["variant"] != 2 else int(np.argmin(r["ms"][:2]))) for c, r in result.items()}
        for c, v in alt.items():
            _b.set_variant(c, v)
        t_alt = _time_plan(torch, sizes, W, D, P, max(reps, 5))
        # variant 2 stays only if the mixed batch is clearly (3 %) faster with it
        if t_alt <= 1.03 * t_mixed:
            for c, v in alt.items():
                result[c]["variant"] = v
                result[c]["shape"] = _b.variant_info(v)
        else:
            for c, r in result.items():
                _b.set_variant(c, r["variant"])
        if verbose:
            print(f"mixed batch: per-class choice {t_mixed:.3f} ms, without variant 2 {t_alt:.3f} ms")
        del W, D, P
    if save:
        name = torch.cuda.get_device_name(torch.device(device))
        cache = {}
        if os.path.exists(CACHE):
            try:
                cache = json.load(open(CACHE))
            except Exception:
                cache = {}
        cache[name] = {str(c): r["variant"] for c, r in result.items()}
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return result


def apply_cached(device="cuda:0") -> bool:
    """Apply cached choices for this device, if any.  Returns whether any were applied."""
    import torch
    if not os.path.exists(CACHE):
        return False
    try:
        cache = json.load(open(CACHE))
    except Exception:
        return False
    choice = cache.get(torch.cuda.get_device_name(torch.device(device)))
    if not choice:
        return False
    for c, v in choice.items():
        _b.set_variant(int(c), int(v))
    return True
