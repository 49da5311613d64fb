"""Sharding a batch of independent graphs over ranks (one process per GPU).

The graphs of a batched workload are independent, so a batch splits across
ranks with no exchange on the data path: each rank packs its own graphs, runs
one batched launch on its GPU, and the results meet again only if the caller
gathers them.  The split balances the work, which for Floyd-Warshall is n^3
relaxations per graph: longest processing time first (graphs by decreasing
n^3, each to the rank with the least work so far; Graham's LPT bound keeps the
largest rank load within 4/3 of the optimum).

Host logic only (numpy); the solving itself is the library's batched entry
point, called by whoever runs the shard.
"""
from __future__ import annotations

import heapq

import numpy as np

from .batched import packed_offsets, packed_numel


def lpt_partition(sizes, world: int) -> list[np.ndarray]:
    """Global graph indices per rank (each sorted ascending), balancing sum n^3."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = np.asarray(sizes, dtype=np.int64)
    work = sizes.astype(np.float64) ** 3
    order = np.argsort(-work, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for g in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(g))
        heapq.heappush(heap, (load + float(work[g]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def rank_loads(sizes, parts) -> np.ndarray:
    """Sum of n^3 per rank."""
    sizes = np.asarray(sizes, dtype=np.float64)
    return np.array([float(np.sum(sizes[p] ** 3)) for p in parts])


class Shard:
    """One rank's share of a packed batch: which global graphs it holds and where
    each sits in the rank's own packed buffer (back to back, 16-byte aligned)."""

    def __init__(self, sizes, ids):
        self.ids = np.asarray(ids, dtype=np.int64)
        self.sizes = np.asarray(sizes, dtype=np.int64)[self.ids]
        self.offsets = packed_offsets(self.sizes)
        self.numel = packed_numel(self.sizes)

    def scatter_into(self, local, global_buf, global_offsets):
        """Copy every graph of the rank's packed buffer ``local`` to its place in
        the global packed buffer (numpy arrays or torch tensors)."""
        for n, lo, g in zip(self.sizes, self.offsets, self.ids):
            e = int(n) * int(n)
            go = int(global_offsets[g])
            global_buf[go:go + e] = local[int(lo):int(lo) + e]

    def gather_from(self, global_buf, global_offsets, local):
        """Copy the rank's graphs out of a global packed buffer into ``local``."""
        for n, lo, g in zip(self.sizes, self.offsets, self.ids):
            e = int(n) * int(n)
            go = int(global_offsets[g])
            local[int(lo):int(lo) + e] = global_buf[go:go + e]


def shards(sizes, world: int) -> list[Shard]:
    """The LPT split of ``sizes`` over ``world`` ranks, as Shard objects."""
    return [Shard(sizes, p) for p in lpt_partition(sizes, world)]
