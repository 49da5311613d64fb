"""Sharding a batch of independent graphs over ranks (the multi-GPU split of the
batched workload), tested with two gloo ranks on CPU.

Each rank packs the graphs its LPT share names, solves them (here with the CPU
oracle standing in for the GPU launch: there is no GPU in these tests), and
rank 0 places every rank's results into the global packed layout.  Checked:
every graph is solved exactly once, the n^3 work is balanced, and each graph's
result sits at its own global offset, equal to the oracle's solve of it.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import graphgen
from paper_2105_07298_gb300 import batched as B
from paper_2105_07298_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SIZES = graphgen.batch_sizes(48, 16, 64, 5)
SEED = 9


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        sh = shard.shards(SIZES, world)[rank]
        local = graphgen.batched_graphs_torch(sh.sizes, 0.3, SEED, sh.offsets, sh.numel,
                                              graph_ids=sh.ids).numpy().copy()
        for n, lo in zip(sh.sizes, sh.offsets):
            e = int(n) * int(n)
            local[lo:lo + e] = oracle.fw(local[lo:lo + e].reshape(n, n))[0].reshape(-1)
        gathered = [None] * world
        dist.all_gather_object(gathered, (rank, sh.ids.tolist(), local))
        if rank == 0:
            goff = B.packed_offsets(SIZES)
            gbuf = np.full(B.packed_numel(SIZES), np.nan, dtype=np.float32)
            seen = []
            for r, ids, buf in gathered:
                shard.Shard(SIZES, ids).scatter_into(buf, gbuf, goff)
                seen += ids
            out.put((sorted(seen), gbuf))
    finally:
        dist.destroy_process_group()


def test_two_ranks_solve_every_graph_once_at_its_place():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    seen, gbuf = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert seen == list(range(len(SIZES)))  # every graph exactly once
    goff = B.packed_offsets(SIZES)
    W = graphgen.batched_graphs_torch(SIZES, 0.3, SEED, goff, B.packed_numel(SIZES)).numpy()
    for g, (n, o) in enumerate(zip(SIZES, goff)):
        e = int(n) * int(n)
        ref = oracle.fw(W[o:o + e].reshape(n, n))[0]
        np.testing.assert_array_equal(gbuf[o:o + e].reshape(n, n), ref)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_lpt_split_of_the_batched_workload_is_balanced(world):
    """4096 graphs, n uniform on [16, 512]: a disjoint cover, and the largest
    rank load within 1 % of the mean (well inside Graham's 4/3 bound)."""
    sizes = graphgen.batch_sizes(4096, 16, 512, 1)
    parts = shard.lpt_partition(sizes, world)
    allg = np.sort(np.concatenate(parts))
    np.testing.assert_array_equal(allg, np.arange(len(sizes)))
    loads = shard.rank_loads(sizes, parts)
    assert loads.sum() == pytest.approx(float(np.sum(sizes.astype(np.float64) ** 3)))
    assert loads.max() <= 1.01 * loads.mean()


def test_shard_layout_round_trip():
    sizes = [5, 17, 3, 64, 9]
    sh = shard.Shard(sizes, [3, 0, 4])
    goff = B.packed_offsets(sizes)
    g = np.arange(B.packed_numel(sizes), dtype=np.float32)
    local = np.zeros(sh.numel, dtype=np.float32)
    sh.gather_from(g, goff, local)
    back = np.full_like(g, -1)
    sh.scatter_into(local, back, goff)
    for idx in (3, 0, 4):
        e = sizes[idx] ** 2
        np.testing.assert_array_equal(back[goff[idx]:goff[idx] + e], g[goff[idx]:goff[idx] + e])
    assert (sh.offsets % 4 == 0).all()
