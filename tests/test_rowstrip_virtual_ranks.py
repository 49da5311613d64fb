"""Row-strip split of one graph's blocked FW over ranks, on CPU virtual ranks.

The design for several GPUs (not built as a device path: every run here has
one GPU): rank g holds only its strip of block rows of D and P plus one
receive buffer of T rows.  In round r the owner of block row r runs phase 1 on
the diagonal block and phase 2 on the rest of its pivot row of blocks (§2.2,
"Blocked FW Algorithm"), then broadcasts that row of blocks (T x n values, the
round's only exchange); every rank runs phase 3 on its blocks of column r and
phase 4 on its other blocks, reading the pivot row only from the broadcast.

Checked with gloo ranks (2 and 3, ragged last block, a rank whose strip holds
the ragged block): D and P gathered from the strips equal the oracle's
sequential blocked FW bit for bit on real FP32 weights (the split changes no
sum and no order of k), and over a solve each rank receives 4 bytes for
every element of the rows it does not hold (n^2 x 4 bytes less its own strip).  The per-rank arithmetic below is the four phases written out in numpy,
k ascending with the strict test, standing in for the kernels.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import graphgen


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def strip_of(rank, world, R):
    """Block rows [I0, I1) held by ``rank``: contiguous, as even as R allows."""
    return R * rank // world, R * (rank + 1) // world


def _relax(X, PX, a, b, k):
    """X = min(X, a[:, None] + b[None, :]) with P = k where strictly smaller."""
    cand = a[:, None] + b[None, :]
    better = cand < X
    X[better] = cand[better]
    PX[better] = k


def _worker(rank, world, port, n, T, weights, seed, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        R = (n + T - 1) // T
        I0, I1 = strip_of(rank, world, R)
        a, b = min(n, I0 * T), min(n, I1 * T)  # global rows a..b-1 live here
        W = graphgen.dense_graph(n, 0.4, seed, weights=weights,
                                 lo=0.5 if weights == "real" else 1, hi=2.0 if weights == "real" else 100)
        L = W[a:b].astype(np.float32).copy()            # this rank's strip of D
        PL = np.full(L.shape, -1, dtype=np.int32)       # and of P
        del W                                           # nothing else of the graph is kept
        panel = torch.empty((T, n), dtype=torch.float32)  # receive buffer for the pivot row
        received = 0
        for r in range(R):
            k0, k1 = r * T, min(n, r * T + T)
            m = k1 - k0
            owner = next(g for g in range(world) if strip_of(g, world, R)[0] <= r < strip_of(g, world, R)[1])
            if rank == owner:
                pr = slice(k0 - a, k1 - a)
                rest = np.r_[0:k0, k1:n]
                for k in range(k0, k1):  # phase 1: the diagonal block against itself
                    blk, pblk = L[pr, k0:k1], PL[pr, k0:k1]
                    _relax(blk, pblk, blk[:, k - k0].copy(), blk[k - k0].copy(), k)
                for k in range(k0, k1):  # phase 2: the pivot row of blocks
                    rowblk, prow = L[pr][:, rest], PL[pr][:, rest]
                    _relax(rowblk, prow, L[pr, k].copy(), L[k - a, rest].copy(), k)
                    L[pr, rest], PL[pr, rest] = rowblk, prow
                panel[:m] = torch.from_numpy(L[pr])
            dist.broadcast(panel[:m], src=owner)
            if rank != owner:
                received += m * n * 4
            piv = panel[:m].numpy()
            mine = np.array([i - a for i in range(a, b) if not (k0 <= i < k1)], dtype=np.int64)
            if len(mine) == 0:
                continue
            rest = np.r_[0:k0, k1:n]
            for k in range(k0, k1):  # phase 3: this rank's blocks of column r
                colblk, pcol = L[mine, k0:k1], PL[mine, k0:k1]
                _relax(colblk, pcol, colblk[:, k - k0].copy(), piv[k - k0, :].copy()[k0:k1], k)
                L[mine, k0:k1], PL[mine, k0:k1] = colblk, pcol
            for k in range(k0, k1):  # phase 4: every other block of the strip
                blk, pblk = L[mine][:, rest], PL[mine][:, rest]
                _relax(blk, pblk, L[mine, k].copy(), piv[k - k0, rest].copy(), k)
                L[mine[:, None], rest[None, :]] = blk
                PL[mine[:, None], rest[None, :]] = pblk
        parts = [None] * world
        dist.all_gather_object(parts, (a, b, L, PL, received, panel.shape))
        if rank == 0:
            out.put(parts)
    finally:
        dist.destroy_process_group()


def _run(world, n, T, weights, seed):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, T, weights, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return parts


@pytest.mark.parametrize("world,n,T", [(2, 150, 32), (3, 150, 32), (3, 97, 16)])
def test_row_strips_equal_the_sequential_blocked_fw(world, n, T):
    import oracle
    parts = _run(world, n, T, "real", 31 + world)
    D = np.concatenate([p[2] for p in parts])
    P = np.concatenate([p[3] for p in parts])
    assert D.shape == (n, n) and parts[0][0] == 0 and parts[-1][1] == n
    assert all(parts[g][1] == parts[g + 1][0] for g in range(world - 1))  # strips tile the rows
    W = graphgen.dense_graph(n, 0.4, 31 + world, weights="real", lo=0.5, hi=2.0)
    Db, Pb = oracle.bfw(W, T)
    np.testing.assert_array_equal(D, Db)
    np.testing.assert_array_equal(P, Pb)
    # one pivot row of blocks per round is the only exchange: n^2 values in all,
    # less the rows a rank owns itself
    for a, b, L, _, received, shape in parts:
        assert received == (n - (b - a)) * n * 4
        assert L.shape == (b - a, n) and shape == (T, n)


def test_row_strips_integer_weights_equal_classic_fw():
    import oracle
    n, T, world = 130, 32, 2
    parts = _run(world, n, T, "int", 5)
    D = np.concatenate([p[2] for p in parts])
    P = np.concatenate([p[3] for p in parts])
    W = graphgen.dense_graph(n, 0.4, 5)
    np.testing.assert_array_equal(D.astype(np.float64), oracle.fw(W.astype(np.float64))[0])
    assert oracle.check_paths(W, D, P) == 0
