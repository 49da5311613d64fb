"""Seeded synthetic graph inputs for all-pairs shortest paths.

This module only *draws* inputs.  It holds none of the shortest-path
arithmetic: no relaxation, no path logic, no gradient rule.  Both the CPU
oracle tests and the CUDA path take their inputs from here, so the two see the
same bytes without either importing the other.

Graphs are dense weight matrices ``W`` (row-major, ``W[i, j]`` = weight of the
directed edge i -> j).  Missing edges are ``+inf`` and the diagonal is 0, which
is the input convention of the Floyd-Warshall algorithm (paper §2.2,
Algorithm 1: a dense N x N distance matrix, infinity where there is no edge).

Randomness is counter based: every element (i, j) of graph ``seed`` gets two
32-bit hashes of its linear index ``e = i * n + j`` (MurmurHash3's 32-bit
finaliser, Appleby 2011, applied to ``lo32(e) xor fmix(hi32(e))`` xor a
per-stream key; fmix(0) = 0, so below 2^32 elements this is ``e`` xor the key).
The numpy and the torch implementations below compute the same integers, so a
matrix drawn on the GPU for a large benchmark equals the one numpy draws on
the host.

* edge present   <=>  h_edge < round(p * 2**32)
* integer weight  =   lo + h_weight mod (hi - lo + 1)
* real weight     =   lo + (hi - lo) * h_weight / 2**32   (computed in float64)
"""
from __future__ import annotations

import numpy as np

_M32 = 0xFFFFFFFF
_C1 = 0x85EBCA6B
_C2 = 0xC2B2AE35


def _fmix32_np(h: np.ndarray) -> np.ndarray:
    h = h.astype(np.uint64) & _M32
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(_C1)) & np.uint64(_M32)
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(_C2)) & np.uint64(_M32)
    h ^= h >> np.uint64(16)
    return h


def _fmix32_int(h: int) -> int:
    h &= _M32
    h ^= h >> 16
    h = (h * _C1) & _M32
    h ^= h >> 13
    h = (h * _C2) & _M32
    h ^= h >> 16
    return h


def _index_word_np(e: np.ndarray) -> np.ndarray:
    """32-bit word hashed for linear index e (uint64): lo32(e) xor fmix(hi32(e))."""
    e = e.astype(np.uint64)
    return (e & np.uint64(_M32)) ^ _fmix32_np(e >> np.uint64(32))


def stream_keys(seed: int) -> tuple[int, int]:
    """The two 32-bit keys (edge stream, weight stream) of graph ``seed``."""
    s = int(seed) & _M32
    return _fmix32_int(2 * s + 0x9E3779B9), _fmix32_int(2 * s + 1 + 0x7F4A7C15)


def _check_size(n: int) -> None:
    if n < 0 or n > (1 << 31):
        raise ValueError(f"n={n}: out of range")


def dense_graph(n: int, p: float, seed: int, *, weights: str = "int", lo: float = 1,
                hi: float = 100, dtype=np.float32) -> np.ndarray:
    """Seeded Bernoulli(p) directed graph as a dense n x n weight matrix (numpy).

    ``weights="int"``: integer weights uniform on [lo, hi]; ``"real"``: uniform
    on [lo, hi).  Non-edges are +inf, the diagonal is 0.
    """
    _check_size(n)
    ke, kw = stream_keys(seed)
    e = _index_word_np(np.arange(n * n, dtype=np.uint64))
    he = _fmix32_np(e ^ np.uint64(ke))
    hw = _fmix32_np(e ^ np.uint64(kw))
    thr = np.uint64(min(int(round(p * 2.0 ** 32)), 1 << 32))
    present = he < thr
    if weights == "int":
        span = np.uint64(int(hi) - int(lo) + 1)
        w = (np.float64(lo) + (hw % span).astype(np.float64))
    elif weights == "real":
        w = np.float64(lo) + (np.float64(hi) - np.float64(lo)) * (hw.astype(np.float64) / 2.0 ** 32)
    else:
        raise ValueError(weights)
    out = np.where(present, w, np.inf).astype(dtype).reshape(n, n)
    np.fill_diagonal(out, 0)
    return out


def _torch_fmix(torch, device):
    M = torch.tensor(_M32, dtype=torch.int64, device=device)

    def fmix(h):
        h = h & M
        h = h ^ (h >> 16)
        h = (h * _C1) & M
        h = h ^ (h >> 13)
        h = (h * _C2) & M
        h = h ^ (h >> 16)
        return h
    return fmix, M


def dense_graph_rows_torch(n: int, r0: int, r1: int, p: float, seed: int, *, weights: str = "int",
                           lo: float = 1, hi: float = 100, dtype=None, device="cpu"):
    """Rows r0..r1-1 of the matrix :func:`dense_graph` draws (same values), as an
    (r1 - r0, n) torch tensor on ``device``."""
    import torch

    _check_size(n)
    dtype = dtype or torch.float32
    ke, kw = stream_keys(seed)
    thr = min(int(round(p * 2.0 ** 32)), 1 << 32)
    fmix, M = _torch_fmix(torch, device)
    cols = torch.arange(n, dtype=torch.int64, device=device)
    rows = torch.arange(r0, r1, dtype=torch.int64, device=device)
    e = rows[:, None] * n + cols[None, :]
    e = (e & M) ^ fmix(e >> 32)
    he = fmix(e ^ ke)
    hw = fmix(e ^ kw)
    del e
    if weights == "int":
        w = float(lo) + (hw % (int(hi) - int(lo) + 1)).to(torch.float64)
    elif weights == "real":
        w = float(lo) + (float(hi) - float(lo)) * (hw.to(torch.float64) / 2.0 ** 32)
    else:
        raise ValueError(weights)
    w = torch.where(he < thr, w, torch.full_like(w, float("inf")))
    blk = w.to(dtype)
    idx = torch.arange(r0, r1, device=device)
    blk[idx - r0, idx] = 0
    return blk


def dense_graph_torch(n: int, p: float, seed: int, *, weights: str = "int", lo: float = 1,
                      hi: float = 100, dtype=None, device="cpu", out=None, ld: int | None = None,
                      rows_per_chunk: int = 2048):
    """The same matrix as :func:`dense_graph`, drawn with torch on ``device``.

    Works in row chunks so that a 32768 x 32768 draw needs only a few GB of
    temporaries.  ``out`` (optional) is an (n, ld) tensor to fill in place.
    """
    import torch

    _check_size(n)
    dtype = dtype or torch.float32
    ld = ld or n
    if out is None:
        out = torch.empty((n, ld), dtype=dtype, device=device)
    rows_per_chunk = max(1, min(rows_per_chunk, (1 << 27) // max(n, 1)))
    for r0 in range(0, n, rows_per_chunk):
        r1 = min(n, r0 + rows_per_chunk)
        out[r0:r1, :n] = dense_graph_rows_torch(n, r0, r1, p, seed, weights=weights, lo=lo, hi=hi,
                                                dtype=dtype, device=device)
    if ld > n:
        out[:, n:] = float("nan")  # padding columns: never read by a correct kernel
    return out


def batch_sizes(num_graphs: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Seeded vertex counts, uniform on [lo, hi], one per graph (int64)."""
    k, _ = stream_keys(seed ^ 0x5BD1E995)
    g = np.arange(num_graphs, dtype=np.uint64)
    h = _fmix32_np(g ^ np.uint64(k))
    return (lo + (h % np.uint64(hi - lo + 1))).astype(np.int64)


def batch_offsets(sizes) -> np.ndarray:
    """Element offsets of graphs packed back to back, each n_g x n_g row-major."""
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes * sizes, out=off[1:])
    return off


def batched_graphs(sizes, p: float, seed: int, **kw) -> list[np.ndarray]:
    """One dense graph per entry of ``sizes``; graph g uses seed ``seed * 1000003 + g``."""
    return [dense_graph(int(n), p, seed * 1000003 + g, **kw) for g, n in enumerate(sizes)]


def pack(mats) -> np.ndarray:
    """Concatenate row-major matrices into one flat buffer (see :func:`batch_offsets`)."""
    return np.concatenate([np.ascontiguousarray(m).reshape(-1) for m in mats]) if len(mats) else np.zeros(0)


def normal(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """Seeded standard-normal array (upstream gradients for the backward pass)."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


# ---- structured graphs with known shortest paths (inputs for closed-form tests) ----

def chain_graph(weights, dtype=np.float64) -> np.ndarray:
    """Directed chain 0 -> 1 -> ... -> m with edge (t, t+1) of weight weights[t]."""
    m = len(weights)
    W = np.full((m + 1, m + 1), np.inf, dtype=dtype)
    np.fill_diagonal(W, 0)
    for t, w in enumerate(weights):
        W[t, t + 1] = w
    return W


def complete_graph(n: int, w: float, dtype=np.float64) -> np.ndarray:
    W = np.full((n, n), w, dtype=dtype)
    np.fill_diagonal(W, 0)
    return W


def grid_graph(rows: int, cols: int, dtype=np.float64) -> np.ndarray:
    """Unit-weight 4-neighbour grid, both directions; vertex (r, c) = r * cols + c."""
    n = rows * cols
    W = np.full((n, n), np.inf, dtype=dtype)
    np.fill_diagonal(W, 0)
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                W[v, v + 1] = W[v + 1, v] = 1
            if r + 1 < rows:
                W[v, v + cols] = W[v + cols, v] = 1
    return W


def star_graph(spoke_in, spoke_out, dtype=np.float64) -> np.ndarray:
    """Centre 0; leaf t (1..m) has edge t -> 0 of weight spoke_in[t-1] and 0 -> t of spoke_out[t-1]."""
    m = len(spoke_in)
    W = np.full((m + 1, m + 1), np.inf, dtype=dtype)
    np.fill_diagonal(W, 0)
    for t in range(1, m + 1):
        W[t, 0] = spoke_in[t - 1]
        W[0, t] = spoke_out[t - 1]
    return W


def random_tree_graph(n: int, seed: int, lo=0.5, hi=2.0, dtype=np.float64) -> tuple[np.ndarray, np.ndarray]:
    """Random out-tree rooted at 0 (edge parent[v] -> v), real weights; returns (W, parent)."""
    rng = np.random.default_rng(seed)
    parent = np.full(n, -1, dtype=np.int64)
    W = np.full((n, n), np.inf, dtype=dtype)
    np.fill_diagonal(W, 0)
    for v in range(1, n):
        parent[v] = rng.integers(0, v)
        W[parent[v], v] = rng.uniform(lo, hi)
    return W, parent


def batched_graphs_torch(sizes, p: float, seed: int, offsets, total: int, *, weights: str = "int",
                         lo: float = 1, hi: float = 100, device="cpu", dtype=None, graph_ids=None):
    """All graphs of :func:`batched_graphs` drawn at once with torch into one packed
    buffer of ``total`` elements (graph g at element offsets[g]); element values are
    identical to the numpy draw (same per-graph seeds and hashes).  ``graph_ids``
    (optional) gives each entry's index in a larger batch, whose seed it then
    uses (a rank drawing only its share of a batch)."""
    import torch

    dtype = dtype or torch.float32
    sizes = np.asarray(sizes, dtype=np.int64)
    out = torch.full((total,), float("nan"), dtype=dtype, device=device)
    if len(sizes) == 0:
        return out
    ids = range(len(sizes)) if graph_ids is None else [int(g) for g in graph_ids]
    keys = np.array([stream_keys(seed * 1000003 + g) for g in ids], dtype=np.int64)
    thr = min(int(round(p * 2.0 ** 32)), 1 << 32)
    M = torch.tensor(_M32, dtype=torch.int64, device=device)

    def fmix(h):
        h = h & M
        h = h ^ (h >> 16)
        h = (h * _C1) & M
        h = h ^ (h >> 13)
        h = (h * _C2) & M
        h = h ^ (h >> 16)
        return h

    # process graphs in groups to bound temporaries
    g0 = 0
    while g0 < len(sizes):
        g1 = g0
        acc = 0
        while g1 < len(sizes) and (acc == 0 or acc + sizes[g1] ** 2 <= (1 << 26)):
            acc += int(sizes[g1]) ** 2
            g1 += 1
        cnt = torch.as_tensor(sizes[g0:g1] ** 2, device=device)
        gid = torch.repeat_interleave(torch.arange(g0, g1, device=device), cnt)
        start = torch.cumsum(cnt, 0) - cnt
        e = torch.arange(acc, device=device) - torch.repeat_interleave(start, cnt)  # local index i*n+j
        ke = torch.as_tensor(keys[g0:g1, 0], device=device)[gid - g0]
        kw = torch.as_tensor(keys[g0:g1, 1], device=device)[gid - g0]
        he = fmix(e ^ ke)
        hw = fmix(e ^ kw)
        if weights == "int":
            w = float(lo) + (hw % (int(hi) - int(lo) + 1)).to(torch.float64)
        else:
            w = float(lo) + (float(hi) - float(lo)) * (hw.to(torch.float64) / 2.0 ** 32)
        w = torch.where(he < thr, w, torch.full_like(w, float("inf")))
        nn = torch.as_tensor(sizes[g0:g1], device=device)[gid - g0]
        w = torch.where((e // nn) == (e % nn), torch.zeros_like(w), w)
        dst = torch.as_tensor(np.asarray(offsets, dtype=np.int64)[g0:g1], device=device)[gid - g0] + e
        out[dst] = w.to(dtype)
        g0 = g1
    return out
