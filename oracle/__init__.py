"""CPU oracle for Floyd-Warshall all-pairs shortest paths (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2105_07298_gb300`` never does, and this package never imports it.

The arithmetic lives in ``fw_oracle.c`` (plain C, built with gcc, OpenMP over
independent rows only).  This module builds it, loads it with ctypes and adds
numpy-level helpers: path reconstruction/validation and a pure-Python
simple-path enumerator for tiny graphs.

Readings of the paper used here:
  * strict "<" in Algorithm 1 (the printed ">=" makes path reconstruction loop
    forever at k = j);
  * P = -1 marks "no intermediate vertex" (direct edge, i == j or unreachable);
  * IEEE +inf for "no path" (§2.2's footnote uses the maximum positive number).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fw_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def compile_library(src: str, out: str) -> str:
    """Compile a C source with the oracle's flags (gcc, -O2, OpenMP, no fp
    contraction) into the shared library ``out``."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile fw_oracle.c into liboracle.so (if missing or older than the source)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_library(_SRC, _LIB_PATH)


def load_library(path: str):
    """Load a build of fw_oracle.c and declare its exported signatures."""
    L = ctypes.CDLL(path)
    for name in ("oracle_fw_f64", "oracle_fw_f32"):
        getattr(L, name).argtypes = [_p, _i64, _p, _i64]
        getattr(L, name).restype = None
    for name in ("oracle_bfw_f64", "oracle_bfw_f32"):
        getattr(L, name).argtypes = [_p, _i64, _i64, _p]
        getattr(L, name).restype = ctypes.c_int
    L.oracle_dijkstra_f64.argtypes = [_p, _i64, _i64, _p]
    L.oracle_dijkstra_rows.argtypes = [_p, ctypes.c_int, _i64, _p, _i64, _p]
    L.oracle_bellman_ford_f64.argtypes = [_p, _i64, _i64, _p]
    L.oracle_bellman_ford_f64.restype = ctypes.c_int
    L.oracle_reconstruct_path.argtypes = [_p, _i64, _i64, _i64, _p, _i64]
    L.oracle_reconstruct_path.restype = _i64
    L.oracle_fw_backward_f64.argtypes = [_p, _p, _p, _i64, _p]
    L.oracle_fw_backward_f64.restype = ctypes.c_int
    L.oracle_num_threads.restype = ctypes.c_int
    L.oracle_minplus_rows_f32.argtypes = [_p, _i64, _i64, _p, _i64, _i64, _p]
    L.oracle_minplus_rows_f32.restype = None
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _real(dtype):
    dt = np.dtype(dtype)
    if dt == np.float32:
        return np.float32, "f32"
    if dt == np.float64:
        return np.float64, "f64"
    raise TypeError(f"unsupported dtype {dtype}")


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def fw(W: np.ndarray, with_path: bool = True, k_end: int | None = None):
    """Classic Floyd-Warshall (Algorithm 1, strict '<') in W's precision.

    Returns (D, P) with P None when ``with_path`` is false.  ``k_end`` runs only
    the first k_end outer iterations (each is n^2 relaxations).
    """
    dt, tag = _real(W.dtype)
    n = W.shape[0]
    D = np.ascontiguousarray(W, dtype=dt).copy()
    P = np.empty((n, n), dtype=np.int32) if with_path else None
    getattr(lib(), f"oracle_fw_{tag}")(_ptr(D), n, _ptr(P) if P is not None else None,
                                         -1 if k_end is None else int(k_end))
    return D, P


def bfw(W: np.ndarray, TB: int, with_path: bool = True):
    """Blocked Floyd-Warshall (§2.2 'Blocked FW Algorithm', 4 phases/round) in W's precision."""
    dt, tag = _real(W.dtype)
    n = W.shape[0]
    D = np.ascontiguousarray(W, dtype=dt).copy()
    P = np.empty((n, n), dtype=np.int32) if with_path else None
    rc = getattr(lib(), f"oracle_bfw_{tag}")(_ptr(D), n, int(TB), _ptr(P) if P is not None else None)
    if rc:
        raise ValueError("bad block size")
    return D, P


def dijkstra(W: np.ndarray, src: int) -> np.ndarray:
    """Single-source Dijkstra (non-negative weights), fp64."""
    W64 = np.ascontiguousarray(W, dtype=np.float64)
    n = W64.shape[0]
    out = np.empty(n, dtype=np.float64)
    lib().oracle_dijkstra_f64(_ptr(W64), n, int(src), _ptr(out))
    return out


def dijkstra_rows(W: np.ndarray, srcs) -> np.ndarray:
    """Dijkstra from each source in ``srcs`` (threads over sources); rows in fp64."""
    W = np.ascontiguousarray(W)
    if W.dtype not in (np.float32, np.float64):
        W = W.astype(np.float64)
    srcs = np.ascontiguousarray(srcs, dtype=np.int64)
    n = W.shape[0]
    out = np.empty((len(srcs), n), dtype=np.float64)
    lib().oracle_dijkstra_rows(_ptr(W), int(W.dtype == np.float32), n, _ptr(srcs), len(srcs), _ptr(out))
    return out


def minplus_rows_accumulate(Drows: np.ndarray, Wchunk: np.ndarray, k0: int, best: np.ndarray) -> None:
    """best[t, j] = min(best[t, j], min over chunk rows k != j of Drows[t, k] + W[k, j])
    (float32 inputs, float64 accumulator, in place).  With best started at +inf
    and every chunk of W fed once, a sampled row of exact distances from source
    i has Drows[t, i] = 0 and Drows[t, j] == best[t, j] for all j != i (the
    Bellman equations; positive weights)."""
    Drows = np.ascontiguousarray(Drows, dtype=np.float32)
    Wchunk = np.ascontiguousarray(Wchunk, dtype=np.float32)
    s, n = Drows.shape
    kc = Wchunk.shape[0]
    assert Wchunk.shape[1] == n and best.shape == (s, n) and best.dtype == np.float64 and best.flags.c_contiguous
    lib().oracle_minplus_rows_f32(_ptr(Drows), s, n, _ptr(Wchunk), int(k0), kc, _ptr(best))


def bellman_ford(W: np.ndarray, src: int):
    """Single-source Bellman-Ford (any sign), fp64.  Returns (dist, has_negative_cycle)."""
    W64 = np.ascontiguousarray(W, dtype=np.float64)
    n = W64.shape[0]
    out = np.empty(n, dtype=np.float64)
    neg = lib().oracle_bellman_ford_f64(_ptr(W64), n, int(src), _ptr(out))
    return out, bool(neg)


def reconstruct_path(P: np.ndarray, i: int, j: int, max_len: int | None = None):
    """Vertex list of path(i, j) encoded by P, or None if it does not terminate within max_len."""
    P = np.ascontiguousarray(P, dtype=np.int32)
    n = P.shape[0]
    ld = P.shape[1]
    max_len = max_len or (n + 1)
    buf = np.empty(max_len, dtype=np.int64)
    ln = lib().oracle_reconstruct_path(_ptr(P), ld, int(i), int(j), _ptr(buf), max_len)
    return None if ln < 0 else buf[:ln].tolist()


def reconstruct_path_lookup(p_at, i: int, j: int, max_len: int):
    """path(i, j) from a path matrix read one entry at a time (``p_at(a, c)`` returns
    P[a][c]), for matrices too large to copy whole: path(a, c) = [a, c] when
    P[a][c] = -1, else path(a, k) ++ path(k, c) with k = P[a][c].  Returns the
    vertex list ([i] when i == j), or None if it does not end within max_len vertices."""
    if i == j:
        return [i]
    out = [i]
    stack = [j]
    a = i
    while stack:
        c = stack[-1]
        k = int(p_at(a, c))
        if k < 0:
            out.append(c)
            stack.pop()
            a = c
            if len(out) > max_len:
                return None
        else:
            if len(stack) > max_len:
                return None
            stack.append(k)
    return out


def fw_backward(gD: np.ndarray, P: np.ndarray, D: np.ndarray) -> np.ndarray:
    """Reference gradient dL/dW = sum of gD[i, j] over the edges of path(i, j), in fp64."""
    n = gD.shape[0]
    g = np.ascontiguousarray(gD, dtype=np.float64)
    Pc = np.ascontiguousarray(P, dtype=np.int32)
    Dc = np.ascontiguousarray(D, dtype=np.float64)
    gW = np.empty((n, n), dtype=np.float64)
    if lib().oracle_fw_backward_f64(_ptr(g), _ptr(Pc), _ptr(Dc), n, _ptr(gW)):
        raise ValueError("path matrix does not encode a path for some reachable pair")
    return gW


def check_paths(W: np.ndarray, D: np.ndarray, P: np.ndarray, pairs=None, rtol: float = 0.0):
    """Validate P against (W, D): every reconstructed path uses existing edges and its
    weight (summed in fp64 along the path) equals D[i, j] (exactly when rtol = 0).

    ``pairs``: iterable of (i, j); default all pairs.  Returns the number of
    failures (0 = valid).  An unreachable pair (D = inf) must have P = -1.
    """
    n = W.shape[0]
    W64 = np.asarray(W, dtype=np.float64)
    if pairs is None:
        pairs = ((i, j) for i in range(n) for j in range(n))
    bad = 0
    for i, j in pairs:
        d = float(D[i, j])
        if i == j:
            bad += int(d != 0.0)
            continue
        if not np.isfinite(d):
            bad += int(P[i, j] != -1)
            continue
        path = reconstruct_path(P, i, j)
        if path is None or path[0] != i or path[-1] != j:
            bad += 1
            continue
        s = 0.0
        ok = True
        for a, b in zip(path[:-1], path[1:]):
            w = W64[a, b]
            if not np.isfinite(w) or a == b:
                ok = False
                break
            s += w
        if not ok:
            bad += 1
        elif rtol == 0.0:
            bad += int(s != d)
        else:
            bad += int(abs(s - d) > rtol * max(abs(d), 1.0))
    return bad


def enumerate_simple_paths(W: np.ndarray) -> np.ndarray:
    """Brute force: minimum over every simple directed path of its weight (tiny n only)."""
    n = W.shape[0]
    best = np.full((n, n), np.inf)
    for s in range(n):
        best[s, s] = 0.0
        stack = [(s, 0.0, 1 << s)]
        while stack:
            u, dist, seen = stack.pop()
            for v in range(n):
                if seen >> v & 1 or not np.isfinite(W[u, v]):
                    continue
                nd = dist + float(W[u, v])
                if nd < best[s, v]:
                    best[s, v] = nd
                stack.append((v, nd, seen | (1 << v)))
    return best
