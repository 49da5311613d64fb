"""The oracle's pins catch plausible mistakes (planted on the CPU, never on a GPU).

Each case plants one mistake into a plain numpy restatement of the oracle's
algorithm (Algorithm 1 / the four-phase blocked FW / the path-sum gradient)
and checks that at least one of the pin checks used by test_oracle_pins.py
rejects it, while the unplanted restatement passes them all.
"""
import numpy as np
import pytest

import graphgen
import oracle


def fw_np(W, mutant=None):
    """Algorithm 1 (strict '<'), with an optional planted mistake."""
    D = W.astype(np.float64).copy()
    n = D.shape[0]
    P = np.full((n, n), -1, dtype=np.int32)
    for k in range(n):
        if mutant == "skip_last_k" and k == n - 1:
            break
        if mutant == "transposed_operand":
            cand = D[k, :][:, None] + D[k, :][None, :]  # D[k][i] instead of D[i][k]
        elif mutant == "wrong_index":
            cand = D[:, k][:, None] + D[:, k][None, :]  # D[j][k] instead of D[k][j]
        else:
            cand = D[:, k][:, None] + D[k, :][None, :]
        better = cand <= D if mutant == "le_tie_rule" else cand < D
        if mutant == "p_off_by_one":
            P[better] = k + 1
        else:
            P[better] = k
        D = np.where(better, cand, D)
    return D, P


def bfw_np(W, TB, mutant=None):
    """Blocked FW (four phases per round), with an optional planted mistake."""
    D = W.astype(np.float64).copy()
    n = D.shape[0]
    P = np.full((n, n), -1, dtype=np.int32)

    def upd(i0, i1, j0, j1, k0, k1):
        for k in range(k0, k1):
            cand = D[i0:i1, k][:, None] + D[k, j0:j1][None, :]
            blk = D[i0:i1, j0:j1]
            better = cand < blk
            blk[better] = cand[better]
            P[i0:i1, j0:j1][better] = k

    R = (n + TB - 1) // TB
    for r in range(R):
        k0, k1 = r * TB, min(n, r * TB + TB)
        if mutant == "short_k_range":
            k1 = max(k0, k1 - 1)
        upd(k0, k1, k0, k1, k0, k1)
        for J in range(R):
            if J != r:
                upd(k0, k1, J * TB, min(n, J * TB + TB), k0, k1)
        if mutant != "drop_phase3":
            for I in range(R):
                if I != r:
                    upd(I * TB, min(n, I * TB + TB), k0, k1, k0, k1)
        for I in range(R):
            for J in range(R):
                if I != r and J != r:
                    upd(I * TB, min(n, I * TB + TB), J * TB, min(n, J * TB + TB), k0, k1)
    return D, P


def grad_np(gD, P, D, mutant=None):
    n = gD.shape[0]
    gW = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j or not np.isfinite(D[i, j]):
                continue
            path = oracle.reconstruct_path(P, i, j)
            for a, b in zip(path[:-1], path[1:]):
                if mutant == "transposed_edge":
                    gW[b, a] += gD[i, j]
                elif mutant == "drop_last_edge" and b == j:
                    continue
                else:
                    gW[a, b] += gD[i, j]
    return gW


def pins_pass(W, D, P):
    """The distance/path pins: Dijkstra from every source and path validity."""
    n = W.shape[0]
    ref = oracle.dijkstra_rows(W, np.arange(n))
    if not np.array_equal(D, ref):
        return False
    try:
        return oracle.check_paths(W, D, P, pairs=[(i, j) for i in range(n) for j in range(n)]) == 0
    except RecursionError:
        return False


W_INT = graphgen.dense_graph(40, 0.3, 123, dtype=np.float64)


def test_unplanted_restatements_pass_the_pins():
    assert pins_pass(W_INT, *fw_np(W_INT))
    assert pins_pass(W_INT, *bfw_np(W_INT, 8))


@pytest.mark.parametrize("mutant", ["transposed_operand", "wrong_index", "skip_last_k",
                                    "le_tie_rule", "p_off_by_one"])
def test_fw_mutants_are_caught(mutant):
    D, P = fw_np(W_INT, mutant)
    assert not pins_pass(W_INT, D, P)


@pytest.mark.parametrize("mutant", ["drop_phase3", "short_k_range"])
def test_blocked_mutants_are_caught(mutant):
    D, P = bfw_np(W_INT, 8, mutant)
    assert not pins_pass(W_INT, D, P)


@pytest.mark.parametrize("mutant", ["transposed_edge", "drop_last_edge"])
def test_gradient_mutants_are_caught(mutant):
    """The chain closed form (edge (m, m+1) lies on path(i, j) iff i <= m < j)."""
    w = [1.5, 0.7, 2.2, 0.9, 1.1]
    W = graphgen.chain_graph(w)
    D, P = oracle.fw(W)
    gD = graphgen.normal(W.shape, 5, np.float64)
    m = len(w) + 1
    expect = np.zeros((m, m))
    for e in range(m - 1):
        expect[e, e + 1] = sum(gD[i, j] for i in range(e + 1) for j in range(e + 1, m))
    np.testing.assert_allclose(grad_np(gD, P, D), expect, atol=1e-12)
    assert not np.allclose(grad_np(gD, P, D, mutant), expect, atol=1e-12)
