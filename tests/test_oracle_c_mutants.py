"""Mistakes planted in the oracle itself are caught by its pins (CPU only).

Each case copies ``oracle/fw_oracle.c``, plants one plausible mistake (a
dropped term, a wrong index or sign, a transposed operand, a skipped phase, a
wrong tie rule, an off-by-one), builds the copy with the oracle's own compiler
flags and binds it in place of the real library.  The battery below — the
kinds of evidence ``test_oracle_pins.py`` relies on: brute force (Dijkstra,
Bellman-Ford, simple-path enumeration), closed forms, path validity, Johnson
reweighting, blocked = classic where the schedules coincide, finite
differences, the Bellman row equations — must reject every mutant and accept
the unmodified copy.  Nothing here touches a GPU or the CUDA library.
"""
import itertools
import os

import numpy as np
import pytest

import graphgen
import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "fw_oracle.c")

# name -> (text to replace, replacement, which occurrence in the source (0-based)).
# Occurrence 0 of the relaxation lines is Algorithm 1 (classic FW); occurrence 1
# is the blocked FW's block update (§2.2 "Blocked FW Algorithm").
MUTANTS = {
    # Algorithm 1
    "fw_tie_rule_le": ("if (cand < D[i * n + j]) {", "if (cand <= D[i * n + j]) {", 0),
    "fw_wrong_index_dkj": ("const REAL cand = dik + D[k * n + j];", "const REAL cand = dik + D[j * n + k];", 0),
    "fw_transposed_dik": ("const REAL dik = D[i * n + k];", "const REAL dik = D[k * n + i];", 0),
    "fw_dropped_term": ("const REAL cand = dik + D[k * n + j];", "const REAL cand = D[k * n + j];", 0),
    "fw_path_off_by_one": ("if (P) P[i * n + j] = (int32_t)k;", "if (P) P[i * n + j] = (int32_t)(k + 1);", 0),
    "fw_last_k_dropped": ("for (int64_t k = 0; k < k_end; ++k) {", "for (int64_t k = 0; k + 1 < k_end; ++k) {", 0),
    "fw_path_init_zero": ("for (int64_t e = 0; e < n * n; ++e) P[e] = -1;",
                          "for (int64_t e = 0; e < n * n; ++e) P[e] = 0;", 0),
    # blocked FW, four phases per round
    "bfw_tie_rule_le": ("if (cand < D[i * n + j]) {", "if (cand <= D[i * n + j]) {", 1),
    "bfw_transposed_dik": ("const REAL dik = D[i * n + k];", "const REAL dik = D[k * n + i];", 1),
    "bfw_phase1_skipped": ("UPD(D, P, n, k0, k1, k0, k1, k0, k1);", "(void)0;", 0),
    "bfw_phase2_on_columns": ("UPD(D, P, n, k0, k1, j0, j1, k0, k1);", "UPD(D, P, n, j0, j1, k0, k1, k0, k1);", 0),
    "bfw_phase3_on_rows": ("UPD(D, P, n, i0, i1, k0, k1, k0, k1);", "UPD(D, P, n, k0, k1, i0, i1, k0, k1);", 0),
    "bfw_phase4_first_k_dropped": ("UPD(D, P, n, i0, i1, j0, j1, k0, k1);",
                                   "UPD(D, P, n, i0, i1, j0, j1, k0 + 1, k1);", 0),
    "bfw_round_short_by_one": ("const int64_t k0 = r * TB, k1 = (k0 + TB < n) ? k0 + TB : n;",
                               "const int64_t k0 = r * TB, k1 = (k0 + TB < n) ? k0 + TB - 1 : n;", 0),
    # independent checks the pins lean on
    "dijkstra_single_prim": ("best + w < dist[v]) dist[v] = best + w;", "w < dist[v]) dist[v] = w;", 0),
    "dijkstra_rows_prim": ("best + w < dist[v]) dist[v] = best + w;", "w < dist[v]) dist[v] = w;", 1),
    "bellman_ford_one_pass": ("for (int64_t pass = 0; pass < n; ++pass) {",
                              "for (int64_t pass = 0; pass < 1; ++pass) {", 0),
    "bellman_ford_cycle_missed": ("if (pass == n - 1) return 1;", "if (pass == n - 1) return 0;", 0),
    "walk_appends_source": ("out[len] = j;", "out[len] = i;", 0),
    "backward_edge_transposed": ("gW[buf[t] * n + buf[t + 1]] += gD[i * n + j];",
                                 "gW[buf[t + 1] * n + buf[t]] += gD[i * n + j];", 0),
    "backward_pair_transposed": ("gW[buf[t] * n + buf[t + 1]] += gD[i * n + j];",
                                 "gW[buf[t] * n + buf[t + 1]] += gD[j * n + i];", 0),
    "bellman_rows_self_term": ("if (k == j) continue;", "if (0) continue;", 0),
    "bellman_rows_wrong_operand": ("(double)Drows[t * n + k]", "(double)Drows[t * n + j]", 0),
}


def _plant(src: str, old: str, new: str, nth: int) -> str:
    at = -1
    for _ in range(nth + 1):
        at = src.index(old, at + 1)  # ValueError if the source no longer has it
    return src[:at] + new + src[at + len(old):]


def _battery():
    """Names of the failed checks (empty = every pin holds).  A check that
    raises (a path that does not end, say) counts as failed."""
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)

    for section in _SECTIONS:
        try:
            section(check)
        except Exception as e:  # noqa: BLE001 - any error is a rejection
            failed.append(f"{section.__name__}: {type(e).__name__}")
    return failed


def _fw_and_brute_force(check):
    # FW (Algorithm 1) = Dijkstra from every source, both precisions; P valid
    n = 40
    W = graphgen.dense_graph(n, 0.25, 11, dtype=np.float64)
    ref_rows = oracle.dijkstra_rows(W, np.arange(n))
    for dt in (np.float64, np.float32):
        D, P = oracle.fw(W.astype(dt))
        check(f"fw_{np.dtype(dt).name}=dijkstra", np.array_equal(D.astype(np.float64), ref_rows))
        check(f"fw_{np.dtype(dt).name}_paths", oracle.check_paths(W, D, P) == 0)
    check("dijkstra_single=rows", all(np.array_equal(oracle.dijkstra(W, s), ref_rows[s]) for s in (0, 9, 31)))


def _closed_forms(check):
    # chain prefix sums (forward reachable only)
    w = [3.0, 1.0, 4.0, 1.0, 5.0, 9.0, 2.0, 6.0]
    Wc = graphgen.chain_graph(w)
    m = len(w) + 1
    exp = np.full((m, m), np.inf)
    for i in range(m):
        for j in range(i, m):
            exp[i, j] = sum(w[i:j])
    Dc, Pc = oracle.fw(Wc)
    check("chain_fw", np.array_equal(Dc, exp))
    check("chain_bfw", np.array_equal(oracle.bfw(Wc, 4)[0], exp))
    check("chain_bellman_ford", all(np.array_equal(oracle.bellman_ford(Wc, s)[0], exp[s]) for s in range(m)))


def _negative_weights(check):
    # simple-path enumeration with negative weights (no negative cycle: potentials)
    Wn = graphgen.dense_graph(6, 0.5, 3, dtype=np.float64)
    h = np.array([0.0, 4.0, -3.0, 7.0, 2.0, -5.0])
    fin = np.isfinite(Wn)
    Wn[fin] = (Wn + h[:, None] - h[None, :])[fin]
    Dn, Pn = oracle.fw(Wn)
    check("fw=simple_paths", np.array_equal(Dn, oracle.enumerate_simple_paths(Wn)))
    check("neg_paths", oracle.check_paths(Wn, Dn, Pn) == 0)

    # Johnson reweighting: Bellman-Ford on reweighted graph = FW, exactly
    Wj = graphgen.dense_graph(30, 0.2, 21, dtype=np.float64)
    hj = np.arange(30, dtype=np.float64) * 3.0 - 40.0
    fin = np.isfinite(Wj)
    Wr = np.where(fin, Wj + hj[:, None] - hj[None, :], np.inf)
    Dj, _ = oracle.fw(Wj)
    Dr, _ = oracle.fw(Wr)
    check("johnson", np.array_equal(np.where(np.isfinite(Dj), Dj + hj[:, None] - hj[None, :], np.inf), Dr))
    check("bellman_ford=fw", all(np.array_equal(oracle.bellman_ford(Wr, s)[0], Dr[s]) for s in (0, 7, 29)))

    # negative cycle is reported
    Wcyc = graphgen.chain_graph([1.0, 1.0, 1.0])
    Wcyc[3, 0] = -4.0
    check("negative_cycle", oracle.bellman_ford(Wcyc, 0)[1])


def _blocked(check):
    n = 40
    W = graphgen.dense_graph(n, 0.25, 11, dtype=np.float64)
    # blocked FW: distances = classic on integer weights for any block size;
    # D and P bit for bit where the schedules coincide (TB = 1, TB >= n)
    Dref, _ = oracle.fw(W)
    for TB in (1, 5, 16, 40, 64):
        Db, Pb = oracle.bfw(W, TB)
        check(f"bfw_TB{TB}=fw", np.array_equal(Db, Dref))
        check(f"bfw_TB{TB}_paths", oracle.check_paths(W, Db, Pb) == 0)
    Wreal = graphgen.dense_graph(24, 0.4, 5, weights="real", lo=0.5, hi=2.0, dtype=np.float64)
    Df, Pf = oracle.fw(Wreal)
    for TB in (1, 24, 32):
        Db, Pb = oracle.bfw(Wreal, TB)
        check(f"bfw_real_TB{TB}", np.array_equal(Db, Df) and np.array_equal(Pb, Pf))


def _gradient(check):
    # chain closed form and central finite differences
    w = [3.0, 1.0, 4.0, 1.0, 5.0, 9.0, 2.0, 6.0]
    Wc = graphgen.chain_graph(w)
    m = len(w) + 1
    Dc, Pc = oracle.fw(Wc)
    gD = graphgen.normal((m, m), 5, np.float64)
    expect = np.zeros((m, m))
    for e in range(m - 1):
        expect[e, e + 1] = sum(gD[i, j] for i in range(e + 1) for j in range(e + 1, m))
    check("grad_chain", np.allclose(oracle.fw_backward(gD, Pc, Dc), expect, rtol=1e-13, atol=1e-13))
    ng = 10
    gD2 = graphgen.normal((ng, ng), 2, np.float64)
    Wg = graphgen.dense_graph(ng, 0.5, 52, weights="real", lo=0.5, hi=2.0, dtype=np.float64)
    Dg, Pg = oracle.fw(Wg)
    finite = np.isfinite(Dg)
    gW = oracle.fw_backward(gD2, Pg, Dg)
    step = 1e-6
    fd_ok = True
    for u, v in itertools.product(range(ng), range(ng)):
        if u == v or not np.isfinite(Wg[u, v]):
            continue
        Wp, Wm = Wg.copy(), Wg.copy()
        Wp[u, v] += step
        Wm[u, v] -= step
        Dp, Pp = oracle.fw(Wp)
        Dm, Pm = oracle.fw(Wm)
        if not (np.array_equal(Pp, Pg) and np.array_equal(Pm, Pg)):
            continue
        fd = (np.sum(gD2[finite] * Dp[finite]) - np.sum(gD2[finite] * Dm[finite])) / (2 * step)
        fd_ok &= abs(fd - gW[u, v]) <= 1e-5 * max(1.0, abs(gW[u, v]))
    check("grad_fd", fd_ok)


def _bellman_rows(check):
    n = 40
    # Bellman row equations: exact rows accepted, rows with one entry moved by +-1 rejected
    Wb = graphgen.dense_graph(n, 0.3, 77, dtype=np.float32)
    srcs = np.array([0, 13])
    rows = oracle.dijkstra_rows(Wb, srcs).astype(np.float32)

    def equations_hold(R):
        best = np.full(R.shape, np.inf)
        for k0 in range(0, n, 16):
            oracle.minplus_rows_accumulate(R, Wb[k0:k0 + 16], k0, best)
        return all(R[t, s] == 0 and np.array_equal(np.delete(R[t], s).astype(np.float64), np.delete(best[t], s))
                   for t, s in enumerate(srcs))

    check("bellman_rows_accept", equations_hold(rows))
    for delta in (1.0, -1.0):
        bad = rows.copy()
        j = int(np.flatnonzero(np.isfinite(bad[0]) & (np.arange(n) != 0))[3])
        bad[0, j] += delta
        check(f"bellman_rows_reject_{delta:+.0f}", not equations_hold(bad))


_SECTIONS = (_fw_and_brute_force, _closed_forms, _negative_weights, _blocked, _gradient, _bellman_rows)


@pytest.fixture
def bind(tmp_path, monkeypatch):
    """Build a (possibly mutated) copy of the oracle and bind it for the battery."""
    def _bind(src_text, tag):
        c = tmp_path / f"{tag}.c"
        c.write_text(src_text)
        so = oracle.compile_library(str(c), str(tmp_path / f"lib{tag}.so"))
        monkeypatch.setattr(oracle, "_lib", oracle.load_library(so))
    return _bind


def test_unmodified_copy_passes_every_check(bind):
    bind(open(SRC).read(), "clean")
    assert _battery() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(bind, name):
    old, new, nth = MUTANTS[name]
    bind(_plant(open(SRC).read(), old, new, nth), name)
    assert _battery(), f"mutant {name} passed every check"
