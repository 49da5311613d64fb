"""Pins for the CPU oracle: each checks it against something other than itself.

Every test here runs without a GPU.  The checks are chosen so that a plausible
slip in the oracle (a dropped candidate, a swapped index i/j or i/k, a wrong
sign, "<=" for "<", a missing phase of the blocked schedule, a wrong path
split) fails at least one of them:

* brute force: Dijkstra, Bellman-Ford, enumeration of all simple paths;
* closed forms: chain prefix sums, complete graph, grid (Manhattan), star,
  disconnected components, tree (gradient = subtree sums);
* invariants: zero diagonal, triangle inequality, D <= W, every path rebuilt
  from P is made of existing edges and weighs exactly D;
* Johnson reweighting (negative weights): D'[i][j] = D[i][j] + h(i) - h(j);
* blocked FW (§2.2 "Blocked FW Algorithm") equals classic FW (Algorithm 1)
  bit for bit, P included, at TB = 1 and TB >= n, where the two schedules
  coincide; equal distances for every TB on integer weights;
* finite differences for the gradient.
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle


def _rand_graph(n, p, seed, weights="int", dtype=np.float64, lo=1, hi=100):
    return graphgen.dense_graph(n, p, seed, weights=weights, lo=lo, hi=hi, dtype=dtype)


# --------------------------------------------------------------- brute force
@pytest.mark.parametrize("n,p,seed", [(1, 0.5, 0), (2, 0.5, 1), (5, 0.4, 2), (17, 0.2, 3),
                                      (33, 0.1, 4), (64, 0.3, 5), (64, 0.9, 6)])
@pytest.mark.parametrize("weights", ["int", "real"])
def test_fw_equals_dijkstra(n, p, seed, weights):
    W = _rand_graph(n, p, seed, weights, lo=1 if weights == "int" else 0.5,
                    hi=100 if weights == "int" else 2.0)
    D, P = oracle.fw(W)
    ref = oracle.dijkstra_rows(W, np.arange(n))
    if weights == "int":
        np.testing.assert_array_equal(D, ref)
    else:
        fin = np.isfinite(ref)
        np.testing.assert_array_equal(np.isfinite(D), fin)
        np.testing.assert_allclose(D[fin], ref[fin], rtol=1e-12)
    assert oracle.check_paths(W, D, P, rtol=0.0 if weights == "int" else 1e-12) == 0


def test_dijkstra_single_and_rows_agree():
    W = _rand_graph(40, 0.2, 11)
    rows = oracle.dijkstra_rows(W.astype(np.float32), [0, 7, 39])
    for r, s in enumerate([0, 7, 39]):
        np.testing.assert_array_equal(rows[r], oracle.dijkstra(W, s))


@pytest.mark.parametrize("seed", range(6))
def test_fw_equals_simple_path_enumeration(seed):
    """n <= 7 with negative weights (no negative cycle): minimum over all simple paths."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 8))
    W = _rand_graph(n, 0.5, 200 + seed)
    h = rng.integers(-20, 20, size=n).astype(np.float64)
    Wp = W + h[:, None] - h[None, :]
    np.fill_diagonal(Wp, 0)
    D, P = oracle.fw(Wp)
    np.testing.assert_array_equal(D, oracle.enumerate_simple_paths(Wp))
    assert oracle.check_paths(Wp, D, P) == 0


@pytest.mark.parametrize("n,seed", [(24, 1), (50, 2)])
def test_bellman_ford_and_johnson_reweighting(n, seed):
    """Edge potentials h give negative weights but no negative cycle; distances
    shift by exactly h(i) - h(j) (integer arithmetic, so exact)."""
    W = _rand_graph(n, 0.3, seed)
    rng = np.random.default_rng(seed)
    h = rng.integers(-60, 60, size=n).astype(np.float64)
    Wp = np.where(np.isfinite(W), W + h[:, None] - h[None, :], np.inf)
    np.fill_diagonal(Wp, 0)
    assert (Wp[np.isfinite(Wp)] < 0).any()
    D, _ = oracle.fw(W)
    Dp, Pp = oracle.fw(Wp)
    expect = np.where(np.isfinite(D), D + h[:, None] - h[None, :], np.inf)
    np.testing.assert_array_equal(Dp, expect)
    for s in (0, n // 2, n - 1):
        bf, neg = oracle.bellman_ford(Wp, s)
        assert not neg
        np.testing.assert_array_equal(Dp[s], bf)
    assert oracle.check_paths(Wp, Dp, Pp) == 0


def test_bellman_ford_detects_negative_cycle():
    W = graphgen.chain_graph([1.0, 1.0, 1.0])
    W[3, 0] = -5.0
    _, neg = oracle.bellman_ford(W, 0)
    assert neg


# --------------------------------------------------------------- closed forms
def test_chain_prefix_sums():
    w = [3.0, 1.0, 4.0, 1.0, 5.0, 9.0, 2.0, 6.0]
    W = graphgen.chain_graph(w)
    D, P = oracle.fw(W)
    m = len(w) + 1
    pre = np.concatenate([[0.0], np.cumsum(w)])
    for i in range(m):
        for j in range(m):
            assert D[i, j] == (pre[j] - pre[i] if j >= i else np.inf)
    # the path from 0 to the end visits every vertex in order
    assert oracle.reconstruct_path(P, 0, m - 1) == list(range(m))


def test_complete_graph_constant_weight():
    D, P = oracle.fw(graphgen.complete_graph(9, 2.5))
    expect = np.full((9, 9), 2.5)
    np.fill_diagonal(expect, 0)
    np.testing.assert_array_equal(D, expect)
    assert (P == -1).all()  # no intermediate vertex ever improves a direct edge


def test_grid_manhattan():
    rows, cols = 5, 7
    D, P = oracle.fw(graphgen.grid_graph(rows, cols))
    for a in range(rows * cols):
        for b in range(rows * cols):
            ra, ca = divmod(a, cols)
            rb, cb = divmod(b, cols)
            assert D[a, b] == abs(ra - rb) + abs(ca - cb)
    assert oracle.check_paths(graphgen.grid_graph(rows, cols), D, P) == 0


def test_star_two_spokes():
    sin = [2.0, 7.0, 1.0, 8.0]
    sout = [3.0, 5.0, 4.0, 6.0]
    D, P = oracle.fw(graphgen.star_graph(sin, sout))
    m = len(sin)
    for a in range(1, m + 1):
        assert D[a, 0] == sin[a - 1] and D[0, a] == sout[a - 1]
        for b in range(1, m + 1):
            if a != b:
                assert D[a, b] == sin[a - 1] + sout[b - 1]
                assert P[a, b] == 0


def test_disconnected_components_stay_infinite():
    A = _rand_graph(10, 0.5, 1)
    B = _rand_graph(7, 0.5, 2)
    W = np.full((17, 17), np.inf)
    W[:10, :10] = A
    W[10:, 10:] = B
    D, P = oracle.fw(W)
    assert np.isinf(D[:10, 10:]).all() and np.isinf(D[10:, :10]).all()
    assert (P[:10, 10:] == -1).all() and (P[10:, :10] == -1).all()
    np.testing.assert_array_equal(D[:10, :10], oracle.fw(A)[0])


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_invariants_random(dtype):
    W = _rand_graph(96, 0.3, 9, dtype=dtype)
    D, P = oracle.fw(W)
    assert (np.diag(D) == 0).all()
    assert (D <= W).all()
    # triangle inequality for every (i, k, j)
    for k in range(96):
        assert (D <= D[:, k:k + 1] + D[k:k + 1, :]).all()
    assert oracle.check_paths(W, D, P) == 0
    # P = -1 only for the direct edge, the diagonal or an unreachable pair
    m = P == -1
    assert ((D == W) | np.isinf(D))[m].all()


def test_f32_equals_f64_on_integer_weights():
    W = _rand_graph(128, 0.3, 21)
    D64, _ = oracle.fw(W)
    D32, _ = oracle.fw(W.astype(np.float32))
    np.testing.assert_array_equal(D32.astype(np.float64), D64)


def test_partial_run_is_prefix():
    W = _rand_graph(50, 0.3, 22)
    Dk, Pk = oracle.fw(W, k_end=7)
    D = W.copy()
    for k in range(7):  # the definition of the first 7 outer iterations, vectorised
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    np.testing.assert_array_equal(Dk, D)


# --------------------------------------------------------------- blocked FW
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("TB", [1, 70, 128])
def test_bfw_equals_fw_where_schedules_coincide(dtype, TB):
    """TB = 1: phase 4 of round k is iteration k of Algorithm 1; TB >= n: one
    phase-1 block is Algorithm 1.  Bit-exact on real weights, P included."""
    W = _rand_graph(70, 0.3, 31, weights="real", lo=0.5, hi=2.0, dtype=dtype)
    D, P = oracle.fw(W)
    Db, Pb = oracle.bfw(W, TB)
    np.testing.assert_array_equal(Db, D)
    np.testing.assert_array_equal(Pb, P)


@pytest.mark.parametrize("n,TB", [(64, 8), (70, 16), (100, 32), (33, 5), (129, 64)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_bfw_distances_equal_fw_integer(n, TB, dtype):
    W = _rand_graph(n, 0.3, n + TB, dtype=dtype)
    D, _ = oracle.fw(W)
    Db, Pb = oracle.bfw(W, TB)
    np.testing.assert_array_equal(Db, D)
    assert oracle.check_paths(W, Db, Pb) == 0


def test_bfw_real_weights_close_to_fp64():
    W = _rand_graph(100, 0.4, 41, weights="real", lo=0.5, hi=2.0, dtype=np.float32)
    D64, _ = oracle.fw(W.astype(np.float64))
    Db, Pb = oracle.bfw(W, 16)
    fin = np.isfinite(D64)
    np.testing.assert_array_equal(np.isfinite(Db), fin)
    np.testing.assert_allclose(Db[fin], D64[fin], rtol=1e-5)
    assert oracle.check_paths(W, Db, Pb, rtol=1e-5) == 0


@pytest.mark.parametrize("TB", [None, 16, 128])
def test_fp32_error_within_the_rounding_bound_of_its_paths(TB):
    """FP32 against FP64 on the same (float) weights, entry by entry.  Rounding
    is monotone and a positive sum of L terms rounded L - 1 times lies within
    (1 -+ u)^(L-1) of the exact sum (u = 2^-24).  The FP32 run evaluates
    (a composition of rounded sub-results no larger than) the FP64 optimum's
    path p*, so D32 <= D64 (1 + u)^(|p*| - 1); and D32 is the rounded sum of the
    path q its own P encodes, whose exact sum is >= D64, so
    D32 >= D64 (1 - u)^(|q| - 1).  Much tighter than the 1e-5 tolerance: a
    double rounding, a lost term or a wrong operand would break it."""
    n = 120
    W = _rand_graph(n, 0.4, 61, weights="real", lo=0.5, hi=2.0, dtype=np.float32)
    D32, P32 = oracle.fw(W) if TB is None else oracle.bfw(W, TB)
    D64, P64 = oracle.fw(W.astype(np.float64))
    u, eps = 2.0 ** -24, n * 2.0 ** -52
    checked = 0
    for i in range(n):
        for j in range(n):
            d64 = D64[i, j]
            if i == j or not np.isfinite(d64):
                assert D32[i, j] == d64
                continue
            lq = len(oracle.reconstruct_path(P32, i, j)) - 1
            lp = len(oracle.reconstruct_path(P64, i, j)) - 1
            d32 = float(D32[i, j])
            assert d64 * (1 - u) ** (lq - 1) * (1 - eps) <= d32 <= d64 * (1 + u) ** (lp - 1) * (1 + eps), \
                (i, j, d32, d64, lq, lp)
            checked += 1
    assert checked > n * n // 2
    assert np.any(D32.astype(np.float64) != D64)  # the bound is exercised, not trivially equal


def test_bfw_rejects_bad_block():
    with pytest.raises(ValueError):
        oracle.bfw(np.zeros((3, 3)), 0)


# --------------------------------------------------------------- gradient
def test_gradient_chain_closed_form():
    """Edge (m, m+1) of a chain lies on path(i, j) iff i <= m < j."""
    w = [1.5, 0.7, 2.2, 0.9, 1.1, 1.9]
    W = graphgen.chain_graph(w)
    D, P = oracle.fw(W)
    gD = graphgen.normal(W.shape, 5, np.float64)
    gW = oracle.fw_backward(gD, P, D)
    m = len(w) + 1
    expect = np.zeros((m, m))
    for e in range(m - 1):
        expect[e, e + 1] = sum(gD[i, j] for i in range(e + 1) for j in range(e + 1, m))
    np.testing.assert_allclose(gW, expect, rtol=1e-13, atol=1e-13)


def test_gradient_tree_subtree_sums():
    """Out-tree rooted at 0: edge parent(v) -> v is on path(i, j) iff v is an
    ancestor-or-self of j and i is an ancestor of parent(v)... i.e. i is a
    proper ancestor of v and j lies in the subtree of v."""
    n = 30
    W, parent = graphgen.random_tree_graph(n, 3)
    D, P = oracle.fw(W)
    gD = graphgen.normal((n, n), 6, np.float64)

    def ancestors(v):  # proper ancestors of v
        out = []
        while parent[v] >= 0:
            v = parent[v]
            out.append(v)
        return out

    anc = [set(ancestors(v)) for v in range(n)]
    expect = np.zeros((n, n))
    for v in range(1, n):
        sub = [j for j in range(n) if j == v or v in anc[j]]
        expect[parent[v], v] = sum(gD[i, j] for i in anc[v] for j in sub)
    np.testing.assert_allclose(oracle.fw_backward(gD, P, D), expect, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_central_finite_differences(seed):
    n = 14
    W = _rand_graph(n, 0.4, 50 + seed, weights="real", lo=0.5, hi=2.0)
    gD = graphgen.normal((n, n), seed, np.float64)
    D, P = oracle.fw(W)
    fin = np.isfinite(D)
    gW = oracle.fw_backward(gD, P, D)
    h = 1e-6
    checked = 0
    for u, v in itertools.product(range(n), range(n)):
        if u == v or not np.isfinite(W[u, v]):
            continue
        Wp, Wm = W.copy(), W.copy()
        Wp[u, v] += h
        Wm[u, v] -= h
        Dp, Pp = oracle.fw(Wp)
        Dm, Pm = oracle.fw(Wm)
        if not (np.array_equal(Pp, P) and np.array_equal(Pm, P)):
            continue  # a path switches inside [w-h, w+h]: D is not differentiable there
        fd = (np.sum(gD[fin] * Dp[fin]) - np.sum(gD[fin] * Dm[fin])) / (2 * h)
        assert abs(fd - gW[u, v]) <= 1e-5 * max(1.0, abs(gW[u, v])), (u, v, fd, gW[u, v])
        checked += 1
    assert checked > 20
    # unused edges, non-edges and the diagonal carry no gradient
    assert (gW[~np.isfinite(W)] == 0).all() and (np.diag(gW) == 0).all()


# --------------------------------------------------------------- input generator
def test_generator_numpy_equals_torch():
    torch = pytest.importorskip("torch")
    for weights in ("int", "real"):
        a = graphgen.dense_graph(77, 0.3, 5, weights=weights, lo=1 if weights == "int" else 0.5,
                                 hi=100 if weights == "int" else 2.0)
        b = graphgen.dense_graph_torch(77, 0.3, 5, weights=weights, lo=1 if weights == "int" else 0.5,
                                       hi=100 if weights == "int" else 2.0, rows_per_chunk=13)
        np.testing.assert_array_equal(a, b.numpy())


def test_generator_shape_of_workload():
    W = graphgen.dense_graph(512, 0.3, 1)
    off = ~np.eye(512, dtype=bool)
    dens = np.isfinite(W[off]).mean()
    assert abs(dens - 0.3) < 0.01
    w = W[off & np.isfinite(W)]
    assert w.min() == 1 and w.max() == 100 and (w == np.round(w)).all()
    assert (np.diag(W) == 0).all()
    sizes = graphgen.batch_sizes(4096, 16, 512, 1)
    assert sizes.min() >= 16 and sizes.max() <= 512 and abs(sizes.mean() - 264) < 10


def test_batched_generator_numpy_equals_torch():
    pytest.importorskip("torch")
    sizes = [3, 17, 1, 40]
    off = np.array([0, 12, 304, 308], dtype=np.int64)
    total = 308 + 1600
    packed = graphgen.batched_graphs_torch(sizes, 0.3, 9, off, total).numpy()
    for g, m in enumerate(graphgen.batched_graphs(sizes, 0.3, 9)):
        np.testing.assert_array_equal(packed[off[g]:off[g] + m.size], m.reshape(-1))


def test_bellman_row_check_accepts_exact_rows_and_rejects_planted_errors():
    """The Bellman-equation row check (used at sizes no whole-matrix oracle fits)
    accepts the rows of Dijkstra's distances and rejects a row with one entry
    lowered or raised by 1."""
    n = 257
    W = graphgen.dense_graph(n, 0.3, 77)
    srcs = [0, 100, 256]
    rows = oracle.dijkstra_rows(W, srcs).astype(np.float32)

    def check(R):
        best = np.full((len(srcs), n), np.inf)
        for k0 in range(0, n, 50):
            oracle.minplus_rows_accumulate(R, W[k0:k0 + 50], k0, best)
        return all(R[t, i] == 0 and np.array_equal(R[t][np.arange(n) != i], best[t][np.arange(n) != i])
                   for t, i in enumerate(srcs))

    assert check(rows)
    for delta in (-1.0, 1.0):
        bad = rows.copy()
        bad[1, 7] += delta
        assert not check(bad)


def test_path_lookup_walk_matches_whole_matrix_walk():
    W = graphgen.dense_graph(120, 0.2, 3)
    D, P = oracle.fw(W)
    for i, j in [(0, 5), (7, 119), (50, 50), (3, 99)]:
        assert oracle.reconstruct_path_lookup(lambda a, c: P[a, c], i, j, 121) == oracle.reconstruct_path(P, i, j)
