"""GPU parity: the CUDA blocked FW (through the C ABI) against the CPU oracle.

Inputs come from graphgen (seeded); expected values only from ``oracle``.
Bars (the readings behind them are in the oracle's header):
  * integer weights: D bit-exact with classic FW (every sum is exact);
  * real weights: D and P bit-exact with the oracle's blocked FW at the
    library's block size in the same precision (same candidate sums, same
    ascending-k strict-"<" tie rule), and within 1e-5 (FP32) / 1e-12 (FP64)
    relative of an FP64 classic FW;
  * P: every path rebuilt from it is made of existing edges and weighs D.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_2105_07298_gb300 as apsp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _run(W, dtype, with_path=True, ld=None):
    n = W.shape[0]
    ld = ld or n
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    buf = torch.full((max(n, 1), max(ld, 1)), float("nan"), dtype=tdt, device=DEV)
    D = buf[:n, :n] if n else buf[:0, :0]
    D.copy_(torch.from_numpy(np.ascontiguousarray(W, dtype=dtype)))
    P = None
    if with_path:
        pbuf = torch.full((max(n, 1), max(ld, 1)), 12345, dtype=torch.int32, device=DEV)
        P = pbuf[:n, :n]
    apsp.apsp_fw(D, P)
    torch.cuda.synchronize()
    pad_ok = bool(torch.isnan(buf[:n, n:ld]).all()) if ld > n else True
    return D.cpu().numpy(), (P.cpu().numpy() if P is not None else None), pad_ok


def _sample_pairs(n, count, seed):
    rng = np.random.default_rng(seed)
    return list(zip(rng.integers(0, n, count).tolist(), rng.integers(0, n, count).tolist()))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 64, 65, 127, 128, 129, 200, 255, 257, 300, 384, 385, 513])
def test_integer_weights_bit_exact(n, dtype):
    W = graphgen.dense_graph(n, 0.3, 1000 + n, dtype=dtype)
    D, P, _ = _run(W, dtype)
    Dref, _ = oracle.fw(W.astype(np.float64))
    np.testing.assert_array_equal(D.astype(np.float64), Dref)
    assert oracle.check_paths(W, D, P) == 0


@pytest.mark.parametrize("n", [70, 200, 333, 513])
def test_real_weights_f32_match_blocked_oracle_bitwise(n):
    """FP32 follows the paper's four phases exactly: same sums, same order of k."""
    W = graphgen.dense_graph(n, 0.4, 77 + n, weights="real", lo=0.5, hi=2.0, dtype=np.float32)
    D, P, _ = _run(W, np.float32)
    Db, Pb = oracle.bfw(W, apsp.block_size(torch.float32))
    np.testing.assert_array_equal(D, Db)
    np.testing.assert_array_equal(P, Pb)
    D64, _ = oracle.fw(W.astype(np.float64))
    fin = np.isfinite(D64)
    np.testing.assert_array_equal(np.isfinite(D), fin)
    rel = np.abs(D[fin].astype(np.float64) - D64[fin]) / np.maximum(np.abs(D64[fin]), 1e-300)
    assert rel.max() <= 1e-5, rel.max()
    assert oracle.check_paths(W, D, P, rtol=1e-5) == 0


@pytest.mark.parametrize("n,p", [(70, 0.4), (200, 0.4), (333, 0.4), (300, 0.05), (513, 0.4)])
def test_real_weights_f64_match_blocked_oracle_bitwise(n, p):
    """FP64 follows the paper's four phases in its k order with IEEE FP64 sums:
    D and P bit-exact with the oracle's blocked FW at the library's block size,
    and within 1e-12 relative of the classic FP64 FW."""
    W = graphgen.dense_graph(n, p, 177 + n, weights="real", lo=0.5, hi=2.0, dtype=np.float64)
    D, P, _ = _run(W, np.float64)
    Db, Pb = oracle.bfw(W, apsp.block_size(torch.float64))
    np.testing.assert_array_equal(D, Db)
    np.testing.assert_array_equal(P, Pb)
    D64, _ = oracle.fw(W)
    fin = np.isfinite(D64)
    np.testing.assert_array_equal(np.isfinite(D), fin)
    rel = np.abs(D[fin] - D64[fin]) / np.maximum(np.abs(D64[fin]), 1e-300)
    assert rel.max() <= 1e-12, rel.max()
    assert oracle.check_paths(W, D, P, rtol=1e-12) == 0
    assert apsp.device_status() == apsp.APSP_OK


def test_f64_values_beyond_float_range_and_fractions():
    """FP64 inputs FP32 cannot hold exactly (2^-30 fractions, magnitudes near 1e300,
    tiny values): the interval filter must still give exact FP64 results, bit
    for bit those of the sequential blocked FW."""
    rng = np.random.default_rng(8)
    n = 260
    W = graphgen.dense_graph(n, 0.3, 99, dtype=np.float64)
    fin = np.isfinite(W) & ~np.eye(n, dtype=bool)
    W[fin] = W[fin] + rng.integers(0, 4, fin.sum()) * 2.0 ** -30
    D, P, _ = _run(W, np.float64)
    np.testing.assert_array_equal(D, oracle.fw(W)[0])  # dyadic sums: exact in FP64
    for scale in (1e300, 1e-300):
        Ws = np.where(np.isfinite(W), W * scale, np.inf)
        np.fill_diagonal(Ws, 0)
        D, P, _ = _run(Ws, np.float64)
        Dref = oracle.fw(Ws)[0]
        ok = np.isfinite(Dref)
        np.testing.assert_array_equal(np.isfinite(D), ok)
        np.testing.assert_allclose(D[ok], Dref[ok], rtol=1e-12)
        Db, Pb = oracle.bfw(Ws, apsp.block_size(torch.float64))
        np.testing.assert_array_equal(D, Db)
        np.testing.assert_array_equal(P, Pb)


def test_config_small_n1024_full():
    """n = 1024, edge probability 0.3, integer weights [1, 100], FP32 + int32 path."""
    W = graphgen.dense_graph(1024, 0.3, 1)
    D, P, _ = _run(W, np.float32)
    Dref, Pref = oracle.fw(W)
    np.testing.assert_array_equal(D, Dref)
    assert oracle.check_paths(W, D, P, pairs=_sample_pairs(1024, 4000, 3)) == 0
    # blocked oracle at the library's block size: identical P as well
    Db, Pb = oracle.bfw(W, apsp.block_size(torch.float32))
    np.testing.assert_array_equal(P, Pb)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_n2048_full_bit_exact(dtype):
    W = graphgen.dense_graph(2048, 0.5, 2048, dtype=dtype)
    D, P, _ = _run(W, dtype)
    Dref, _ = oracle.fw(W.astype(np.float64))
    np.testing.assert_array_equal(D.astype(np.float64), Dref)
    assert oracle.check_paths(W, D, P, pairs=_sample_pairs(2048, 3000, 4)) == 0


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_leading_dimension_and_padding(dtype):
    """ld > n (aligned and unaligned): padding columns are never touched."""
    for n, ld in ((130, 136), (130, 131), (257, 259)):
        W = graphgen.dense_graph(n, 0.3, n * 7 + ld, dtype=dtype)
        D, P, pad_ok = _run(W, dtype, ld=ld)
        assert pad_ok
        Dref, _ = oracle.fw(W.astype(np.float64))
        np.testing.assert_array_equal(D.astype(np.float64), Dref)
        assert oracle.check_paths(W, D, P) == 0


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_without_path_matrix(dtype):
    W = graphgen.dense_graph(300, 0.3, 9, dtype=dtype)
    D, _, _ = _run(W, dtype, with_path=False)
    np.testing.assert_array_equal(D.astype(np.float64), oracle.fw(W.astype(np.float64))[0])


def test_host_buffer_entry_matches_device_path():
    """apsp_fw_f32_host (host buffers in and out, one C-ABI call) gives the
    device entry point's D and P bit for bit, from page-locked and pageable
    buffers, with and without caller work buffers, with and without P, in
    place; integer weights also against the oracle."""
    n = 700
    W = graphgen.dense_graph(n, 0.3, 77, weights="real", lo=0.5, hi=2.0)
    Dd = torch.from_numpy(W.copy()).to(DEV)
    Pd = torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.apsp_fw_f32(Dd, Pd)
    torch.cuda.synchronize()
    Dref, Pref = Dd.cpu(), Pd.cpu()
    for pinned in (True, False):
        Wh = torch.from_numpy(W.copy())
        if pinned:
            Wh = Wh.pin_memory()
        for work in (False, True):
            wd = torch.empty(n * n, device=DEV) if work else None
            wp = torch.empty(n * n, dtype=torch.int32, device=DEV) if work else None
            D, P = apsp.apsp_fw_f32_host(Wh, work_dist=wd, work_path=wp)
            assert torch.equal(D, Dref) and torch.equal(P, Pref)
            assert torch.equal(Wh, torch.from_numpy(W))  # the input is read only
    D, P = apsp.apsp_fw_f32_host(torch.from_numpy(W.copy()), with_path=False)
    assert P is None and torch.equal(D, Dref)
    Wi = torch.from_numpy(W.copy())
    apsp.apsp_fw_f32_host(Wi, dist=Wi, with_path=False)
    assert torch.equal(Wi, Dref)
    Wint = graphgen.dense_graph(300, 0.3, 78)
    D, P = apsp.apsp_fw_f32_host(torch.from_numpy(Wint.copy()))
    np.testing.assert_array_equal(D.numpy(), oracle.fw(Wint)[0])
    assert oracle.check_paths(Wint, D.numpy(), P.numpy()) == 0
    with pytest.raises(TypeError):
        apsp.apsp_fw_f32_host(Dd)  # device tensors go to apsp_fw_f32


def test_structured_graphs():
    # chain across several blocks, grid, disconnected halves, negative weights via potentials
    W = graphgen.chain_graph(np.arange(1, 300, dtype=np.float64) % 7 + 1).astype(np.float32)
    D, P, _ = _run(W, np.float32)
    np.testing.assert_array_equal(D, oracle.fw(W)[0])
    assert oracle.check_paths(W, D, P, pairs=_sample_pairs(300, 500, 1)) == 0
    G = graphgen.grid_graph(13, 17).astype(np.float32)
    D, P, _ = _run(G, np.float32)
    np.testing.assert_array_equal(D, oracle.fw(G)[0])
    A = graphgen.dense_graph(150, 0.2, 5)
    Wd = np.full((300, 300), np.inf, dtype=np.float32)
    Wd[:150, :150] = A
    Wd[150:, 150:] = A
    D, P, _ = _run(Wd, np.float32)
    assert np.isinf(D[:150, 150:]).all() and (P[:150, 150:] == -1).all()
    h = np.random.default_rng(3).integers(-40, 40, 260).astype(np.float64)
    W0 = graphgen.dense_graph(260, 0.3, 6, dtype=np.float64)
    Wn = np.where(np.isfinite(W0), W0 + h[:, None] - h[None, :], np.inf)
    np.fill_diagonal(Wn, 0)
    for dt in (np.float32, np.float64):
        D, P, _ = _run(Wn.astype(dt), dt)
        np.testing.assert_array_equal(D.astype(np.float64), oracle.fw(Wn)[0])


def test_argument_errors():
    lib = apsp.load()
    x = torch.zeros((4, 4), device=DEV)
    assert lib.apsp_fw_f32(None, 4, 4, None, None) == apsp.APSP_EINVAL
    assert lib.apsp_fw_f32(x.data_ptr(), 4, 3, None, None) == apsp.APSP_EINVAL
    assert lib.apsp_fw_f32(x.data_ptr(), -1, 4, None, None) == apsp.APSP_EINVAL
    assert lib.apsp_fw_f32(x.data_ptr(), (1 << 18) + 1, (1 << 18) + 1, None, None) == apsp.APSP_EINVAL
    assert lib.apsp_fw_f32(None, 0, 0, None, None) == apsp.APSP_OK  # empty graph: no-op
    with pytest.raises(ValueError):
        apsp.apsp_fw_f32(x.t())  # columns not contiguous
    with pytest.raises(TypeError):
        apsp.apsp_fw_f32(x.double())


def _dijkstra_check(D_dev, W_host, srcs):
    ref = oracle.dijkstra_rows(W_host, srcs)
    got = D_dev[torch.as_tensor(srcs, device=D_dev.device)].double().cpu().numpy()
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("n,dtype", [(16384, torch.float32), (16384, torch.float64),
                                     (32768, torch.float32), (32768, torch.float64),
                                     (65536, torch.float32)])
def test_full_size_sampled_rows(n, dtype):
    """Full-size blocked FW (edge probability 0.5, integer weights): sampled
    rows against Dijkstra (exact; 64 rows at n = 16384, 8 at the larger sizes)
    and 40 sampled paths per row against the weights."""
    W = graphgen.dense_graph_torch(n, 0.5, 20210517, dtype=dtype, device=DEV)
    W_host = W.cpu().numpy()
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.apsp_fw(W, P)
    torch.cuda.synchronize()
    srcs = np.random.default_rng(n).integers(0, n, 64 if n == 16384 else 8)
    _dijkstra_check(W, W_host, srcs)
    # path validation on sampled pairs, reading rows of P and D on demand
    rows = sorted(set(srcs.tolist()))
    pairs = [(int(i), int(j)) for i in rows for j in np.random.default_rng(int(i)).integers(0, n, 40)]
    Ph = P.cpu().numpy()
    Dh = W[torch.as_tensor(rows, device=DEV)].double().cpu().numpy()
    dmap = {r: Dh[t] for t, r in enumerate(rows)}
    bad = 0
    for i, j in pairs:
        path = oracle.reconstruct_path(Ph, i, j)
        if i == j:
            continue
        s = 0.0
        for a, b in zip(path[:-1], path[1:]):
            s += float(W_host[a, b])
        bad += int(s != dmap[i][j])
    assert bad == 0


def test_phase_timing_hook_and_device_status():
    """The timing hook brackets every launch (path init, R diagonal and R panel
    launches, and phase 4 as two launches per round but the last, when the next
    round's phases 1-3 overlap it) and no bounded wait runs out on a normal solve."""
    n = 1000
    W = torch.from_numpy(graphgen.dense_graph(n, 0.3, 5)).to(DEV)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.profile_enable(True)
    apsp.apsp_fw_f32(W, P)
    prof = apsp.profile_collect()
    apsp.profile_enable(False)
    R = (n + 127) // 128
    assert prof["path_init"][1] == 1
    k3 = 2 * R - 1 if R > 2 else R
    assert prof["phase1_diag"][1] == R and prof["phase2_panels"][1] == R and prof["phase3_minplus"][1] == k3
    assert all(ms >= 0 for ms, _ in prof.values())
    recs = apsp.profile_records()
    assert [p for p, _ in recs].count("phase3_minplus") == k3 and recs[0][0] == "path_init"
    for ph, (ms, cnt) in prof.items():
        assert sum(t for p, t in recs if p == ph) == pytest.approx(ms, rel=1e-4, abs=1e-4)
    assert apsp.device_status() == apsp.APSP_OK


def test_measured_pair_rate_is_plausible():
    """The inner-loop instruction pair sustains a large part of the 128
    relaxations per clock per SM of the unit-count model (FP32), and the FP64
    path's lower-bound pair (add.rm instead of add.rn) the same rate; bad
    arguments are rejected."""
    r32 = apsp.measure_peak(4)
    r64 = apsp.measure_peak(8)
    assert 64.0 < r32 <= 132.0, r32
    assert 0.85 * r32 < r64 < 1.15 * r32, (r32, r64)
    with pytest.raises(apsp.ApspError):
        apsp.measure_peak(2)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_solve_captured_in_cuda_graph(dtype):
    """A solve captured into a CUDA graph (all phases on the capturing stream)
    replays to the same D and P as a direct call."""
    n = 700
    W = torch.from_numpy(graphgen.dense_graph(n, 0.4, 77, dtype=dtype)).to(DEV)
    D0, P0 = W.clone(), torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.apsp_fw(D0, P0)
    D, P = W.clone(), torch.empty((n, n), dtype=torch.int32, device=DEV)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        apsp.apsp_fw(D, P)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        D.copy_(W)
        apsp.apsp_fw(D, P)
    P.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(D, D0) and torch.equal(P, P0)
    assert apsp.device_status() == apsp.APSP_OK


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_negative_cycle_check(dtype):
    """A graph with a negative cycle leaves D[i][i] < 0 on the cycle's vertices;
    the check reports it, and reports nothing for the same graph without it."""
    n = 300
    W = graphgen.dense_graph(n, 0.3, 31, dtype=dtype)
    D, _, _ = _run(W, dtype)
    Dt = torch.from_numpy(D).to(DEV)
    assert not apsp.check_negative_cycle(Dt)
    Wn = W.copy()
    Wn[5, 250] = -1000.0  # cycle 5 -> 250 -> ... -> 5 of weight below zero
    D, _, _ = _run(Wn, dtype)
    assert (np.diag(D)[[5, 250]] < 0).all()
    assert apsp.check_negative_cycle(torch.from_numpy(D).to(DEV))
    lib = apsp.load()
    assert lib.apsp_check_negative_cycle(None, 4, 0, 0, None) == apsp.APSP_OK
    assert lib.apsp_check_negative_cycle(None, 4, 3, 3, None) == apsp.APSP_EINVAL
    assert lib.apsp_check_negative_cycle(Dt.data_ptr(), 2, n, n, None) == apsp.APSP_EINVAL


def test_bounded_wait_timeout_is_reported_and_context_survives():
    """The bounded mbarrier wait of the bulk-copy kernels, on a barrier nothing
    completes, gives up, records APSP_ETIMEOUT and returns: the status reads
    back once (then clears), and the next solve is correct."""
    assert apsp.device_status() == apsp.APSP_OK
    apsp.wait_timeout_selftest(4096)
    assert apsp.device_status() == apsp.APSP_ETIMEOUT
    assert apsp.device_status() == apsp.APSP_OK
    W = graphgen.dense_graph(260, 0.3, 8)
    D, P, _ = _run(W, np.float32)
    np.testing.assert_array_equal(D, oracle.fw(W)[0])
    assert apsp.device_status() == apsp.APSP_OK
    with pytest.raises(apsp.ApspError):
        apsp.wait_timeout_selftest(0)


def test_n131072_sampled_rows_bellman_and_paths():
    """n = 131072 (above the former 65536 cap; 1.7e10 elements, 64-bit element
    offsets and 64-bit generator indices), edge probability 0.5, integer
    weights, FP32 + path matrix (128 GiB on the device).  No whole-matrix oracle
    fits, so sampled rows are checked against the Bellman equations (exact:
    every sum is an integer below 2^24), streaming W in row chunks, and sampled
    paths are walked on the device copy of P and summed against W."""
    n, seed = 131072, 20210517
    torch.cuda.empty_cache()
    D = graphgen.dense_graph_torch(n, 0.5, seed, device=DEV)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.apsp_fw_f32(D, P)
    assert apsp.device_status() == apsp.APSP_OK
    srcs = np.random.default_rng(n).integers(0, n, 4)
    rows = D[torch.as_tensor(srcs, device=DEV)].cpu().numpy()
    best = np.full((len(srcs), n), np.inf)
    chunk = 2048
    for k0 in range(0, n, chunk):
        Wc = graphgen.dense_graph_rows_torch(n, k0, min(n, k0 + chunk), 0.5, seed, device=DEV).cpu().numpy()
        oracle.minplus_rows_accumulate(rows, Wc, k0, best)
    for t, i in enumerate(srcs):
        others = np.arange(n) != i
        assert rows[t, i] == 0
        np.testing.assert_array_equal(rows[t][others].astype(np.float64), best[t][others])
    # sampled paths: P read entry by entry from the device, weights drawn per row
    rng = np.random.default_rng(1)
    w_rows = {}

    def w_at(a, b):
        if a not in w_rows:
            w_rows[a] = graphgen.dense_graph_rows_torch(n, a, a + 1, 0.5, seed, device=DEV)[0].cpu().numpy()
        return float(w_rows[a][b])

    for t, i in enumerate(srcs):
        for j in rng.integers(0, n, 10):
            path = oracle.reconstruct_path_lookup(lambda a, c: P[a, c].item(), int(i), int(j), n + 1)
            assert path is not None and path[0] == i and path[-1] == j
            assert sum(w_at(a, b) for a, b in zip(path[:-1], path[1:])) == float(rows[t, j])
    del D, P
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [1, 130, 300, 513])
def test_int32_weights_beyond_float_exactness(n):
    """int32 weights up to 2^26 (path sums far above 2^24, where FP32 sums are
    no longer exact): apsp_fw_i32 equals the oracle's FP64 FW exactly and its
    paths sum to D; negative weights (potentials, no negative cycle) too."""
    rng = np.random.default_rng(n)
    W = graphgen.dense_graph(n, 0.3, 4000 + n, dtype=np.float64)
    fin = np.isfinite(W) & ~np.eye(n, dtype=bool)
    W[fin] = rng.integers(1, 1 << 26, fin.sum())
    for shift in (False, True):
        Wk = W.copy()
        if shift:  # Johnson-style potentials keep shortest paths, make weights negative
            h = rng.integers(-(1 << 20), 1 << 20, n).astype(np.float64)
            Wk = np.where(np.isfinite(W), W + h[:, None] - h[None, :], np.inf)
            np.fill_diagonal(Wk, 0)
        Wi = np.where(np.isfinite(Wk), Wk, apsp.I32_INF).astype(np.int32)
        D = torch.from_numpy(Wi).to(DEV)
        P = torch.empty((n, n), dtype=torch.int32, device=DEV)
        apsp.apsp_fw(D, P)
        Dh = D.cpu().numpy()
        ref = oracle.fw(Wk)[0]
        expect = np.where(np.isfinite(ref), ref, apsp.I32_INF).astype(np.int64)
        np.testing.assert_array_equal(Dh.astype(np.int64), expect)
        Df = np.where(Dh == apsp.I32_INF, np.inf, Dh.astype(np.float64))
        assert oracle.check_paths(Wk, Df, P.cpu().numpy()) == 0
        assert apsp.device_status() == apsp.APSP_OK


def test_int32_saturation_is_reported():
    """A chain whose distances leave the int32 range: saturated values and
    APSP_EUNSUPPORTED from the next device status; in-range entries exact."""
    W = graphgen.chain_graph(np.full(4, float(1 << 30)))  # 0 -> 1 -> 2 -> 3 -> 4, 2^30 each
    Wi = np.where(np.isfinite(W), W, apsp.I32_INF).astype(np.int64)
    Wi[Wi > apsp.I32_INF] = apsp.I32_INF
    D = torch.from_numpy(Wi.astype(np.int32)).to(DEV)
    apsp.apsp_fw(D)
    Dh = D.cpu().numpy().astype(np.int64)
    assert Dh[0, 1] == 1 << 30 and Dh[0, 2] == 2147483646  # 2^31 saturates to 2^31 - 2
    assert Dh[1, 0] == apsp.I32_INF
    assert apsp.device_status() == apsp.APSP_EUNSUPPORTED
    assert apsp.device_status() == apsp.APSP_OK


def test_dpx_add_min_rate_is_measured():
    """The int32 DPX fused add-min alternative is measured on this GPU (its rate
    is what keeps the integer path on the FP64/FP32-pipe kernels)."""
    r_dpx = apsp.measure_peak(-4)
    r32 = apsp.measure_peak(4)
    assert 8.0 < r_dpx <= 132.0 and r32 > 0


def test_int32_leading_dimension_and_no_path():
    """int32 with ld > n (padding columns untouched) and without a path matrix."""
    n, ld = 130, 133
    W = graphgen.dense_graph(n, 0.3, 55, dtype=np.float64)
    Wi = np.where(np.isfinite(W), W, apsp.I32_INF).astype(np.int32)
    buf = torch.full((n, ld), -5, dtype=torch.int32, device=DEV)
    buf[:, :n] = torch.from_numpy(Wi).to(DEV)
    apsp.apsp_fw_i32(buf[:, :n])
    Dh = buf[:, :n].cpu().numpy().astype(np.int64)
    ref = oracle.fw(W)[0]
    np.testing.assert_array_equal(Dh, np.where(np.isfinite(ref), ref, apsp.I32_INF).astype(np.int64))
    assert (buf[:, n:] == -5).all()
