"""GPU parity of the backward (path-walk scatter) kernel and the autograd wrapper."""
import numpy as np
import pytest
import torch

import graphgen
import oracle
import paper_2105_07298_gb300 as apsp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _grad_tol(gD, P, D):
    """FP32 atomic sums in any order: error bound ~ eps * sum of |terms| per edge."""
    return oracle.fw_backward(np.abs(gD).astype(np.float64), P, D)


@pytest.mark.parametrize("n,seed", [(40, 1), (130, 2), (256, 3)])
def test_backward_matches_oracle_gradient(n, seed):
    W = graphgen.dense_graph(n, 0.4, 300 + seed, weights="real", lo=0.5, hi=2.0)
    Wt = torch.from_numpy(W).to(DEV)
    D = Wt.clone()
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.apsp_fw_f32(D, P)
    gD = graphgen.normal((n, n), seed)
    gW = apsp.apsp_fw_backward_f32(torch.from_numpy(gD).to(DEV), P, D).cpu().numpy()
    Dh, Ph = D.cpu().numpy(), P.cpu().numpy()
    ref = oracle.fw_backward(gD, Ph, Dh)
    bound = _grad_tol(gD, Ph, Dh)
    assert (np.abs(gW - ref) <= 1e-5 * np.maximum(bound, 1e-30) + 1e-30).all()
    assert (gW[~np.isfinite(W)] == 0).all() and (np.diag(gW) == 0).all()


def test_backward_batch_and_autograd_vs_finite_differences():
    """Batch of graphs through autograd; gradient vs FP64 central differences of the
    oracle's distances (h = 1e-4) on sampled edges whose paths do not switch."""
    Bn, n = 4, 48
    Ws = np.stack([graphgen.dense_graph(n, 0.4, 700 + b, weights="real", lo=0.5, hi=2.0) for b in range(Bn)])
    gD = graphgen.normal((Bn, n, n), 11)
    Wt = torch.from_numpy(Ws).to(DEV).requires_grad_(True)
    D = apsp.shortest_path_distances(Wt)
    loss = (D.masked_fill(torch.isinf(D), 0) * torch.from_numpy(gD).to(DEV)).sum()
    loss.backward()
    gW = Wt.grad.cpu().numpy()
    rng = np.random.default_rng(5)
    h = 1e-4
    checked = 0
    for b in range(Bn):
        W64 = Ws[b].astype(np.float64)
        D0, P0 = oracle.fw(W64)
        fin = np.isfinite(D0)
        edges = np.argwhere(np.isfinite(W64) & ~np.eye(n, dtype=bool))
        for u, v in edges[rng.choice(len(edges), 25, replace=False)]:
            Wp, Wm = W64.copy(), W64.copy()
            Wp[u, v] += h
            Wm[u, v] -= h
            Dp, Pp = oracle.fw(Wp)
            Dm, Pm = oracle.fw(Wm)
            if not (np.array_equal(Pp, P0) and np.array_equal(Pm, P0)):
                continue
            fd = (np.sum(gD[b][fin] * Dp[fin]) - np.sum(gD[b][fin] * Dm[fin])) / (2 * h)
            assert abs(fd - gW[b, u, v]) <= 1e-3 * max(1.0, abs(fd)), (b, u, v, fd, gW[b, u, v])
            checked += 1
    assert checked >= 40


def test_backward_config_shape_vs_oracle():
    """256 graphs, n = 256, edge probability 0.4, real weights [0.5, 2.0], dL/dD ~ N(0, 1):
    batched forward + backward; 6 sampled graphs against the oracle gradient."""
    Bn, n = 256, 256
    Ws = np.stack([graphgen.dense_graph(n, 0.4, 5000 + b, weights="real", lo=0.5, hi=2.0) for b in range(Bn)])
    gD = graphgen.normal((Bn, n, n), 12)
    Wt = torch.from_numpy(Ws).to(DEV).requires_grad_(True)
    D = apsp.shortest_path_distances(Wt)
    D.backward(torch.from_numpy(gD).to(DEV))
    gW = Wt.grad.cpu().numpy()
    Dh = D.detach().cpu().numpy()
    for b in np.random.default_rng(1).choice(Bn, 6, replace=False):
        D64, P64 = oracle.fw(Ws[b].astype(np.float64))
        fin = np.isfinite(D64)
        np.testing.assert_allclose(Dh[b][fin], D64[fin], rtol=1e-5)
        ref = oracle.fw_backward(gD[b], P64, D64)
        bound = _grad_tol(gD[b], P64, D64)
        # FP32 forward and FP64 oracle pick the same (unique) shortest paths
        assert (np.abs(gW[b] - ref) <= 1e-5 * np.maximum(bound, 1e-30) + 1e-30).all()


def test_backward_errors_and_empty():
    with pytest.raises(TypeError):
        apsp.apsp_fw_backward_f32(torch.zeros(3, 3, device=DEV), torch.zeros(3, 3, device=DEV),
                                  torch.zeros(3, 3, device=DEV))
    lib = apsp.load()
    assert lib.apsp_fw_backward_f32(None, None, None, None, 0, 0, 1, 0, None, None) == apsp.APSP_OK
    assert lib.apsp_fw_backward_f32(None, None, None, None, 4, 4, 1, 16, None, None) == apsp.APSP_EINVAL


def test_packed_uneven_backward_matches_oracle():
    """Packed batch of uneven graphs (odd sizes, 16-byte aligned offsets):
    forward through one batched launch, backward through the packed scatter
    kernel, each graph against the oracle gradient; gaps get zero gradient."""
    from paper_2105_07298_gb300 import batched as B
    sizes = [33, 5, 130, 64, 1, 97, 256]
    off = B.packed_offsets(sizes)
    total = B.packed_numel(sizes)
    Wp = np.zeros(total, dtype=np.float32)
    gDp = np.zeros(total, dtype=np.float32)
    mats = []
    for g, (n, o) in enumerate(zip(sizes, off)):
        W = graphgen.dense_graph(n, 0.4, 40 + g, weights="real", lo=0.5, hi=2.0)
        mats.append(W)
        Wp[o:o + n * n] = W.reshape(-1)
        gDp[o:o + n * n] = graphgen.normal((n, n), 60 + g).reshape(-1)
    Wt = torch.from_numpy(Wp).to(DEV).requires_grad_(True)
    D = apsp.shortest_path_distances_packed(Wt, sizes, off)
    gD = torch.from_numpy(gDp).to(DEV)
    (D.masked_fill(torch.isinf(D), 0) * gD).sum().backward()
    gW = Wt.grad.cpu().numpy()
    Dh = D.detach().cpu().numpy()
    inside = np.zeros(total, dtype=bool)
    for g, (n, o) in enumerate(zip(sizes, off)):
        inside[o:o + n * n] = True
        D64, P64 = oracle.fw(mats[g].astype(np.float64))
        fin = np.isfinite(D64)
        np.testing.assert_allclose(Dh[o:o + n * n].reshape(n, n)[fin], D64[fin], rtol=1e-5)
        gd = gDp[o:o + n * n].reshape(n, n).astype(np.float64)
        ref = oracle.fw_backward(gd, P64, D64)
        bound = _grad_tol(gd, P64, D64)
        got = gW[o:o + n * n].reshape(n, n)
        assert (np.abs(got - ref) <= 1e-5 * np.maximum(bound, 1e-30) + 1e-30).all(), g
    assert (gW[~inside] == 0).all()
    lib = apsp.load()
    assert lib.apsp_fw_backward_packed_f32(None, None, None, None, None, None, 0, None, None) == apsp.APSP_OK
    assert lib.apsp_fw_backward_packed_f32(None, None, None, None, None, None, 3, None, None) == apsp.APSP_EINVAL


@pytest.mark.parametrize("Bn,n", [(3, 33), (2, 1030)])
def test_autograd_stack_odd_and_large_n(Bn, n):
    """(B, n, n) stacks whose graphs are not 16-byte aligned back to back (odd n)
    or too large for the batched kernel (n > 1024) still solve and differentiate.
    The reference gradient walks the forward's own path matrix (from a second,
    identical solve), which must itself be valid; D is held to the FP64 oracle."""
    from paper_2105_07298_gb300 import backward as bw
    Ws = np.stack([graphgen.dense_graph(n, 0.4, 900 + b, weights="real", lo=0.5, hi=2.0) for b in range(Bn)])
    gD = graphgen.normal((Bn, n, n), 13)
    Wt = torch.from_numpy(Ws).to(DEV).requires_grad_(True)
    D = apsp.shortest_path_distances(Wt)
    D.backward(torch.from_numpy(gD).to(DEV))
    gW = Wt.grad.cpu().numpy()
    Dh = D.detach().cpu().numpy()
    D2 = torch.from_numpy(Ws).to(DEV).contiguous()
    P2 = torch.empty(D2.shape, dtype=torch.int32, device=DEV)
    bw._solve_stack(D2, P2)
    np.testing.assert_array_equal(D2.cpu().numpy(), Dh)
    Ph = P2.cpu().numpy()
    for b in range(Bn):
        D64 = oracle.fw(Ws[b].astype(np.float64))[0]
        fin = np.isfinite(D64)
        np.testing.assert_allclose(Dh[b][fin], D64[fin], rtol=1e-5)
        pairs = list(zip(*np.random.default_rng(b).integers(0, n, (2, 2000))))
        assert oracle.check_paths(Ws[b], Dh[b], Ph[b], pairs=pairs, rtol=1e-5) == 0
        ref = oracle.fw_backward(gD[b], Ph[b], Dh[b])
        bound = _grad_tol(gD[b], Ph[b], Dh[b])
        assert (np.abs(gW[b] - ref) <= 1e-5 * np.maximum(bound, 1e-30) + 1e-30).all()
