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
