"""Differentiable shortest-path distances: forward = Floyd-Warshall with a path
matrix, backward = the library's path-walk scatter kernel.

D[i][j] is the sum of the weights on path(i,j) (the path P encodes), so
dL/dW[u][v] sums dL/dD[i][j] over the pairs whose path uses edge (u,v).  The
forward pass keeps only D and P; the backward kernel recomputes every path.
"""
from __future__ import annotations

import ctypes


def apsp_fw_backward_f32(grad_dist, path, dist, grad_w=None, stream=None, check=True):
    """dL/dW from dL/dD for one graph (n x n) or a batch (B x n x n) of CUDA tensors."""
    import torch
    from . import load, _check, _stream_ptr, ApspError, APSP_OK
    for t, dt in ((grad_dist, torch.float32), (path, torch.int32), (dist, torch.float32)):
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise TypeError("expected contiguous CUDA tensors: float32 grad/dist, int32 path")
    if not (grad_dist.shape == path.shape == dist.shape) or grad_dist.dim() not in (2, 3):
        raise ValueError("grad_dist, path and dist must share an (n, n) or (B, n, n) shape")
    batch = 1 if grad_dist.dim() == 2 else grad_dist.shape[0]
    n = grad_dist.shape[-1]
    if grad_w is None:
        grad_w = torch.empty_like(grad_dist)
    status = torch.zeros(1, dtype=torch.int32, device=grad_dist.device) if check else None
    _check(load().apsp_fw_backward_f32(
        ctypes.c_void_p(grad_dist.data_ptr()), ctypes.c_void_p(path.data_ptr()),
        ctypes.c_void_p(dist.data_ptr()), ctypes.c_void_p(grad_w.data_ptr()), n, n, batch, n * n,
        ctypes.c_void_p(status.data_ptr()) if status is not None else None, _stream_ptr(stream)),
        "apsp_fw_backward_f32")
    if status is not None:
        st = int(status.item())
        if st != APSP_OK:
            raise ApspError(st, "apsp_fw_backward_f32")
    return grad_w


class ShortestPathDistances:
    """torch.autograd.Function factory (built lazily so importing needs no torch)."""
    _fn = None

    @classmethod
    def get(cls):
        if cls._fn is None:
            import torch
            from . import apsp_fw_f32
            from .batched import BatchedPlan

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, W):
                    if W.dtype != torch.float32 or not W.is_cuda:
                        raise TypeError("W must be a CUDA float32 tensor")
                    D = W.detach().contiguous().clone()
                    P = torch.empty(D.shape, dtype=torch.int32, device=D.device)
                    if D.dim() == 2:
                        apsp_fw_f32(D, P)
                    elif D.dim() == 3:
                        B, n, _ = D.shape
                        plan = BatchedPlan([n] * B, [b * n * n for b in range(B)])
                        plan.run(D.view(-1), P.view(-1))
                        plan.close()
                    else:
                        raise ValueError("W must be (n, n) or (B, n, n)")
                    ctx.save_for_backward(D, P)
                    return D

                @staticmethod
                def backward(ctx, gD):
                    D, P = ctx.saved_tensors
                    return apsp_fw_backward_f32(gD.contiguous(), P, D)

            cls._fn = _Fn
        return cls._fn


def shortest_path_distances(W):
    """All-pairs shortest-path distances of W (n x n or B x n x n), differentiable in W."""
    return ShortestPathDistances.get().apply(W)
