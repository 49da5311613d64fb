"""Differentiable shortest-path distances: forward = Floyd-Warshall with a path
matrix, backward = the library's path-walk scatter kernel.

D[i][j] is the sum of the weights on path(i,j) (the path P encodes), so
dL/dW[u][v] sums dL/dD[i][j] over the pairs whose path uses edge (u,v).  The
forward pass keeps only D and P; the backward kernel recomputes every path.
Argument marshalling only: the solves and the scatter run in the library.
"""
from __future__ import annotations

import ctypes

import numpy as np


def _raise_status(status):
    from . import ApspError, APSP_OK
    if status is not None:
        st = int(status.item())
        if st != APSP_OK:
            raise ApspError(st, "backward")


def apsp_fw_backward_f32(grad_dist, path, dist, grad_w=None, stream=None, check=True):
    """dL/dW from dL/dD for one graph (n x n) or a batch (B x n x n) of CUDA tensors."""
    import torch
    from . import load, _check, _stream_ptr
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
    _raise_status(status)
    return grad_w


def apsp_fw_backward_packed_f32(grad_dist, path, dist, sizes_dev, offsets_dev, grad_w=None, stream=None,
                                check=True):
    """dL/dW for a packed batch of uneven graphs (the batched forward's layout).

    ``grad_dist``, ``path``, ``dist`` (and ``grad_w``) are 1-D packed CUDA
    buffers; ``sizes_dev`` / ``offsets_dev`` are CUDA int32 / int64 tensors with
    one entry per graph.  Regions between graphs of ``grad_w`` are left as they are.
    """
    import torch
    from . import load, _check, _stream_ptr
    for t, dt in ((grad_dist, torch.float32), (path, torch.int32), (dist, torch.float32),
                  (sizes_dev, torch.int32), (offsets_dev, torch.int64)):
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise TypeError("expected contiguous CUDA tensors: float32 grad/dist, int32 path and sizes, "
                            "int64 offsets")
    if sizes_dev.shape != offsets_dev.shape or sizes_dev.dim() != 1:
        raise ValueError("sizes and offsets must be 1-D with one entry per graph")
    if not (grad_dist.numel() == path.numel() == dist.numel()):
        raise ValueError("packed buffers must have the same length")
    if grad_w is None:
        grad_w = torch.zeros_like(grad_dist)
    status = torch.zeros(1, dtype=torch.int32, device=grad_dist.device) if check else None
    _check(load().apsp_fw_backward_packed_f32(
        ctypes.c_void_p(grad_dist.data_ptr()), ctypes.c_void_p(path.data_ptr()),
        ctypes.c_void_p(dist.data_ptr()), ctypes.c_void_p(grad_w.data_ptr()),
        ctypes.c_void_p(sizes_dev.data_ptr()), ctypes.c_void_p(offsets_dev.data_ptr()), int(sizes_dev.numel()),
        ctypes.c_void_p(status.data_ptr()) if status is not None else None, _stream_ptr(stream)),
        "apsp_fw_backward_packed_f32")
    _raise_status(status)
    return grad_w


def _solve_stack(D, P):
    """Solve every graph of the contiguous (B, n, n) float32 tensor D in place,
    writing P.  Graphs the batched kernel takes (n <= 1024) go through one
    persistent launch: directly when every graph starts 16-byte aligned (n^2 a
    multiple of 4), otherwise through a copy in the aligned packed layout.
    Larger graphs are solved one by one by the single-graph path."""
    from . import apsp_fw_f32
    from .batched import BatchedPlan, packed_offsets, packed_numel, MAX_N
    B, n, _ = D.shape
    if n > MAX_N:
        for b in range(B):
            apsp_fw_f32(D[b], P[b])
        return
    sizes = [n] * B
    if (n * n) % 4 == 0:
        plan = BatchedPlan(sizes, [b * n * n for b in range(B)])
        plan.run(D.view(-1), P.view(-1))
        plan.close()
        return
    import torch
    off = packed_offsets(sizes)
    total = packed_numel(sizes)
    idx = (torch.from_numpy(off).to(D.device)[:, None] + torch.arange(n * n, device=D.device)[None, :])
    Dp = torch.empty(total, dtype=D.dtype, device=D.device)
    Pp = torch.empty(total, dtype=torch.int32, device=D.device)
    Dp[idx] = D.view(B, -1)
    plan = BatchedPlan(sizes, off)
    plan.run(Dp, Pp)
    plan.close()
    D.view(B, -1).copy_(Dp[idx])
    P.view(B, -1).copy_(Pp[idx])


class ShortestPathDistances:
    """torch.autograd.Function factory (built lazily so importing needs no torch)."""
    _fn = None
    _packed = None

    @classmethod
    def get(cls):
        if cls._fn is None:
            import torch
            from . import apsp_fw_f32

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
                        _solve_stack(D, P)
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

    @classmethod
    def get_packed(cls):
        if cls._packed is None:
            import torch
            from .batched import BatchedPlan

            class _Packed(torch.autograd.Function):
                @staticmethod
                def forward(ctx, Wp, sizes, offsets):
                    if Wp.dtype != torch.float32 or not Wp.is_cuda or Wp.dim() != 1:
                        raise TypeError("W must be a 1-D CUDA float32 packed buffer")
                    D = Wp.detach().contiguous().clone()
                    P = torch.full(D.shape, -1, dtype=torch.int32, device=D.device)
                    plan = BatchedPlan(sizes, offsets)
                    plan.run(D, P)
                    plan.close()
                    n_dev = torch.from_numpy(np.ascontiguousarray(plan.sizes)).to(D.device)
                    off_dev = torch.from_numpy(np.ascontiguousarray(plan.offsets)).to(D.device)
                    ctx.save_for_backward(D, P, n_dev, off_dev)
                    return D

                @staticmethod
                def backward(ctx, gD):
                    D, P, n_dev, off_dev = ctx.saved_tensors
                    return apsp_fw_backward_packed_f32(gD.contiguous(), P, D, n_dev, off_dev), None, None

            cls._packed = _Packed
        return cls._packed


def shortest_path_distances(W):
    """All-pairs shortest-path distances of W (n x n or B x n x n), differentiable in W."""
    return ShortestPathDistances.get().apply(W)


def shortest_path_distances_packed(W_packed, sizes, offsets=None):
    """Distances of a packed batch of uneven graphs (the batched layout: graph g
    has sizes[g] vertices at element offset offsets[g], default back to back
    with 16-byte alignment), differentiable in the packed weights.  The forward
    is one batched launch, the backward one packed scatter launch; entries
    between graphs pass through unchanged and get a zero gradient."""
    from .batched import packed_offsets
    if offsets is None:
        offsets = packed_offsets(sizes)
    return ShortestPathDistances.get_packed().apply(W_packed, sizes, offsets)
