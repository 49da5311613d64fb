"""The no-allocation batched entry point, called through the C ABI.

It serves callers that cannot allocate device memory at call time (a serving
loop that forbids cudaMalloc on its hot path, memory owned by a foreign
allocator, embeddings where hidden allocations are errors): its work list
lives in a fixed device array of the library.  Checked against the allocating
entry point on two calls in a row (the shared array keeps the previous call's
contents, which must not leak into the next result).  This file is collected
last on purpose, and must pass alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen
import paper_2105_07298_gb300 as apsp
from paper_2105_07298_gb300 import batched as B

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _packed(sizes, seed):
    off = B.packed_offsets(sizes)
    total = B.packed_numel(sizes)
    W = graphgen.batched_graphs_torch(sizes, 0.3, seed, off, total, device=DEV)
    return W, off


def _call(fn, W, sizes, off):
    lib = apsp.load()
    n = np.ascontiguousarray(sizes, dtype=np.int32)
    o = np.ascontiguousarray(off, dtype=np.int64)
    D = W.clone()
    P = torch.full_like(D, 7, dtype=torch.int32)
    st = getattr(lib, fn)(ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                          n.ctypes.data_as(ctypes.c_void_p), o.ctypes.data_as(ctypes.c_void_p),
                          len(n), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, D, P


def test_no_alloc_matches_allocating_entry_point_twice():
    runs = [([300, 17, 64, 129, 1, 512, 250, 96], 3), ([40, 256, 257, 3, 128, 65], 4)]
    for sizes, seed in runs:  # two calls in a row, different batches
        W, off = _packed(sizes, seed)
        st_ref, D_ref, P_ref = _call("apsp_fw_batched_f32", W, sizes, off)
        st, D, P = _call("apsp_fw_batched_f32_noalloc", W, sizes, off)
        assert st_ref == apsp.APSP_OK and st == apsp.APSP_OK
        # integer weights: every sum is exact, so the distances agree bit for bit;
        # compare graph by graph (the alignment gaps between graphs hold NaN and
        # must stay untouched)
        for n, o in zip(sizes, off):
            sl = slice(int(o), int(o) + n * n)
            assert torch.equal(D[sl], D_ref[sl])
            assert torch.equal(P[sl], P_ref[sl])
        gaps = torch.isnan(W)
        assert torch.isnan(D[gaps]).all() and torch.isnan(D_ref[gaps]).all()


def test_no_alloc_rejects_oversized_batch():
    lib = apsp.load()
    num = 65537
    n = np.full(num, 2, dtype=np.int32)
    o = (np.arange(num, dtype=np.int64) * 4)
    st = lib.apsp_fw_batched_f32_noalloc(None, None, n.ctypes.data_as(ctypes.c_void_p),
                                         o.ctypes.data_as(ctypes.c_void_p), num, None)
    assert st == apsp.APSP_EUNSUPPORTED
