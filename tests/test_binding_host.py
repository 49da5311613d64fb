"""Host-side argument checks of the Python binding (no GPU: every bad call must
raise before anything reaches the library or a device)."""
import numpy as np
import pytest
import torch

import paper_2105_07298_gb300 as apsp
from paper_2105_07298_gb300 import batched as B


class _Buf:
    """Stand-in for a tensor: only the attributes the checks read."""

    def __init__(self, dtype=torch.float32, cuda=True, contiguous=True, numel=64, device="cuda:0"):
        self.dtype, self.is_cuda, self._c, self._n = dtype, cuda, contiguous, numel
        self.device = torch.device(device)

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n


def test_packed_buffers_accepted():
    B._check_buffers(_Buf(), None, 64)
    B._check_buffers(_Buf(), _Buf(dtype=torch.int32), 64)
    B._check_buffers(_Buf(numel=70), _Buf(dtype=torch.int32, numel=80), 64)


@pytest.mark.parametrize("dist", [_Buf(dtype=torch.float64), _Buf(cuda=False, device="cpu"),
                                  _Buf(contiguous=False)])
def test_packed_distances_rejected(dist):
    with pytest.raises(TypeError):
        B._check_buffers(dist, None, 64)


@pytest.mark.parametrize("path", [_Buf(dtype=torch.float32), _Buf(dtype=torch.int32, cuda=False, device="cpu"),
                                  _Buf(dtype=torch.int32, device="cuda:1"),
                                  _Buf(dtype=torch.int32, contiguous=False),
                                  _Buf(dtype=torch.int32, numel=63)])
def test_packed_path_rejected(path):
    """A host, other-device, strided, mistyped or short path buffer would be
    written out of bounds by the kernel: refused before the call."""
    with pytest.raises(TypeError):
        B._check_buffers(_Buf(), path, 64)


def test_packed_distances_shorter_than_layout_rejected():
    sizes = [5, 17, 3]
    n, off = B._host_arrays(sizes, None)
    need = B._layout_numel(n, off)
    assert need == B.packed_numel(sizes) == off[-1] + 9
    with pytest.raises(ValueError):
        B._check_buffers(_Buf(numel=need - 1), None, need)
    assert B._layout_numel(np.zeros(0, np.int32), np.zeros(0, np.int64)) == 0


def test_packed_layout_is_aligned_and_ordered():
    sizes = [1, 2, 3, 5, 7, 64, 129]
    off = B.packed_offsets(sizes)
    assert (off % 4 == 0).all() and off[0] == 0
    ends = off + np.asarray(sizes, dtype=np.int64) ** 2
    assert (ends[:-1] <= off[1:]).all()          # no overlap
    assert (off[1:] - ends[:-1] < 4).all()       # at most 3 padding elements
    with pytest.raises(ValueError):
        B._host_arrays([3, 4], [0])


def test_single_graph_binding_rejects_host_and_malformed_tensors():
    with pytest.raises(TypeError):
        apsp.apsp_fw_f32(torch.zeros(4, 4))                       # host tensor
    with pytest.raises(TypeError):
        apsp.apsp_fw(torch.zeros(4, 4, dtype=torch.float16))     # unsupported dtype
    with pytest.raises(ValueError):
        apsp.apsp_fw_f32_host(torch.zeros(4, 4, dtype=torch.float64))   # wrong dtype
    with pytest.raises(ValueError):
        apsp.apsp_fw_f32_host(torch.zeros(4, 5))                        # not square


def test_backward_binding_rejects_host_tensors():
    g = torch.zeros(4, 4)
    with pytest.raises(TypeError):
        apsp.apsp_fw_backward_f32(g, torch.zeros(4, 4, dtype=torch.int32), g)
    with pytest.raises(TypeError):
        apsp.apsp_fw_backward_packed_f32(g.view(-1), torch.zeros(16, dtype=torch.int32), g.view(-1),
                                         torch.ones(1, dtype=torch.int32), torch.zeros(1, dtype=torch.int64))
