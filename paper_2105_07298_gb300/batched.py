"""Binding for the batched entry points (packed graphs, one persistent launch).

Argument marshalling only; the graphs are solved by the library's
``fw_batched_persistent_f32`` kernel.
"""
from __future__ import annotations

import ctypes

import numpy as np

MAX_N = 1024  # largest graph the batched kernel takes (apsp_batched_class_bounds)


def _host_arrays(sizes, offsets):
    n = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32))
    if offsets is None:
        off = np.zeros(len(n), dtype=np.int64)
        if len(n) > 1:
            sq = n.astype(np.int64) ** 2
            sq = (sq + 3) // 4 * 4  # keep every graph 16-byte aligned
            off[1:] = np.cumsum(sq)[:-1]
    else:
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if off.shape != n.shape:
        raise ValueError("sizes and offsets must have the same length")
    return n, off


def _layout_numel(n, off) -> int:
    """Elements the packed layout spans (end of its last-ending graph)."""
    return int(np.max(off + n.astype(np.int64) ** 2)) if len(n) else 0


def _check_buffers(dist, path, need: int):
    """The packed buffers a batched call writes: ``dist`` a contiguous CUDA
    float32 tensor of at least ``need`` elements; ``path`` (optional) a
    contiguous int32 tensor on the same device, as large as ``dist``."""
    import torch
    if dist.dtype != torch.float32 or not dist.is_cuda or not dist.is_contiguous():
        raise TypeError("dist must be a contiguous CUDA float32 tensor")
    if path is not None and (path.dtype != torch.int32 or not path.is_cuda or path.device != dist.device
                             or not path.is_contiguous() or path.numel() < dist.numel()):
        raise TypeError("path must be a contiguous int32 tensor on dist's device, as large as dist")
    if dist.numel() < need:
        raise ValueError(f"dist has {dist.numel()} elements, layout needs {need}")


def packed_offsets(sizes):
    """Element offsets for graphs packed back to back, each rounded up to 4 elements."""
    return _host_arrays(sizes, None)[1]


def packed_numel(sizes) -> int:
    n, off = _host_arrays(sizes, None)
    return int(off[-1] + int(n[-1]) ** 2) if len(n) else 0


class BatchedPlan:
    """A reusable plan (size classes, LPT order, device work list) for a fixed layout."""

    def __init__(self, sizes, offsets=None):
        from . import load, _check
        self._lib = load()
        self.sizes, self.offsets = _host_arrays(sizes, offsets)
        self._h = ctypes.c_void_p()
        _check(self._lib.apsp_batched_plan_create(
            self.sizes.ctypes.data_as(ctypes.c_void_p), self.offsets.ctypes.data_as(ctypes.c_void_p),
            len(self.sizes), ctypes.byref(self._h)), "apsp_batched_plan_create")

    def run(self, dist, path=None, stream=None):
        """Solve every graph in the packed FP32 buffer ``dist`` (and write ``path``) in place."""
        from . import _check, _stream_ptr
        _check_buffers(dist, path, _layout_numel(self.sizes, self.offsets))
        _check(self._lib.apsp_fw_batched_run_f32(
            self._h, ctypes.c_void_p(dist.data_ptr()),
            ctypes.c_void_p(path.data_ptr()) if path is not None else None, _stream_ptr(stream)),
            "apsp_fw_batched_run_f32")
        return dist, path

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.apsp_batched_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apsp_fw_batched_f32(dist, sizes, offsets=None, path=None, stream=None):
    """One-shot batched solve (plan, run and free in one call)."""
    from . import load, _check, _stream_ptr
    n, off = _host_arrays(sizes, offsets)
    _check_buffers(dist, path, _layout_numel(n, off))
    _check(load().apsp_fw_batched_f32(
        ctypes.c_void_p(dist.data_ptr()), ctypes.c_void_p(path.data_ptr()) if path is not None else None,
        n.ctypes.data_as(ctypes.c_void_p), off.ctypes.data_as(ctypes.c_void_p), len(n),
        _stream_ptr(stream)), "apsp_fw_batched_f32")
    return dist, path


apsp_fw_batched = apsp_fw_batched_f32


def num_classes() -> int:
    from . import load
    return int(load().apsp_batched_num_classes())


def class_bounds(cls: int):
    from . import load, _check
    lo, hi = ctypes.c_int32(), ctypes.c_int32()
    _check(load().apsp_batched_class_bounds(cls, ctypes.byref(lo), ctypes.byref(hi)), "class_bounds")
    return lo.value, hi.value


def num_variants(cls: int) -> int:
    from . import load
    return int(load().apsp_batched_num_variants(cls))


def set_variant(cls: int, variant: int):
    from . import load, _check
    _check(load().apsp_batched_set_variant(cls, variant), "set_variant")


def get_variant(cls: int) -> int:
    from . import load
    return int(load().apsp_batched_get_variant(cls))


def variant_info(variant: int) -> dict:
    """Block edge, register tile and path tracking of a batched kernel variant."""
    from . import load, _check
    b, tr, tc, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().apsp_batched_variant_info(variant, ctypes.byref(b), ctypes.byref(tr), ctypes.byref(tc),
                                            ctypes.byref(e)), "variant_info")
    return {"block": b.value, "tile": f"{tr.value}x{tc.value}", "path": "eager" if e.value else "lazy"}
