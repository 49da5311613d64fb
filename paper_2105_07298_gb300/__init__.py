"""GB300 (sm_103a) blocked Floyd-Warshall all-pairs shortest paths.

A thin Python binding over the C ABI in ``include/apsp_fw.h`` (``libapspfw.so``,
built from ``csrc/`` by :mod:`paper_2105_07298_gb300.build`).  Every function
here only marshals arguments (device pointers, sizes, the current CUDA stream)
and calls the library; all of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the library cannot be loaded, every call
raises.

Method: Costanzo et al., arXiv 2105.07298, §2.2 (Algorithm 1, blocked FW with
four phases per round) and §3.2 (kernel split per round).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libapspfw.so")

(APSP_OK, APSP_EINVAL, APSP_ECUDA, APSP_ENOMEM, APSP_EUNSUPPORTED, APSP_ETOODEEP, APSP_ENEGCYCLE,
 APSP_ETIMEOUT) = range(8)

# Every symbol include/apsp_fw.h declares, with its ctypes signature.
_i32, _i64, _p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
SIGNATURES = {
    "apsp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "apsp_version": (ctypes.c_int, []),
    "apsp_fw_block_size": (ctypes.c_int, [ctypes.c_int]),
    "apsp_fw_f32": (ctypes.c_int, [_p, _i64, _i64, _p, _p]),
    "apsp_fw_f64": (ctypes.c_int, [_p, _i64, _i64, _p, _p]),
    "apsp_fw_i32": (ctypes.c_int, [_p, _i64, _i64, _p, _p]),
    "apsp_batched_plan_create": (ctypes.c_int, [_p, _p, _i32, ctypes.POINTER(_p)]),
    "apsp_batched_plan_destroy": (ctypes.c_int, [_p]),
    "apsp_fw_batched_run_f32": (ctypes.c_int, [_p, _p, _p, _p]),
    "apsp_fw_batched_f32": (ctypes.c_int, [_p, _p, _p, _p, _i32, _p]),
    "apsp_fw_batched_f32_noalloc": (ctypes.c_int, [_p, _p, _p, _p, _i32, _p]),
    "apsp_batched_num_classes": (ctypes.c_int, []),
    "apsp_batched_class_bounds": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "apsp_batched_num_variants": (ctypes.c_int, [ctypes.c_int]),
    "apsp_batched_set_variant": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "apsp_batched_get_variant": (ctypes.c_int, [ctypes.c_int]),
    "apsp_batched_variant_info": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                                 ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "apsp_fw_backward_f32": (ctypes.c_int, [_p, _p, _p, _p, _i64, _i64, _i64, _i64, _p, _p]),
    "apsp_fw_backward_packed_f32": (ctypes.c_int, [_p, _p, _p, _p, _p, _p, _i32, _p, _p]),
    "apsp_check_negative_cycle": (ctypes.c_int, [_p, ctypes.c_int, _i64, _i64, _p]),
    "apsp_fw_f32_host": (ctypes.c_int, [_p, _p, _p, _i64, _p, _p, _p]),
    "apsp_wait_timeout_selftest": (ctypes.c_int, [ctypes.c_uint32, _p]),
    "apsp_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "apsp_device_status": (ctypes.c_int, [_p]),
    "apsp_measure_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _p]),
    "apsp_profile_collect": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)]),
    "apsp_profile_records": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
                                            _i64, ctypes.POINTER(_i64)]),
}

_lock = threading.Lock()
_lib = None


class ApspError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = load().apsp_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg}" if where else msg)


def load(path: str | None = None):
    """Load libapspfw.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                from . import build as _build
                _build.build()
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != APSP_OK:
        raise ApspError(status, where)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(int(s.cuda_stream))


def _matrix_args(t, dtype):
    """(ptr, n, ld) of an n x n row-major view with unit column stride."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError(f"expected an n x n matrix, got shape {tuple(t.shape)}")
    n = t.shape[0]
    if n > 1 and t.stride(1) != 1:
        raise ValueError("columns must be contiguous (stride(1) == 1)")
    ld = t.stride(0) if n > 1 else max(n, 1)
    return ctypes.c_void_p(t.data_ptr()), n, ld


def block_size(dtype) -> int:
    """Block edge TB the single-graph kernels use for ``dtype`` (torch.float32/float64)."""
    import torch
    return int(load().apsp_fw_block_size(4 if dtype == torch.float32 else 8))


def _fw(fn_name, dist, path, stream, dtype):
    import torch
    ptr, n, ld = _matrix_args(dist, dtype)
    pptr = None
    if path is not None:
        pp, pn, pld = _matrix_args(path, torch.int32)
        if pn != n or pld != ld or path.device != dist.device:
            raise ValueError("path must be an int32 matrix with the same n, ld and device as dist")
        pptr = pp
    _check(getattr(load(), fn_name)(ptr, n, ld, pptr, _stream_ptr(stream)), fn_name)
    return dist, path


def apsp_fw_f32(dist, path=None, stream=None):
    """In-place FP32 blocked Floyd-Warshall on a CUDA n x n tensor (optionally writing ``path``)."""
    import torch
    return _fw("apsp_fw_f32", dist, path, stream, torch.float32)


def _host_matrix(t, dtype, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("expected a CPU (host) tensor")
    if t.dtype != dtype or t.dim() != 2 or t.shape[0] != t.shape[1] or not t.is_contiguous():
        raise ValueError(f"expected a contiguous n x n {dtype} host matrix")
    if n is not None and t.shape[0] != n:
        raise ValueError("host matrices must have the same n")
    return ctypes.c_void_p(t.data_ptr())


def _device_work(t, dtype, n):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or t.numel() < n * n \
            or not t.is_contiguous():
        raise ValueError(f"work buffer must be a contiguous CUDA {dtype} tensor of at least n*n elements")
    return ctypes.c_void_p(t.data_ptr())


def apsp_fw_f32_host(weights, dist=None, path=None, work_dist=None, work_path=None, stream=None,
                     with_path=True):
    """FP32 solve from and to host memory (the end-to-end call, one C-ABI call):
    ``weights`` is a contiguous CPU float32 n x n tensor; the distances go to
    ``dist`` and the path matrix to ``path`` (CPU tensors; page-locked ones are
    allocated when None; ``with_path=False`` skips P).  ``work_dist`` /
    ``work_path``: optional CUDA tensors the call uses on the device (kept by a
    caller that solves repeatedly).  Returns (dist, path)."""
    import torch
    wp = _host_matrix(weights, torch.float32)
    n = weights.shape[0]
    if dist is None:
        dist = torch.empty((n, n), dtype=torch.float32, pin_memory=torch.cuda.is_available())
    if with_path and path is None:
        path = torch.empty((n, n), dtype=torch.int32, pin_memory=torch.cuda.is_available())
    dp = _host_matrix(dist, torch.float32, n)
    pp = _host_matrix(path, torch.int32, n) if with_path else None
    st = load().apsp_fw_f32_host(wp, dp, pp, n, _device_work(work_dist, torch.float32, n),
                                 _device_work(work_path, torch.int32, n), _stream_ptr(stream))
    _check(st, "apsp_fw_f32_host")
    return dist, (path if with_path else None)


def apsp_fw_f64(dist, path=None, stream=None):
    """In-place FP64 blocked Floyd-Warshall on a CUDA n x n tensor (optionally writing ``path``)."""
    import torch
    return _fw("apsp_fw_f64", dist, path, stream, torch.float64)


I32_INF = 0x7FFFFFFF  # APSP_I32_INF: no edge / no path in an int32 matrix


def apsp_fw_i32(dist, path=None, stream=None):
    """In-place exact blocked Floyd-Warshall on a CUDA int32 n x n tensor
    (``I32_INF`` marks a missing edge), optionally writing ``path``."""
    import torch
    return _fw("apsp_fw_i32", dist, path, stream, torch.int32)


def apsp_fw(dist, path=None, stream=None):
    """Dispatch on dtype to :func:`apsp_fw_f32` / :func:`apsp_fw_f64` / :func:`apsp_fw_i32`."""
    import torch
    if dist.dtype == torch.float32:
        return apsp_fw_f32(dist, path, stream)
    if dist.dtype == torch.float64:
        return apsp_fw_f64(dist, path, stream)
    if dist.dtype == torch.int32:
        return apsp_fw_i32(dist, path, stream)
    raise TypeError(f"unsupported dtype {dist.dtype}")


def device_status(stream=None) -> int:
    """Synchronize the stream; return (and clear) the kernels' device-side error word."""
    return int(load().apsp_device_status(_stream_ptr(stream)))


def wait_timeout_selftest(polls: int = 4096, stream=None):
    """Enqueue the bounded-wait self-test kernel (its wait runs out; see apsp_fw.h)."""
    _check(load().apsp_wait_timeout_selftest(int(polls), _stream_ptr(stream)), "apsp_wait_timeout_selftest")


def check_negative_cycle(dist, stream=None) -> bool:
    """True if the solved CUDA matrix ``dist`` has a negative diagonal entry (a
    negative cycle in the input).  Synchronizes the stream."""
    import torch
    ptr, n, ld = _matrix_args(dist, dist.dtype if dist.dtype in (torch.float32, torch.float64) else torch.float32)
    st = load().apsp_check_negative_cycle(ptr, dist.element_size(), n, ld, _stream_ptr(stream))
    if st == APSP_ENEGCYCLE:
        return True
    _check(st, "apsp_check_negative_cycle")
    return False


def measure_peak(dtype_bytes: int = 4, stream=None) -> float:
    """Relaxations per clock per SM the inner-loop instruction pair sustains on this GPU."""
    out = ctypes.c_double()
    _check(load().apsp_measure_peak(dtype_bytes, ctypes.byref(out), _stream_ptr(stream)), "apsp_measure_peak")
    return out.value


PHASES = ("path_init", "phase1_diag", "phase2_panels", "phase3_minplus")


def profile_enable(on: bool = True):
    """Start (clearing old records) or stop per-phase CUDA-event timing in the library."""
    _check(load().apsp_profile_enable(1 if on else 0), "apsp_profile_enable")


def profile_collect() -> dict:
    """{phase: (total_ms, launches)} of the launches recorded since profile_enable(True)."""
    ms = (ctypes.c_double * 4)()
    cnt = (ctypes.c_int64 * 4)()
    _check(load().apsp_profile_collect(ms, cnt), "apsp_profile_collect")
    return {PHASES[p]: (float(ms[p]), int(cnt[p])) for p in range(4)}


def profile_records() -> list:
    """[(phase, ms)] of every recorded launch, in launch order."""
    lib = load()
    count = _i64(0)
    _check(lib.apsp_profile_records(None, None, 0, ctypes.byref(count)), "apsp_profile_records")
    cap = int(count.value)
    ph = (ctypes.c_int32 * max(cap, 1))()
    ms = (ctypes.c_float * max(cap, 1))()
    _check(lib.apsp_profile_records(ph, ms, cap, ctypes.byref(count)), "apsp_profile_records")
    return [(PHASES[ph[i]], float(ms[i])) for i in range(min(cap, int(count.value)))]


from .batched import BatchedPlan, apsp_fw_batched_f32, apsp_fw_batched  # noqa: E402
from .backward import (apsp_fw_backward_f32, apsp_fw_backward_packed_f32, ShortestPathDistances,  # noqa: E402
                       shortest_path_distances, shortest_path_distances_packed)

__all__ = [
    "load", "ApspError", "block_size", "apsp_fw_f32", "apsp_fw_f64", "apsp_fw_i32", "apsp_fw", "I32_INF",
    "BatchedPlan", "apsp_fw_batched_f32", "apsp_fw_batched", "apsp_fw_backward_f32",
    "apsp_fw_backward_packed_f32", "ShortestPathDistances", "shortest_path_distances",
    "shortest_path_distances_packed", "check_negative_cycle", "wait_timeout_selftest",
]
