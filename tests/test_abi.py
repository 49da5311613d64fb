"""CPU-side checks of the boundary: the library builds for sm_103a, loads, and
exports every symbol include/apsp_fw.h declares (no compute calls here)."""
import ctypes
import os
import re

import paper_2105_07298_gb300 as apsp
from paper_2105_07298_gb300 import build as apsp_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "apsp_fw.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(apsp_\w+)\s*\(", txt)))


def test_header_declarations_match_binding():
    assert _declared() == sorted(apsp.SIGNATURES)


def test_library_builds_loads_and_exports():
    path = apsp_build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    L = apsp.load()
    assert L.apsp_version() >= 100
    assert L.apsp_fw_block_size(4) == 128 and L.apsp_fw_block_size(8) == 128
    assert L.apsp_fw_block_size(2) == 0
    assert L.apsp_status_string(0) == b"APSP_OK"
    assert L.apsp_batched_num_classes() == 4
    lo, hi = ctypes.c_int32(), ctypes.c_int32()
    assert L.apsp_batched_class_bounds(3, ctypes.byref(lo), ctypes.byref(hi)) == 0 and hi.value == 1024
    b, tr, tc, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    assert L.apsp_batched_variant_info(2, ctypes.byref(b), ctypes.byref(tr), ctypes.byref(tc), ctypes.byref(e)) == 0
    assert (b.value, tr.value, tc.value, e.value) == (128, 8, 4, 1)
    assert L.apsp_batched_variant_info(3, ctypes.byref(b), ctypes.byref(tr), ctypes.byref(tc), ctypes.byref(e)) == 1


def test_only_sm103a_code_in_build_flags():
    assert apsp_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_does_not_import_oracle():
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2105_07298_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", src.replace("oracle's", "")) or f.endswith(".md"), f


def test_argument_errors_without_gpu():
    """Argument checks return before any CUDA call."""
    L = apsp.load()
    assert L.apsp_fw_f32(None, 5, 5, None, None) == 1
    assert L.apsp_fw_f64(None, 5, 4, None, None) == 1
    assert L.apsp_fw_f32(None, 0, 0, None, None) == 0
    plan = ctypes.c_void_p()
    n = (ctypes.c_int32 * 1)(2000)
    off = (ctypes.c_int64 * 1)(0)
    assert L.apsp_batched_plan_create(n, off, 1, ctypes.byref(plan)) == 4
    assert L.apsp_batched_plan_create(None, None, 1, ctypes.byref(plan)) == 1


def test_new_entry_points_reject_bad_arguments_without_gpu():
    """Argument checks of the status, self-test and packed-backward entry points
    return before any CUDA call."""
    L = apsp.load()
    assert L.apsp_check_negative_cycle(None, 3, 4, 4, None) == apsp.APSP_EINVAL
    assert L.apsp_check_negative_cycle(None, 4, -1, 4, None) == apsp.APSP_EINVAL
    assert L.apsp_wait_timeout_selftest(0, None) == apsp.APSP_EINVAL
    assert L.apsp_wait_timeout_selftest((1 << 22) + 1, None) == apsp.APSP_EINVAL
    assert L.apsp_fw_backward_packed_f32(None, None, None, None, None, None, -1, None, None) == apsp.APSP_EINVAL
    assert L.apsp_fw_f32_host(None, None, None, 0, None, None, None) == apsp.APSP_OK  # n = 0: no-op
    assert L.apsp_fw_f32_host(None, None, None, 5, None, None, None) == apsp.APSP_EINVAL
    assert L.apsp_fw_f32_host(None, None, None, -1, None, None, None) == apsp.APSP_EINVAL
    assert L.apsp_fw_f32_host(None, None, None, (1 << 18) + 1, None, None, None) == apsp.APSP_EINVAL
    for st in range(8):
        assert L.apsp_status_string(st).startswith(b"APSP_")
    assert L.apsp_status_string(7) == b"APSP_ETIMEOUT: a kernel's bounded wait for an asynchronous copy ran out"


def test_batched_entry_points_reject_bad_layouts_without_gpu():
    """The batched entry points check sizes and offsets on the host before any
    CUDA call: size 0 or negative, a size above the batched limit, an offset
    that is negative or not 16-byte aligned, and (no-allocation form) more
    graphs than its fixed work list holds."""
    L = apsp.load()

    def call(fn, sizes, offs):
        n = (ctypes.c_int32 * len(sizes))(*sizes)
        o = (ctypes.c_int64 * len(offs))(*offs)
        return getattr(L, fn)(None, None, n, o, len(sizes), None)

    for fn in ("apsp_fw_batched_f32", "apsp_fw_batched_f32_noalloc"):
        assert call(fn, [4, 0], [0, 16]) == apsp.APSP_EINVAL
        assert call(fn, [4, -3], [0, 16]) == apsp.APSP_EINVAL
        assert call(fn, [4, 1025], [0, 16]) == apsp.APSP_EUNSUPPORTED
        assert call(fn, [4, 4], [0, 18]) == apsp.APSP_EINVAL      # offset not a multiple of 4
        assert call(fn, [4, 4], [0, -16]) == apsp.APSP_EINVAL
        assert getattr(L, fn)(None, None, None, None, 0, None) == apsp.APSP_OK  # empty batch: no-op
        assert getattr(L, fn)(None, None, None, None, -1, None) == apsp.APSP_EINVAL
    big = 65537
    assert call("apsp_fw_batched_f32_noalloc", [2] * big, [4 * g for g in range(big)]) == apsp.APSP_EUNSUPPORTED


def test_single_graph_and_backward_arguments_without_gpu():
    """int32 entry and the uniform backward entry check their arguments before
    any CUDA call (n out of range, ld < n, null buffers, stride too short)."""
    L = apsp.load()
    for fn in (L.apsp_fw_f32, L.apsp_fw_f64, L.apsp_fw_i32):
        assert fn(None, 0, 0, None, None) == apsp.APSP_OK                 # n = 0: no-op
        assert fn(None, -1, 4, None, None) == apsp.APSP_EINVAL
        assert fn(None, (1 << 18) + 1, (1 << 18) + 1, None, None) == apsp.APSP_EINVAL
        assert fn(None, 8, 8, None, None) == apsp.APSP_EINVAL             # null matrix
        assert fn(ctypes.c_void_p(16), 8, 7, None, None) == apsp.APSP_EINVAL  # ld < n
    bw = L.apsp_fw_backward_f32
    p = ctypes.c_void_p(16)
    assert bw(None, None, None, None, 0, 0, 1, 0, None, None) == apsp.APSP_OK   # nothing to do
    assert bw(None, None, None, None, -1, 4, 1, 16, None, None) == apsp.APSP_EINVAL
    assert bw(None, None, None, None, 4, 4, -1, 16, None, None) == apsp.APSP_EINVAL
    assert bw(p, p, None, p, 4, 4, 1, 16, None, None) == apsp.APSP_EINVAL       # null D
    assert bw(p, p, p, p, 4, 3, 1, 16, None, None) == apsp.APSP_EINVAL          # ld < n
    assert bw(p, p, p, p, 4, 4, 2, 15, None, None) == apsp.APSP_EINVAL          # graphs would overlap
