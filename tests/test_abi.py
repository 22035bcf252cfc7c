"""C-ABI checks that need no GPU: the library loads, exports every entry
point include/mmr.h declares, and reports errors instead of crashing."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2504_20937_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, fn)).read()
            names |= set(re.findall(r"^MMR_API\s+[^;(]*?\b(mmr\w+)\s*\(", text, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mmr_create", "mmr_alloc_points", "mmr_set_camera", "mmr_step_and_render",
                     "mmr_frame_ptr", "mmr_destroy", "mmr_render", "mmr_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for name in _declared():
        assert hasattr(lib, name)


def test_binding_covers_every_declared_symbol():
    assert _declared() <= set(_lib.SIGNATURES)


def test_status_strings():
    lib = _lib.load()
    assert lib.mmr_status_string(0) == b"ok"
    assert lib.mmr_status_string(-3) == b"over device-memory budget"
    assert lib.mmr_status_string(42) == b"unknown status"


def test_invalid_arguments_rejected_without_device():
    lib = _lib.load()
    h = C.c_void_p()
    assert lib.mmr_create(0, 10, C.byref(h)) == -1
    assert h.value is None
    assert b"outside" in lib.mmr_last_error(None)
    assert lib.mmr_create(10, 40000, C.byref(h)) == -1
    assert lib.mmr_create(10, 10, None) == -1
    assert lib.mmr_destroy(None) == 0
    assert lib.mmr_step_and_render(None, None) == -1
    assert lib.mmr_frame_ptr(None, None, None) == -1


def test_create_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = _lib.load()
    h = C.c_void_p()
    st = lib.mmr_create(64, 64, C.byref(h))
    assert st == -4 and h.value is None
    assert b"CUDA" in lib.mmr_last_error(None) or b"cuda" in lib.mmr_last_error(None)


def test_group_counts_at_the_largest_point_counts():
    """groups_of (csrc/mmr_points.cuh) for n up to 2^32 - 1, checked by
    static_asserts that nvcc evaluates on the host (no GPU needed)."""
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    obj = os.path.join(out_dir, f"groups_check_{os.getpid()}.o")
    r = subprocess.run(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
                        "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "paper_2504_20937_b300", "csrc"),
                        "-c", os.path.join(ROOT, "tests", "cuda", "groups_check.cu"), "-o", obj],
                       capture_output=True, text=True)
    if os.path.exists(obj):
        os.remove(obj)
    assert r.returncode == 0, r.stderr
