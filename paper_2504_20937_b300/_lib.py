"""ctypes binding of libmmr (include/mmr.h): argument marshalling only.

Every step of the displace + render path runs in the library's CUDA kernels.
PyTorch is used only to hold device memory (views of library-owned buffers)
and to supply streams.  There is no fallback: if libmmr.so is missing or a
call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmmr.so")

MMR_OK = 0
STATUS = {0: "MMR_OK", -1: "MMR_ERR_INVALID_ARG", -2: "MMR_ERR_OOM", -3: "MMR_ERR_BUDGET",
          -4: "MMR_ERR_CUDA", -5: "MMR_ERR_STATE", -6: "MMR_ERR_TIMEOUT"}
DTYPE_CODE = {"f32": 0, "f16": 1, "bf16": 2}
KERNEL_CODE = {"grid": 0, "tma": 1, "depth_bound": 2, "warp_agg": 3, "auto": 4}

_vp = C.c_void_p
_u64 = C.c_uint64
_u32 = C.c_uint32
_i = C.c_int
_d = C.c_double
_f = C.c_float
_d3 = C.c_double * 3
_f16 = C.c_float * 16

# name -> (restype, argtypes); the exported surface of include/mmr.h
SIGNATURES = {
    "mmr_create": (_i, [_i, _i, C.POINTER(_vp)]),
    "mmr_create_ex": (_i, [_i, _i, _u64, C.POINTER(_vp)]),
    "mmr_destroy": (_i, [_vp]),
    "mmr_last_error": (C.c_char_p, [_vp]),
    "mmr_status_string": (C.c_char_p, [_i]),
    "mmr_alloc_points": (_i, [_vp, _u64, _i, C.POINTER(_vp)]),
    "mmr_alloc_colors": (_i, [_vp, C.POINTER(_vp)]),
    "mmr_alloc_pingpong": (_i, [_vp, _u64, _i, C.POINTER(_vp), C.POINTER(_vp)]),
    "mmr_set_visible": (_i, [_vp, _i]),
    "mmr_get_visible": (_i, [_vp, C.POINTER(_i)]),
    "mmr_step_and_render_pingpong": (_i, [_vp, _vp]),
    "mmr_alloc_indexed_colors": (_i, [_vp, _u32, C.POINTER(_vp), C.POINTER(_vp)]),
    "mmr_alloc_nbody": (_i, [_vp, C.POINTER(_vp), C.POINTER(_vp)]),
    "mmr_nbody_step_and_render": (_i, [_vp, _f, _f, _f, _vp]),
    "mmr_set_camera": (_i, [_vp, _d3, _d3, _d3, _d, _d, _d]),
    "mmr_set_matrix": (_i, [_vp, _f16, _f, _f]),
    "mmr_get_matrix": (_i, [_vp, _f16]),
    "mmr_set_sim": (_i, [_vp, _u64, _u32, _f, _u32]),
    "mmr_set_style": (_i, [_vp, _u32, _u32]),
    "mmr_set_marker": (_i, [_vp, _f]),
    "mmr_set_launch": (_i, [_vp, _i, _i, _i]),
    "mmr_step_and_render": (_i, [_vp, _vp]),
    "mmr_displace": (_i, [_vp, _vp]),
    "mmr_render": (_i, [_vp, _vp]),
    "mmr_step_and_render_roundtrip": (_i, [_vp, _vp, _i]),
    "mmr_frame_ptr": (_i, [_vp, C.POINTER(_vp), C.POINTER(_vp)]),
    "mmr_get_step": (_i, [_vp, C.POINTER(_u32)]),
    "mmr_last_frame_kernels": (_i, [_vp, C.POINTER(_i)]),
    "mmr_frame_kernel_ms": (_i, [_vp, _u32, C.POINTER(_f), C.POINTER(_f)]),
    "mmr_set_depth_bound_split": (_i, [_vp, _i]),
    "mmr_set_timing": (_i, [_vp, _i]),
    "mmr_check_device": (_i, [_vp]),
    "mmr_selftest_bounded_wait": (_i, [_vp, C.c_longlong, _vp]),
    "mmr_last_kernel_ms": (_i, [_vp, C.POINTER(_f), C.POINTER(_f)]),
    "mmr_device_bytes": (_i, [_vp, C.POINTER(_u64)]),
    "mmr_alloc_host_mirror": (_i, [_vp, C.POINTER(_vp)]),
    "mmr_mirror_frame": (_i, [_vp, _vp]),
    "mmr_mirror_bytes": (_i, [_vp, C.POINTER(_u64)]),
}



class CloudDesc(C.Structure):
    """mmr_cloud_desc (include/mmr.h)."""
    _fields_ = [("n", C.c_uint64), ("width", C.c_int), ("height", C.c_int), ("seed", C.c_uint64),
                ("cloud", C.c_uint32), ("amplitude", C.c_float), ("color", C.c_uint32),
                ("background", C.c_uint32)]


SIGNATURES.update({
    "mmr_batch_create": (_i, [_i, C.POINTER(CloudDesc), _i, _i, _u64, C.POINTER(_vp)]),
    "mmr_batch_destroy": (_i, [_vp]),
    "mmr_batch_last_error": (C.c_char_p, [_vp]),
    "mmr_batch_points": (_i, [_vp, _i, C.POINTER(_vp)]),
    "mmr_batch_set_camera": (_i, [_vp, _i, _i, _d3, _d3, _d3, _d, _d, _d]),
    "mmr_batch_set_launch": (_i, [_vp, _i, _i, _i]),
    "mmr_batch_step_and_render": (_i, [_vp, _vp]),
    "mmr_batch_run_graph": (_i, [_vp, _i, _vp]),
    "mmr_batch_autotune": (_i, [_vp, _vp, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_f)]),
    "mmr_batch_frame_ptr": (_i, [_vp, _i, C.POINTER(_vp), C.POINTER(_vp)]),
    "mmr_batch_frames": (_i, [_vp, C.POINTER(_u32)]),
    "mmr_batch_check_device": (_i, [_vp]),
    "mmr_batch_step_and_render_roundtrip": (_i, [_vp, _vp, _i]),
    "mmr_batch_selftest_bounded_wait": (_i, [_vp, _u32, _vp]),
    "mmr_batch_device_bytes": (_i, [_vp, C.POINTER(_u64)]),
})

SIGNATURES.update({
    "mmr_serve_create": (_i, [_u64, _i, _u64, _u32, _f, _u64, C.POINTER(_vp)]),
    "mmr_serve_destroy": (_i, [_vp]),
    "mmr_serve_last_error": (C.c_char_p, [_vp]),
    "mmr_serve_shared_points": (_i, [_vp, C.POINTER(_vp)]),
    "mmr_serve_set_shared_color": (_i, [_vp, _u32]),
    "mmr_serve_add_viewer": (_i, [_vp, _u64, _i, _i, _u64, _u32, _f, _u32, _u32, C.POINTER(_i)]),
    "mmr_serve_viewer_points": (_i, [_vp, _i, C.POINTER(_vp)]),
    "mmr_serve_set_camera": (_i, [_vp, _i, _d3, _d3, _d3, _d, _d, _d]),
    "mmr_serve_remove_viewer": (_i, [_vp, _i]),
    "mmr_serve_tick": (_i, [_vp, _vp]),
    "mmr_serve_tick_roundtrip": (_i, [_vp, _vp]),
    "mmr_serve_frame_ptr": (_i, [_vp, _i, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_u32)]),
    "mmr_serve_status": (_i, [_vp, C.POINTER(_u32), C.POINTER(_i), C.POINTER(_u64)]),
    "mmr_serve_set_timing": (_i, [_vp, _i]),
    "mmr_serve_last_tick_ms": (_i, [_vp, C.POINTER(_f)]),
})
SIGNATURES["mmr_render_static"] = (_i, [_vp, _u64, _i, _f16, _f, _f, _i, _i, _u32, _u32, _vp, _vp])
STATIC_MAX_PIXELS = 4194304

_lib = None


class MmrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def load() -> C.CDLL:
    """Load the in-tree libmmr.so (build it with paper_2504_20937_b300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmmr.so not built at {LIB_PATH}; run paper_2504_20937_b300/build.py")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int, ctx=None, batch=False, serve=False) -> None:
    if status != MMR_OK:
        lib = load()
        if serve:
            msg = lib.mmr_serve_last_error(ctx)
        elif batch:
            msg = lib.mmr_batch_last_error(ctx)
        else:
            msg = lib.mmr_last_error(ctx)
        raise MmrError(status, msg.decode() if msg else "")


def stream_handle(stream) -> int | None:
    """torch.cuda.Stream / raw handle / None -> cudaStream_t as an int."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None
