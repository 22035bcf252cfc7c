"""mmr_render_static: rendering without any device allocation.

Some callers cannot allocate device memory: a simulation living inside a
host program whose memory manager owns the GPU (every allocation must go
through its pool), or a real-time loop that must not allocate per frame
because an allocation can synchronise the device.  They pass their own
point buffer and RGBA output; the only scratch, the per-pixel depth-id
keys, is a fixed array inside the library.  These checks call the entry
point through the C ABI and compare its frames, bit for bit, with the
existing mmr_set_matrix + mmr_render path, on consecutive calls that share
the scratch array.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import _lib, inputs
from paper_2504_20937_b300.api import Context

pytestmark = pytest.mark.gpu

CEN = (0.5, 0.5, 0.5)
UP = (0.0, 1.0, 0.0)


def _matrix(eye, W, H, znear=0.1, zfar=100.0):
    return oracle.camera_f32(eye, CEN, UP, 60.0, W / H, znear, zfar).reshape(-1)


def _points_tensor(stored):
    src = torch.from_numpy(stored if stored.dtype == np.float32 else stored.view(np.int16))
    return src.to("cuda").contiguous()


def _render_existing(stored, dtype, M, W, H, color, background, znear=0.1, zfar=100.0):
    with Context(W, H) as ctx:
        ctx.alloc_points(stored.shape[0], dtype).copy_(_points_tensor(stored))
        ctx.set_matrix(M, znear, zfar)
        ctx.set_style(color, background)
        ctx.render()
        torch.cuda.synchronize()
        return ctx.frame_rgba().cpu().numpy().reshape(-1).view(np.uint32)


def _render_static(pts, n, dtype, M, W, H, color, background, out, znear=0.1, zfar=100.0, rgba_offset=0):
    lib = _lib.load()
    st = lib.mmr_render_static(pts.data_ptr(), n, _lib.DTYPE_CODE[dtype],
                               (C.c_float * 16)(*[float(v) for v in M]), znear, zfar, W, H, color, background,
                               out.data_ptr() + rgba_offset, torch.cuda.current_stream().cuda_stream)
    return st


def test_static_render_matches_existing_on_consecutive_calls():
    cases = [
        # (points, dtype, W, H, eye, colour, background, znear, zfar): each frame is smaller than
        # the one before it, so stale keys left in the shared scratch would show up in it
        (inputs.uniform_cloud(50_001, 71), "f32", 640, 360, (0.5, 0.5, 2.5), 0xFFFFFFFF, 0x00000000, 0.1, 100.0),
        (inputs.gaussian_mixture_cloud(80_000, 72, components=3, sigma=0.05), "f32", 200, 120,
         inputs.orbit_eye(40, 1.0), 0xFF00FF00, 0x11223344, 0.1, 100.0),
        # bfloat16 with a ragged count (n % 8 != 0) and a depth range that keeps only the slab
        # 1.75 < w < 2 of the cloud (w runs from 1.5 to 2.5 from this eye)
        (inputs.uniform_cloud(40_005, 75), "bf16", 160, 90, (0.5, 0.5, 2.5), 0xFF0000FF, 3, 1.75, 2.0),
        (inputs.uniform_cloud(30_007, 73), "f16", 2048, 2048, inputs.orbit_eye(90, 1.0), 0xFFABCDEF, 7,
         0.1, 100.0),
    ]
    for k, (pos64, dtype, W, H, eye, color, bg, znear, zfar) in enumerate(cases):
        stored = inputs.encode(pos64, dtype)
        M = _matrix(eye, W, H, znear, zfar)
        pts = _points_tensor(stored)
        out = torch.full((H * W,), -1, dtype=torch.int32, device="cuda")
        assert _render_static(pts, stored.shape[0], dtype, M, W, H, color, bg, out, znear, zfar) == 0, \
            _lib.load().mmr_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        want = _render_existing(stored, dtype, M, W, H, color, bg, znear, zfar)
        assert np.array_equal(got, want), f"call {k}: {np.count_nonzero(got != want)} pixels differ"
        assert np.count_nonzero(got == color) > 100
        # the point buffer is only read
        assert torch.equal(pts, _points_tensor(stored))


def test_static_render_rejects_bad_sizes_without_launching():
    lib = _lib.load()
    stored = inputs.encode(inputs.uniform_cloud(1000, 74), "f32")
    pts = _points_tensor(stored)
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    M = _matrix((0.5, 0.5, 2.5), 4, 4)
    too_wide = _lib.STATIC_MAX_PIXELS + 1
    assert _render_static(pts, 1000, "f32", M, too_wide, 1, 1, 0, out) == -1
    assert b"MMR_STATIC_MAX_PIXELS" in lib.mmr_last_error(None)
    assert _render_static(pts, 0, "f32", M, 4, 4, 1, 0, out) == -1
    misaligned = lib.mmr_render_static(pts.data_ptr() + 4, 10, 0, (C.c_float * 16)(*[float(v) for v in M]),
                                       0.1, 100.0, 4, 4, 1, 0, out.data_ptr(), None)
    assert misaligned == -1
    # an RGBA pointer that is not 4-byte aligned is refused before anything is launched
    assert _render_static(pts, 1000, "f32", M, 2, 2, 1, 0, out, rgba_offset=1) == -1
    assert b"dev_rgba" in lib.mmr_last_error(None)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0      # nothing was written
    # a frame of exactly the maximum size is accepted
    big = torch.empty(_lib.STATIC_MAX_PIXELS, dtype=torch.int32, device="cuda")
    assert _render_static(pts, 1000, "f32", _matrix((0.5, 0.5, 2.5), 2048, 2048), 2048, 2048, 1, 0, big) == 0
    torch.cuda.synchronize()
