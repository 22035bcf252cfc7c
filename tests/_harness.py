"""Helpers that drive the CUDA path through the C ABI and the oracle on the
same seeded inputs.  The two sides share only the inputs module."""
from __future__ import annotations

import numpy as np
import torch

from paper_2504_20937_b300 import inputs

UP = (0.0, 1.0, 0.0)
CENTRE = (0.5, 0.5, 0.5)


def upload(ctx, stored: np.ndarray):
    """Write host positions (float32[n,3] or uint16[n,3]) into ctx's device buffer."""
    view = ctx.points
    src = torch.from_numpy(np.ascontiguousarray(stored).view(np.float32 if stored.dtype == np.float32
                                                               else np.int16))
    view.copy_(src.reshape(view.shape))
    torch.cuda.synchronize()


def download_points(ctx) -> np.ndarray:
    torch.cuda.synchronize()
    host = ctx.points.cpu().numpy()
    return host if ctx.dtype == "f32" else host.view(np.uint16)


def download_frame(ctx):
    torch.cuda.synchronize()
    keys = ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64)
    rgba = ctx.frame_rgba().cpu().numpy().reshape(-1).view(np.uint32)
    return keys, rgba


def gpu_run(stored, dtype, W, H, seed, amplitude, frames, eye_fn, fovy=60.0, znear=0.1, zfar=100.0,
            cloud=0, first_step=0, launch=None, colors=None, color=0xFFFFFFFF, background=0,
            mode="fused", keep_every=None, bound_shift=None):
    """Run `frames` frames on the GPU; returns (positions, keys, rgba) of the
    last frame, plus the per-frame (keys, rgba) of the frames in keep_every."""
    from paper_2504_20937_b300.api import Context
    n = stored.shape[0]
    kept = {}
    with Context(W, H) as ctx:
        ctx.alloc_points(n, dtype)
        upload(ctx, stored)
        if colors is not None:
            cv = ctx.alloc_colors()
            cv.copy_(torch.from_numpy(np.ascontiguousarray(colors, np.uint32).view(np.int32)))
        if launch:
            ctx.set_launch(*launch)
        if bound_shift is not None:
            ctx.set_depth_bound_split(bound_shift)
        ctx.set_sim(seed, cloud, amplitude, first_step)
        ctx.set_style(color, background)
        for f in range(frames):
            ctx.set_camera(eye_fn(f), CENTRE, UP, fovy, znear, zfar)
            if mode == "fused":
                ctx.step_and_render()
            elif mode == "split":
                ctx.displace()
                ctx.render()
            elif mode == "roundtrip":
                ctx.step_and_render_roundtrip(pinned=True)
            elif mode == "roundtrip_pageable":
                ctx.step_and_render_roundtrip(pinned=False)
            else:
                raise ValueError(mode)
            if keep_every and f in keep_every:
                kept[f] = download_frame(ctx)
        pos = download_points(ctx)
        keys, rgba = download_frame(ctx)
        step = ctx.step
    assert step == first_step + frames
    return pos, keys, rgba, kept


def oracle_run(stored, dtype, W, H, seed, amplitude, frames, eye_fn, fovy=60.0, znear=0.1, zfar=100.0,
               cloud=0, first_step=0, colors=None, color=0xFFFFFFFF, background=0, keep_every=None):
    import oracle
    pos = np.array(stored, copy=True)
    kept = {}
    keys = rgba = None
    for f in range(frames):
        oracle.displace(pos, dtype, seed, cloud, first_step + f, np.float32(amplitude))
        need = (f == frames - 1) or (keep_every and f in keep_every)
        if need:
            M = oracle.camera_f32(eye_fn(f), CENTRE, UP, fovy, W / H, znear, zfar)
            keys, rgba = oracle.render(pos, dtype, M, W, H, np.float32(znear), np.float32(zfar),
                                       colors, color, background)
            if keep_every and f in keep_every:
                kept[f] = (keys, rgba)
    return pos, keys, rgba, kept


def fixed_eye(_f):
    return (0.5, 0.5, 2.5)


def orbit(deg):
    return lambda f: inputs.orbit_eye(f, deg)
