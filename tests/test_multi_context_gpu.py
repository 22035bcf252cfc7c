"""Several contexts in one process: frames of two contexts (different frame
sizes, storage types, kernels and cameras) interleaved on one stream, and on
two streams without synchronisation between them, each context's frames
against the oracle bit for bit.  Nothing a context keeps (depth-id buffers,
chunk tags, tile bounds, timing events, the host mirror) may leak into the
other."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.api import Context

from ._harness import CENTRE, UP, download_frame, download_points, upload

pytestmark = pytest.mark.gpu

SPECS = [dict(n=40_003, W=96, H=64, dtype="f32", kernel="grid", seed=1, eye=lambda f: inputs.orbit_eye(f, 9.0)),
         dict(n=25_001, W=61, H=37, dtype="f16", kernel="depth_bound", seed=2,
              eye=lambda f: inputs.orbit_eye(f, -7.0, 1.5, CENTRE, 0.4, 80.0))]


def _oracle(spec, stored, frames):
    pos = np.array(stored, copy=True)
    out = []
    for f in range(frames):
        oracle.displace(pos, spec["dtype"], spec["seed"], 0, f, np.float32(1e-3))
        M = oracle.camera_f32(spec["eye"](f), CENTRE, UP, 60.0, spec["W"] / spec["H"], 0.1, 100.0)
        out.append(oracle.render(pos, spec["dtype"], M, spec["W"], spec["H"], np.float32(0.1), np.float32(100.0)))
    return pos, out


@pytest.mark.parametrize("two_streams", [False, True])
def test_interleaved_contexts(two_streams):
    frames = 5
    stored = [inputs.encode(inputs.gaussian_mixture_cloud(s["n"], 80 + i, components=3, sigma=0.04), s["dtype"])
              for i, s in enumerate(SPECS)]
    want = [_oracle(s, st, frames) for s, st in zip(SPECS, stored)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()] if two_streams else [torch.cuda.current_stream()] * 2
    ctxs = [Context(s["W"], s["H"]) for s in SPECS]
    try:
        for ctx, s, st in zip(ctxs, SPECS, stored):
            ctx.alloc_points(s["n"], s["dtype"])
            upload(ctx, st)
            ctx.set_sim(s["seed"], 0, 1e-3, 0)
            ctx.set_launch(64, 0, s["kernel"])
            ctx.set_timing(True)
        ctxs[0].alloc_host_mirror()
        for f in range(frames):
            for i, (ctx, s) in enumerate(zip(ctxs, SPECS)):
                ctx.set_camera(s["eye"](f), CENTRE, UP, 60.0, 0.1, 100.0)
                ctx.step_and_render(streams[i])
            ctxs[0].mirror_frame(streams[1])
            for st in streams:
                st.synchronize()
            for i, ctx in enumerate(ctxs):
                keys, rgba = download_frame(ctx)
                assert np.array_equal(keys, want[i][1][f][0]), f"keys of context {i} frame {f}"
                assert np.array_equal(rgba, want[i][1][f][1]), f"rgba of context {i} frame {f}"
            mirror = ctxs[0].alloc_host_mirror()
            assert np.array_equal(mirror.reshape(-1), want[0][1][f][1]), f"mirror frame {f}"
        for i, ctx in enumerate(ctxs):
            assert np.array_equal(download_points(ctx), want[i][0]), f"positions of context {i}"
            assert ctx.frame_kernel_ms(0)[0] > 0.0
    finally:
        for ctx in ctxs:
            ctx.close()
