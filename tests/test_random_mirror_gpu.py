"""A sweep of seeded random host-mirror scenarios against the oracle, bit for
bit: frame size, cloud, a sequence of views (in view, turned away, partly in
view), background changes, which frames the mirror is brought up to date
after, and the update stream (the rendering stream, or another of the default
or the highest priority) are drawn independently.  After every update that
the host waits for, the mirror must equal the oracle's frame."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.api import Context

from ._harness import CENTRE, UP, upload

pytestmark = pytest.mark.gpu

COUNT = 24
VIEWS = [((0.5, 0.5, 2.5), CENTRE), ((0.5, 0.5, -2.5), (0.5, 0.5, -5.0)), ((2.5, 0.5, 0.5), CENTRE),
         ((0.5, 0.5, 2.5), (1.4, 1.3, 0.5)), ((0.5, 2.6, 0.5), (0.5, 0.5, 0.6)), ((-1.2, 0.1, 1.9), CENTRE)]


def _scenario(k):
    rng = np.random.default_rng(90_000 + k)
    W, H = int(rng.integers(1, 300)), int(rng.integers(1, 200))
    n = int(rng.integers(1, 50_000))
    frames = int(rng.integers(2, 12))
    views = [VIEWS[int(v)] for v in rng.integers(0, len(VIEWS), frames)]
    backgrounds = []
    bg = 0
    for _ in range(frames):
        if rng.random() < 0.2:
            bg = int(rng.integers(0, 2**32))
        backgrounds.append(bg)
    update = rng.random(frames) < 0.6
    update[-1] = True
    wait = update & (rng.random(frames) < 0.6)
    wait[-1] = True
    stream_kind = ["same", "default", "highest"][int(rng.integers(3))]
    kind = "uniform" if rng.random() < 0.5 else "gmm"
    return dict(W=W, H=H, n=n, frames=frames, views=views, backgrounds=backgrounds, update=update, wait=wait,
                stream_kind=stream_kind, kind=kind, seed=int(rng.integers(0, 2**31)),
                amplitude=float([0.0, 1e-3, 1e-2][int(rng.integers(3))]))


@pytest.mark.parametrize("k", range(COUNT))
def test_random_mirror(k):
    c = _scenario(k)
    W, H = c["W"], c["H"]
    pos = inputs.uniform_cloud(c["n"], 91_000 + k) if c["kind"] == "uniform" else \
        inputs.gaussian_mixture_cloud(c["n"], 91_000 + k, components=3, sigma=0.04)
    stored = inputs.encode(pos, "f32")
    render = torch.cuda.Stream()
    if c["stream_kind"] == "same":
        side = render
    else:
        prio = torch.cuda.Stream.priority_range()[1] if c["stream_kind"] == "highest" else 0
        side = torch.cuda.Stream(priority=prio)
    want_pos = stored.copy()
    with Context(W, H) as ctx:
        ctx.alloc_points(c["n"], "f32")
        upload(ctx, stored)
        ctx.set_sim(c["seed"], 0, c["amplitude"], 0)
        mirror = ctx.alloc_host_mirror()
        for f in range(c["frames"]):
            eye, target = c["views"][f]
            ctx.set_style(0xFFFFFFFF, c["backgrounds"][f])
            ctx.set_camera(eye, target, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render(render)
            oracle.displace(want_pos, "f32", c["seed"], 0, f, np.float32(c["amplitude"]))
            if c["update"][f]:
                ctx.mirror_frame(side)
            if c["wait"][f]:
                side.synchronize()
                M = oracle.camera_f32(eye, target, UP, 60.0, W / H, 0.1, 100.0)
                _, want = oracle.render(want_pos, "f32", M, W, H, np.float32(0.1), np.float32(100.0), None,
                                        0xFFFFFFFF, c["backgrounds"][f])
                assert np.array_equal(mirror.reshape(-1), want), f"mirror after frame {f}: {c}"
        render.synchronize()
