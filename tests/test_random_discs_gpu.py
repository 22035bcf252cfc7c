"""A sweep of seeded random disc-marker configurations against the oracle,
bit for bit (positions and every frame's keys): radius, cloud, storage type,
frame size, camera, amplitude, the kernel (direct, tile depth bounds, or the
library's choice) and the first pass's share of the points are drawn
independently.  Cloud sizes are capped so that the oracle's candidate boxes
stay below about 2e7 pixel tests a frame."""
import numpy as np
import pytest

import oracle
from paper_2504_20937_b300 import inputs

pytestmark = pytest.mark.gpu

COUNT = 100


def _config(k):
    rng = np.random.default_rng(30_000 + k)
    radius = float(rng.choice([0.5, 0.7, 1.0, 1.5, 2.0, 3.3, 5.0, 8.0, 16.0, 33.0, 64.0]))
    cap = int(2e7 / (2 * radius + 2) ** 2)
    n = int(np.exp(rng.uniform(0, np.log(max(2, min(200_000, cap))))))
    dtype = ["f32", "f16", "bf16"][rng.integers(3)]
    pos = inputs.uniform_cloud(n, 40_000 + k) if rng.random() < 0.4 else \
        inputs.gaussian_mixture_cloud(n, 40_000 + k, components=int(rng.integers(1, 6)), sigma=float(rng.uniform(0.01, 0.08)))
    W, H = int(rng.integers(1, 320)), int(rng.integers(1, 240))
    eye = inputs.orbit_eye(0, 0.0, float(rng.uniform(0.3, 4.0)), (0.5, 0.5, 0.5), float(rng.uniform(-1.0, 1.0)),
                           float(rng.uniform(0, 360)))
    step_deg = float(rng.uniform(-20, 20))
    kernel = [None, "grid", "depth_bound"][rng.integers(3)]
    split = int(rng.integers(0, 6))
    frames = int(rng.integers(1, 4))
    amplitude = float([0.0, 1e-4, 1e-2][rng.integers(3)])
    return dict(radius=radius, n=n, dtype=dtype, stored=inputs.encode(pos, dtype), W=W, H=H, eye=eye,
                step_deg=step_deg, kernel=kernel, split=split, frames=frames, amplitude=amplitude,
                seed=int(rng.integers(0, 2**31)))


@pytest.mark.parametrize("k", range(COUNT))
def test_random_disc_configuration(k):
    import torch

    from paper_2504_20937_b300.api import Context
    from ._harness import CENTRE, UP
    c = _config(k)
    desc = {key: v for key, v in c.items() if key != "stored"}
    stored, dtype, W, H = c["stored"], c["dtype"], c["W"], c["H"]

    def eye(f):
        return inputs.orbit_eye(f, c["step_deg"], float(np.linalg.norm(np.subtract(c["eye"], CENTRE))), CENTRE,
                                0.0, 0.0) if f else c["eye"]

    tview = np.float32 if dtype == "f32" else np.int16
    got = []
    with Context(W, H) as ctx:
        ctx.alloc_points(stored.shape[0], dtype).copy_(torch.from_numpy(stored.view(tview)))
        ctx.set_sim(c["seed"], 0, c["amplitude"], 0)
        ctx.set_marker(c["radius"])
        if c["kernel"] is not None:
            ctx.set_launch(64, 0, c["kernel"])
        if c["split"]:
            ctx.set_depth_bound_split(c["split"])
        for f in range(c["frames"]):
            ctx.set_camera(eye(f), CENTRE, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render()
            torch.cuda.synchronize()
            got.append(ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64).copy())
        gpos = ctx.points.cpu().numpy().view(stored.dtype)
    pos = stored.copy()
    for f in range(c["frames"]):
        oracle.displace(pos, dtype, c["seed"], 0, f, np.float32(c["amplitude"]))
        M = oracle.camera_f32(eye(f), CENTRE, UP, 60.0, W / H, 0.1, 100.0)
        keys, _ = oracle.render_disc(oracle.from_storage(pos, dtype), M, W, H, np.float32(0.1), np.float32(100.0),
                                     np.float32(c["radius"]))
        assert np.array_equal(got[f], keys), f"keys of frame {f}: {desc}"
    assert np.array_equal(gpos, pos), f"positions: {desc}"
