"""A sweep of seeded random batches against the oracle, cloud by cloud, bit
for bit (positions, keys, RGBA after the last frame): the number of clouds,
each cloud's size, shape, frame size, camera, colours and displacement, the
storage type, the launch shape (threads, CTAs per SM, groups per item), the
number of frames and how they run (direct launches, graph replays, the host
round trip, or a mix) are drawn independently."""
import numpy as np
import pytest

from paper_2504_20937_b300 import inputs

from .test_batch_gpu import _check_all, _eye_fn, _set_cameras, _upload

pytestmark = pytest.mark.gpu

COUNT = 30


def _config(k):
    rng = np.random.default_rng(50_000 + k)
    dtype = ["f32", "f16", "bf16"][rng.integers(3)]
    count = int(rng.integers(1, 24))
    clouds, stored, eyes = [], [], []
    for i in range(count):
        n = int(np.exp(rng.uniform(0, np.log(60_000))))
        W, H = int(rng.integers(1, 200)), int(rng.integers(1, 160))
        pos = inputs.uniform_cloud(n, 60_000 + 100 * k + i) if rng.random() < 0.5 else \
            inputs.gaussian_mixture_cloud(n, 60_000 + 100 * k + i, components=4, sigma=0.05)
        stored.append(inputs.encode(pos, dtype))
        clouds.append(dict(n=n, width=W, height=H, seed=int(rng.integers(0, 2**31)), cloud=i,
                           amplitude=float([0.0, 1e-4, 1e-3][rng.integers(3)]),
                           color=int(rng.integers(0, 2**32)), background=int(rng.integers(0, 2**32))))
        eyes.append(_eye_fn(float(rng.uniform(0.3, 4.0)), float(rng.uniform(-1.0, 1.0)),
                            float(rng.uniform(0, 360)), float(rng.uniform(-15, 15))))
    threads = int(rng.choice([32, 64, 128, 256, 512]))
    ctas = int(rng.integers(0, 9))
    groups = int(rng.choice([1, 7, 64, 256, 1024, 4096]))
    frames = int(rng.integers(1, 6))
    runs = [["direct", "graph", "roundtrip"][rng.integers(3)] for _ in range(frames)]
    return dtype, clouds, stored, eyes, (threads, ctas, groups), frames, runs


@pytest.mark.parametrize("k", range(COUNT))
def test_random_batch(k):
    from paper_2504_20937_b300.api import Batch
    dtype, clouds, stored, eyes, launch, frames, runs = _config(k)
    with Batch(clouds, dtype, camera_slots=frames) as b:
        _upload(b, stored)
        _set_cameras(b, eyes, frames)
        b.set_launch(*launch)
        for how in runs:
            if how == "graph":
                b.run_graph(1)
            elif how == "roundtrip":
                b.step_and_render_roundtrip()
            else:
                b.step_and_render()
        assert b.frames == frames
        _check_all(b, clouds, stored, eyes, dtype, frames)
