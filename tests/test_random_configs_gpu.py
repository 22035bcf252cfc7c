"""A sweep of seeded random configurations against the oracle, bit for bit
(positions, and keys and RGBA of every frame): cloud size and shape, storage
type, frame size, camera (eye inside or outside the cloud, field of view,
depth range), colours (default or per point), displacement amplitude, number of frames, render
path, point-kernel variant and launch shape are all drawn independently, so
combinations that no hand-written case pairs up get run too.  The draws are
fixed by the seed: a failing configuration is reproduced by its index."""
import numpy as np
import pytest

from paper_2504_20937_b300 import inputs

from ._harness import gpu_run, oracle_run
from .test_parity_gpu import _assert_same

pytestmark = pytest.mark.gpu

COUNT = 160
KERNELS = [("grid", [(64, 0), (32, 0), (256, 0), (1024, 0), (64, 4), (128, 1)]),
           ("depth_bound", [(64, 0), (256, 2)]),
           ("warp_agg", [(64, 0), (512, 0)]),
           ("tma", [(128, 1), (256, 2), (512, 1)])]


def _config(k):
    rng = np.random.default_rng(10_000 + k)
    dtype = ["f32", "f16", "bf16"][rng.integers(3)]
    n = int(np.exp(rng.uniform(0, np.log(300_000))))
    if rng.random() < 0.5:
        pos = inputs.uniform_cloud(n, 20_000 + k)
    else:
        pos = inputs.gaussian_mixture_cloud(n, 20_000 + k, components=int(rng.integers(1, 8)),
                                            sigma=float(rng.uniform(0.005, 0.1)))
    W, H = int(rng.integers(1, 400)), int(rng.integers(1, 300))
    if rng.random() < 0.2:
        W, H = (W * 9, max(1, H // 9)) if rng.random() < 0.5 else (max(1, W // 9), H * 9)
    inside = rng.random() < 0.2
    radius = float(rng.uniform(0.05, 0.4)) if inside else float(rng.uniform(1.2, 6.0))
    elevation = float(rng.uniform(-1.2, 1.2))
    start = float(rng.uniform(0, 360))
    step = float(rng.uniform(-30, 30))
    fovy = float(rng.uniform(10, 120))
    znear = float(10 ** rng.uniform(-3, -0.5))
    zfar = float(znear * 10 ** rng.uniform(0.5, 4))
    if rng.random() < 0.7:
        zfar = max(zfar, radius + 2.0)          # mostly a far plane behind the cloud; otherwise it may cut it
    amplitude = float([0.0, 1e-5, 1e-3, 0.05][rng.integers(4)])
    frames = int(rng.integers(1, 5))
    color, background = int(rng.integers(0, 2**32)), int(rng.integers(0, 2**32))
    mode = ["fused", "split", "roundtrip"][rng.integers(3)]
    kernel, shapes = KERNELS[rng.integers(len(KERNELS))]
    threads, ctas = shapes[rng.integers(len(shapes))]

    def eye_fn(f):
        return inputs.orbit_eye(f, step, radius, (0.5, 0.5, 0.5), elevation, start)

    args = (inputs.encode(pos, dtype), dtype, W, H, int(rng.integers(0, 2**32)), amplitude, frames, eye_fn)
    kw = dict(fovy=fovy, znear=znear, zfar=zfar, cloud=int(rng.integers(0, 2**32)), color=color,
              background=background)
    if rng.random() < 0.3:
        kw["colors"] = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    desc = (f"#{k}: {dtype} n={n} {W}x{H} r={radius:.2f} fov={fovy:.0f} z=[{znear:.3g},{zfar:.3g}] a={amplitude} "
            f"frames={frames} {mode} {kernel} {threads}x{ctas}")
    return args, kw, mode, (threads, ctas, kernel), desc


@pytest.mark.parametrize("k", range(COUNT))
def test_random_configuration(k):
    args, kw, mode, launch, desc = _config(k)
    keep = set(range(args[6]))
    g = gpu_run(*args, **kw, launch=launch, mode=mode, keep_every=keep)
    o = oracle_run(*args, **kw, keep_every=keep)
    _assert_same(g, o, desc)
    for f in keep:
        assert np.array_equal(g[3][f][0], o[3][f][0]), f"keys of frame {f}, {desc}"
        assert np.array_equal(g[3][f][1], o[3][f][1]), f"rgba of frame {f}, {desc}"
