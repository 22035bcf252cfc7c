"""The OpenMP CPU baseline (oracle/mmr_cpu_omp.c) against the single-threaded
oracle: the same positions, depth-id keys and RGBA, bit for bit, for any
number of threads, including frames where thousands of points contend for
each pixel (the compare-and-swap minimum must keep the smallest key)."""
import numpy as np
import pytest

import oracle
from paper_2504_20937_b300 import inputs

from ._harness import CENTRE, UP


def _oracle_frames(pos, seed, a, frames, eyes, W, H, color, background):
    keys = rgba = None
    for f in range(frames):
        oracle.displace_f32(pos, seed, 0, f, a)
        M = oracle.camera_f32(eyes(f), CENTRE, UP, 60.0, W / H, 0.1, 100.0)
        keys, rgba = oracle.render(pos, "f32", M, W, H, np.float32(0.1), np.float32(100.0),
                                   None, color, background)
    return keys, rgba


@pytest.mark.parametrize("threads", [1, 3, 8])
@pytest.mark.parametrize("n,W,H", [(50_001, 160, 90), (20_000, 4, 3), (1, 8, 8), (7, 1, 1)])
def test_omp_frames_equal_oracle(threads, n, W, H):
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 77, components=4, sigma=0.05), "f32")
    seed, a, frames = 9, 1e-3, 3
    color, background = 0xFF00FF00, 0x11
    eyes = lambda f: inputs.orbit_eye(f, 5.0)
    want_pos = stored.copy()
    want_keys, want_rgba = _oracle_frames(want_pos, seed, a, frames, eyes, W, H, color, background)
    pos = stored.copy()
    for f in range(frames):
        M = oracle.camera_f32(eyes(f), CENTRE, UP, 60.0, W / H, 0.1, 100.0)
        keys, rgba, used = oracle.cpu_omp_frame_f32(pos, seed, 0, f, a, M, W, H, 0.1, 100.0, color, background,
                                                    threads=threads)
        assert used == threads
    assert np.array_equal(pos.view(np.uint32), want_pos.view(np.uint32))
    assert np.array_equal(keys, want_keys)
    assert np.array_equal(rgba, want_rgba)


def test_omp_default_threads_is_positive():
    assert oracle.cpu_omp_threads(0) >= 1
    assert oracle.cpu_omp_threads(5) == 5
