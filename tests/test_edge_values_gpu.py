"""Inputs a caller may write that the benchmark never does, against the
oracle bit for bit (positions, depth-id keys and RGBA): coordinates that are
NaN, infinite, huge, negative, above 1 or subnormal, in every storage type,
with and without displacement (the clamp applies either way); and a cloud
whose points all sit on the same spot, so every point contends for one
pixel and the smallest id must win."""
import numpy as np
import pytest

from paper_2504_20937_b300 import inputs

from ._harness import fixed_eye, gpu_run, oracle_run, orbit
from .test_parity_gpu import _assert_same

pytestmark = pytest.mark.gpu

SPECIAL_F32 = np.array([np.nan, np.inf, -np.inf, 3e38, -3e38, 2.0, -2.0, 1.0, 0.0, -0.0, 1.4e-45, -1.4e-45,
                        1.0 + 2**-23, -(2**-24)], np.float32)
# binary16 / bfloat16 bit patterns: NaN, +inf, -inf, largest finite, its negative, 2, -2, 1, +0, -0, smallest
# subnormal and its negative
SPECIAL_BITS = {
    "f16": [0x7E00, 0x7C00, 0xFC00, 0x7BFF, 0xFBFF, 0x4000, 0xC000, 0x3C00, 0x0000, 0x8000, 0x0001, 0x8001],
    "bf16": [0x7FC0, 0x7F80, 0xFF80, 0x7F7F, 0xFF7F, 0x4000, 0xC000, 0x3F80, 0x0000, 0x8000, 0x0001, 0x8001],
}


def _with_specials(dtype, n, seed):
    """A uniform cloud with special coordinates spread over it: whole special
    points, and single special coordinates in otherwise normal points, at the
    start, in the middle and in the ragged last group."""
    stored = inputs.encode(inputs.uniform_cloud(n, seed), dtype)
    flat = stored.reshape(-1)
    specials = SPECIAL_F32 if dtype == "f32" else np.array(SPECIAL_BITS[dtype], np.uint16)
    rng = np.random.default_rng(seed)
    k = len(specials)
    for j, v in enumerate(specials):
        stored[j] = v                                      # a whole special point at the start
        stored[n // 2 + j, j % 3] = v                      # one special coordinate in the middle
        flat[rng.integers(0, flat.size)] = v
    stored[n - 1, 0] = specials[0]                         # in the ragged last group
    stored[n - 2, 2] = specials[1]
    assert n % (4 if dtype == "f32" else 8) != 0 and n > 2 * k
    return stored


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("amplitude", [0.0, 1e-3])
def test_special_coordinates(dtype, amplitude):
    stored = _with_specials(dtype, 20_003, 95)
    keep = {0, 1, 2}
    args = (stored, dtype, 96, 64, 12, amplitude, 3, orbit(20.0))
    g = gpu_run(*args, keep_every=keep)
    o = oracle_run(*args, keep_every=keep)
    _assert_same(g, o, f"{dtype} a={amplitude}")
    for f in keep:
        assert np.array_equal(g[3][f][0], o[3][f][0]) and np.array_equal(g[3][f][1], o[3][f][1]), f


@pytest.mark.parametrize("amplitude", [0.0, 1e-7, 1e-5])
def test_all_points_on_one_spot(amplitude):
    """100,000 points at the cloud's centre: with no displacement they share
    one pixel and one depth, so id 0 wins; with tiny steps they spread over a
    few pixels and depths."""
    n = 100_000
    stored = np.full((n, 3), 0.5, np.float32)
    args = (stored, "f32", 64, 48, 13, amplitude, 2, fixed_eye)
    g, o = gpu_run(*args), oracle_run(*args)
    _assert_same(g, o, f"one spot a={amplitude}")
    keys = g[1]
    covered = keys[keys != np.uint64(2**64 - 1)]
    if amplitude == 0.0:
        assert covered.size == 1 and int(covered[0]) & 0xFFFFFFFF == 0


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_render_of_special_coordinates_without_displacement(dtype):
    """mmr_render projects the positions as the caller left them: NaN, infinite
    and huge coordinates must be culled or land where the oracle puts them,
    and never index memory outside the frame."""
    import oracle
    from paper_2504_20937_b300.api import Context
    from ._harness import CENTRE, UP, download_frame, upload
    stored = _with_specials(dtype, 20_003, 96)
    W, H = 80, 60
    # outside the cloud, inside it looking along -z, and from below one corner
    for eye, target in [((0.5, 0.5, 2.5), CENTRE), ((0.5, 0.5, 0.5), (0.5, 0.5, 0.0)), ((3.0, -2.0, 1.0), CENTRE)]:
        with Context(W, H) as ctx:
            ctx.alloc_points(stored.shape[0], dtype)
            upload(ctx, stored)
            ctx.set_camera(eye, target, UP, 60.0, 0.1, 100.0)
            ctx.render()
            keys, rgba = download_frame(ctx)
        M = oracle.camera_f32(eye, target, UP, 60.0, W / H, 0.1, 100.0)
        wk, wr = oracle.render(stored, dtype, M, W, H, np.float32(0.1), np.float32(100.0))
        assert np.array_equal(keys, wk), (dtype, eye)
        assert np.array_equal(rgba, wr), (dtype, eye)
