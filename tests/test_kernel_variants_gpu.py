"""Parity of the point-kernel variants with the oracle: the screen-tile
depth-bound passes and the warp-aggregated splat must give the frames of the
direct splat bit for bit (the per-pixel minimum does not depend on which
points are skipped early or in which order the rest arrive), for every
storage type, ragged sizes, frames whose sides are not multiples of the
8-pixel tile, persistent and one-thread-per-group grids, and every path that
renders (fused step, render after a separate displacement, the host round
trip, ping-pong buffers).  Frames of a run are compared one by one, so a
bound left over from an earlier frame would show."""
import numpy as np
import pytest

from paper_2504_20937_b300 import inputs

from ._harness import fixed_eye, gpu_run, oracle_run, orbit
from .test_parity_gpu import _assert_same

pytestmark = pytest.mark.gpu

VARIANTS = {"depth_bound": 2, "warp_agg": 3}


def _kept_same(g, o, frames):
    for f in frames:
        assert np.array_equal(g[3][f][0], o[3][f][0]), f"keys frame {f}"
        assert np.array_equal(g[3][f][1], o[3][f][1]), f"rgba frame {f}"


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("W,H", [(96, 64), (61, 37)])
def test_dense_clusters_every_frame(variant, dtype, W, H):
    """300k points in three tight clusters: about 50 to 130 points per pixel,
    so most tiles get a bound and most points of the second pass are
    dropped.  Five orbiting frames, each compared whole."""
    n = 300_001
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 31, components=3, sigma=0.02), dtype)
    keep = set(range(5))
    args = (stored, dtype, W, H, 11, 5e-4, 5, orbit(9.0))
    g = gpu_run(*args, launch=(64, 0, VARIANTS[variant]), keep_every=keep)
    o = oracle_run(*args, keep_every=keep)
    _assert_same(g, o, f"{variant} {dtype} {W}x{H}")
    _kept_same(g, o, keep)


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("n", [1, 7, 9, 63, 1000, 65537])
def test_ragged_sizes(variant, dtype, n):
    """Counts below one first-pass group, ragged tails, a frame of 37 x 23."""
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 200 + n, components=2, sigma=0.03), dtype)
    args = (stored, dtype, 37, 23, 7, 2e-3, 3, orbit(5.0))
    _assert_same(gpu_run(*args, launch=(64, 0, VARIANTS[variant])), oracle_run(*args), f"{variant} {dtype} n={n}")


@pytest.mark.parametrize("launch", [(32, 0, 2), (1024, 0, 2), (256, 4, 2), (64, 1, 2), (128, 8, 3), (512, 0, 3)])
def test_launch_shapes(launch):
    """Persistent grids (the FP32 prefetch path starting at the second pass's
    first group) and one thread per group."""
    n = 250_003
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 33, components=4, sigma=0.03), "f32")
    args = (stored, "f32", 120, 80, 3, 1e-3, 3, orbit(10.0))
    _assert_same(gpu_run(*args, launch=launch), oracle_run(*args), f"launch {launch}")


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("mode", ["split", "roundtrip"])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_render_paths(variant, mode, dtype):
    """Render-only launches: after a separate displacement, and from the host
    round trip's device copy."""
    n = 150_000
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 34, components=2, sigma=0.02), dtype)
    args = (stored, dtype, 80, 48, 5, 1e-3, 3, orbit(4.0))
    _assert_same(gpu_run(*args, launch=(64, 0, VARIANTS[variant]), mode=mode), oracle_run(*args),
                 f"{variant} {mode} {dtype}")


def test_default_kernel_and_launch_counts():
    """The default kernel for 1-px points is the direct splat (two launches
    per frame); depth bounds chosen explicitly take four."""
    import torch

    from paper_2504_20937_b300.api import Context
    from ._harness import CENTRE, UP, upload
    cases = [((1 << 20), 256, 128, 2), ((1 << 20), 1024, 512, 2), (100_000, 16, 16, 2)]
    for n, W, H, want in cases:
        stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 35, components=4, sigma=0.02), "f32")
        with Context(W, H) as ctx:
            ctx.alloc_points(n, "f32")
            upload(ctx, stored)
            ctx.set_sim(3, 0, 5e-4, 0)
            ctx.set_camera((0.5, 0.5, 2.5), CENTRE, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render()
            torch.cuda.synchronize()
            assert ctx.last_frame_kernels() == want, (n, W, H)
            ctx.set_launch(64, 0, "depth_bound")
            ctx.step_and_render()
            assert ctx.last_frame_kernels() == 4
    # first-pass shares of one half to 1/1024, every frame against the oracle
    n = 1 << 20
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 36, components=4, sigma=0.02), "f32")
    keep = {0, 1, 2}
    args = (stored, "f32", 256, 128, 3, 5e-4, 3, fixed_eye)
    o = oracle_run(*args, keep_every=keep)
    for shift in (1, 5, 10):
        g = gpu_run(*args, keep_every=keep, launch=(64, 0, 2), bound_shift=shift)
        _assert_same(g, o, f"shift {shift}")
        _kept_same(g, o, keep)


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_pingpong(variant):
    import torch

    from paper_2504_20937_b300.api import Context
    import oracle
    from ._harness import CENTRE, UP
    n, W, H, frames = 200_000, 64, 48, 4
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 37, components=2, sigma=0.02), "f32")
    with Context(W, H) as ctx:
        a, b = ctx.alloc_pingpong(n, "f32")
        a.copy_(torch.from_numpy(stored))
        ctx.set_launch(64, 0, VARIANTS[variant])
        ctx.set_sim(4, 0, 1e-3, 0)
        for f in range(frames):
            ctx.set_camera(inputs.orbit_eye(f, 6.0), CENTRE, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render_pingpong()
        torch.cuda.synchronize()
        gpos = ctx.points.cpu().numpy()
        gkeys = ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64)
    pos = stored.copy()
    for f in range(frames):
        oracle.displace_f32(pos, 4, 0, f, np.float32(1e-3))
    M = oracle.camera_f32(inputs.orbit_eye(frames - 1, 6.0), CENTRE, UP, 60.0, W / H, 0.1, 100.0)
    keys, _ = oracle.render(pos, "f32", M, W, H, np.float32(0.1), np.float32(100.0))
    assert np.array_equal(gpos, pos) and np.array_equal(gkeys, keys)


def _disc_run(stored, dtype, W, H, radius, frames, kernel, seed=17, a=1e-3):
    import torch

    from paper_2504_20937_b300.api import Context
    tview = np.float32 if dtype == "f32" else np.int16
    eye = orbit(6.0)
    kept = []
    with Context(W, H) as ctx:
        ctx.alloc_points(stored.shape[0], dtype).copy_(torch.from_numpy(stored.view(tview)))
        ctx.set_sim(seed, 0, a, 0)
        ctx.set_marker(radius)
        if kernel is not None:
            ctx.set_launch(64, 0, kernel)
        for f in range(frames):
            ctx.set_camera(eye(f), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
            ctx.step_and_render()
            torch.cuda.synchronize()
            kept.append(ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64).copy())
        launches = ctx.last_frame_kernels()
        gpos = ctx.points.cpu().numpy().view(stored.dtype)
    return gpos, kept, launches


def _disc_oracle(stored, dtype, W, H, radius, frames, seed=17, a=1e-3):
    import oracle
    eye = orbit(6.0)
    pos = stored.copy()
    kept = []
    for f in range(frames):
        oracle.displace(pos, dtype, seed, 0, f, np.float32(a))
        M = oracle.camera_f32(eye(f), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, W / H, 0.1, 100.0)
        keys, _ = oracle.render_disc(oracle.from_storage(pos, dtype), M, W, H, np.float32(0.1), np.float32(100.0),
                                     np.float32(radius))
        kept.append(keys)
    return pos, kept


@pytest.mark.parametrize("dtype,radius", [("f32", 1.0), ("f32", 2.5), ("f32", 6.0), ("f32", 16.0), ("f16", 4.0),
                                          ("bf16", 3.0)])
def test_disc_markers_with_tile_bounds(dtype, radius):
    """Disc markers culled against 32x32-tile depth bounds: every frame of a
    run equal to the oracle's.  Dense clusters on a frame whose sides are not
    multiples of 32, so most later discs are skipped and edge tiles are
    partial."""
    n, W, H, frames = 120_007, 100, 70, 3
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 38, components=3, sigma=0.05), dtype)
    gpos, gkeys, launches = _disc_run(stored, dtype, W, H, radius, frames, "depth_bound")
    pos, keys = _disc_oracle(stored, dtype, W, H, radius, frames)
    assert launches == 4
    assert np.array_equal(gpos.view(np.uint8), pos.view(np.uint8))
    for f in range(frames):
        assert np.array_equal(gkeys[f], keys[f]), f"frame {f}: {np.count_nonzero(gkeys[f] != keys[f])} pixels differ"


def test_disc_markers_auto_choice():
    """The default kernel bounds discs when n pi r^2 >= 64 W H (and n >= 2^20),
    with a first pass of 1/16 from 1024 discs per pixel."""
    n = 1 << 20
    stored = inputs.encode(inputs.uniform_cloud(n, 39), "f32")
    # 2^20 pi r^2 / (W H): 20 discs per pixel (direct), 181 and 1448 (bounded)
    for radius, W, H, want in ((0.5, 256, 160, 2), (1.5, 256, 160, 4), (4.0, 256, 160, 4)):
        gpos, gkeys, launches = _disc_run(stored, "f32", W, H, radius, 2, None)
        assert launches == want, radius
        pos, keys = _disc_oracle(stored, "f32", W, H, radius, 2)
        assert np.array_equal(gpos, pos) and np.array_equal(gkeys[1], keys[1]), radius


@pytest.mark.parametrize("W,H", [(1, 1), (7, 5), (32768, 32), (33, 4097)])
def test_depth_bound_frame_shapes(W, H):
    """Frames of one pixel, smaller than one tile, one tile row 4096 tiles
    wide, and 4097 rows: every frame against the oracle, with the first pass
    taking half the points so many tiles get bounds."""
    n = 120_001
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 42, components=3, sigma=0.03), "f32")
    keep = {0, 1}
    args = (stored, "f32", W, H, 5, 1e-3, 2, orbit(4.0))
    g = gpu_run(*args, launch=(64, 0, 2), keep_every=keep, bound_shift=1)
    o = oracle_run(*args, keep_every=keep)
    _assert_same(g, o, f"{W}x{H}")
    _kept_same(g, o, keep)


@pytest.mark.parametrize("dtype,radius,W,H", [("f32", 64.0, 200, 150), ("f32", 24.0, 1, 300), ("bf16", 8.0, 301, 7),
                                              ("f16", 0.5, 90, 60)])
def test_disc_tile_bounds_edges(dtype, radius, W, H):
    """Disc markers with tile bounds where discs reach far past the frame
    (r = 64: candidate boxes of 129 px over up to 5x5 tiles), a frame one
    pixel wide, one seven rows high, and the smallest radius."""
    n = 60_007
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 43, components=2, sigma=0.1), dtype)
    gpos, gkeys, launches = _disc_run(stored, dtype, W, H, radius, 2, "depth_bound")
    pos, keys = _disc_oracle(stored, dtype, W, H, radius, 2)
    assert launches == 4
    assert np.array_equal(gpos.view(np.uint8), pos.view(np.uint8))
    for f in range(2):
        assert np.array_equal(gkeys[f], keys[f]), f"frame {f}: {np.count_nonzero(gkeys[f] != keys[f])} pixels differ"
