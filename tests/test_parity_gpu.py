"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP32 storage: positions, depth-id keys and RGBA must be bit-identical.
16-bit storage: bit-identical to the oracle replaying the same storage
rounding.  Sizes span several thread groups and blocks with ragged tails.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs

from ._harness import fixed_eye, gpu_run, oracle_run, orbit

pytestmark = pytest.mark.gpu


def _assert_same(gpu, orc, what=""):
    gpos, gkeys, grgba, _ = gpu
    opos, okeys, orgba, _ = orc
    assert gpos.dtype == opos.dtype
    np.testing.assert_array_equal(gpos.view(np.uint8), opos.view(np.uint8), err_msg=f"positions {what}")
    bad = np.nonzero(gkeys != okeys)[0]
    assert bad.size == 0, f"keys {what}: {bad.size} pixels differ, first {bad[:5]}"
    np.testing.assert_array_equal(grgba, orgba, err_msg=f"rgba {what}")


def test_pr1_reference_config_bit_exact():
    """65,536 uniform points (seed 0), 100 steps of a = 1e-3, 512 x 512,
    fixed camera at (0.5, 0.5, 2.5): final positions and frame bit-exact,
    plus frames 0, 1 and 50 along the way."""
    sc = inputs.PR1
    stored = inputs.encode(sc.positions(), "f32")
    keep = {0, 1, 50}
    g = gpu_run(stored, "f32", sc.W, sc.H, sc.philox_seed, sc.amplitude, sc.frames, fixed_eye, keep_every=keep)
    o = oracle_run(stored, "f32", sc.W, sc.H, sc.philox_seed, sc.amplitude, sc.frames, fixed_eye,
                   keep_every=keep)
    _assert_same(g, o, "PR1 final")
    for f in keep:
        assert np.array_equal(g[3][f][0], o[3][f][0]), f"keys frame {f}"
        assert np.array_equal(g[3][f][1], o[3][f][1]), f"rgba frame {f}"
    covered = (g[1] != oracle.EMPTY_KEY).sum()
    assert covered > 10_000                  # the cloud is actually visible


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("n", [1, 3, 4, 5, 7, 8, 9, 255, 1000, 4097, 65537])
def test_ragged_sizes_bit_exact(dtype, n):
    W, H = 37, 23                             # W*H = 851: not a multiple of 4
    stored = inputs.encode(inputs.uniform_cloud(n, 100 + n), dtype)
    args = (stored, dtype, W, H, 7, 2e-3, 3, orbit(5.0))
    _assert_same(gpu_run(*args), oracle_run(*args), f"{dtype} n={n}")


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_gaussian_cluster_contention_bit_exact(dtype):
    """Many points per pixel: 200k points in a 3-cluster mixture at 96 x 64."""
    n = 200_000
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 21, components=3, sigma=0.02), dtype)
    args = (stored, dtype, 96, 64, 9, 5e-4, 2, fixed_eye)
    _assert_same(gpu_run(*args), oracle_run(*args), dtype)


@pytest.mark.parametrize("launch", [(32, 0, 0), (128, 0, 0), (1024, 0, 0), (256, 1, 0), (64, 3, 0), (512, 8, 0),
                                    (128, 3, 1), (256, 4, 1), (512, 1, 1), (256, 2, 1)])
def test_launch_shape_does_not_change_results(launch):
    n = 70_001
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 22, components=4, sigma=0.05), "f32")
    args = (stored, "f32", 160, 90, 3, 1e-3, 3, orbit(10.0))
    _assert_same(gpu_run(*args, launch=launch), oracle_run(*args), f"launch {launch}")


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("launch", [(32, 0, 0), (1024, 0, 0), (256, 4, 0), (256, 2, 1), (128, 8, 1)])
def test_launch_shapes_16bit(launch, dtype):
    n = 33_333
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 27, components=4, sigma=0.05), dtype)
    args = (stored, dtype, 96, 72, 3, 1e-3, 3, orbit(7.0))
    _assert_same(gpu_run(*args, launch=launch), oracle_run(*args), f"{dtype} launch {launch}")


def test_launch_validation():
    from paper_2504_20937_b300.api import Context, MmrError
    with Context(16, 16) as ctx:
        with pytest.raises(MmrError, match="INVALID"):
            ctx.set_launch(64, 2, 1)         # TMA needs 128/256/512 threads
        with pytest.raises(MmrError, match="INVALID"):
            ctx.set_launch(256, 0, 1)        # and a persistent grid
        with pytest.raises(MmrError, match="INVALID"):
            ctx.set_launch(256, 0, 7)
        ctx.set_launch(256, 2, 1)
        ctx.check_device()


def test_camera_depth_range_validation_and_extremes():
    """Every camera keeps 2^-64 <= znear < zfar <= 2^64, the clip w range on
    which the kernels' perspective divide gives IEEE division's pixels; the
    ends of the range are allowed and render like the oracle."""
    from paper_2504_20937_b300.api import Batch, Context, MmrError, Server
    eye, centre, up = (0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0)
    bad = [(2.0 ** -65, 1.0), (1e-30, 1.0), (0.1, 2.0 ** 65), (0.1, 1e30), (0.0, 1.0), (1.0, 1.0)]
    with Context(16, 16) as ctx:
        for zn, zf in bad:
            with pytest.raises(MmrError, match="INVALID"):
                ctx.set_camera(eye, centre, up, 60.0, zn, zf)
            with pytest.raises(MmrError, match="INVALID"):
                ctx.set_matrix(np.eye(4, dtype=np.float32), zn, zf)
        ctx.set_camera(eye, centre, up, 60.0, 2.0 ** -64, 2.0 ** 64)
        ctx.set_matrix(np.eye(4, dtype=np.float32), 2.0 ** -64, 2.0 ** 64)
    with Batch([dict(n=100, width=8, height=8)]) as b:
        with pytest.raises(MmrError, match="INVALID"):
            b.set_camera(0, 0, eye, centre, up, 60.0, 1e-30, 1.0)
    with Server(1000) as s:
        v = s.add_viewer(10, 8, 8)
        with pytest.raises(MmrError, match="INVALID"):
            s.set_camera(v, eye, centre, up, 60.0, 0.1, 1e30)
    n = 20_001
    stored = inputs.encode(inputs.uniform_cloud(n, 41), "f32")
    for zn, zf in ((2.0 ** -64, 2.0 ** 64), (2.0 ** -64, 3.0), (2.0, 2.0 ** 64)):
        args = (stored, "f32", 120, 80, 6, 1e-3, 2, orbit(5.0))
        kw = dict(znear=zn, zfar=zf)
        _assert_same(gpu_run(*args, **kw), oracle_run(*args, **kw), f"depth range {zn}..{zf}")


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("mode", ["split", "roundtrip", "roundtrip_pageable"])
def test_split_and_roundtrip_paths_match(mode, dtype):
    """Displace and render as separate kernels (split), and through a host
    copy of the positions (round trip), on every storage type: 50,003 points
    leave a ragged last group of 3 points (groups of 4 in FP32, 8 in 16-bit)."""
    n = 50_003
    stored = inputs.encode(inputs.uniform_cloud(n, 23), dtype)
    args = (stored, dtype, 200, 120, 4, 1e-3, 4, orbit(3.0))
    _assert_same(gpu_run(*args, mode=mode), oracle_run(*args), f"{mode} {dtype}")


def test_storage_drift_against_fp64_reported():
    """Multi-frame drift of each storage type against the FP64 trajectory that
    starts from the same stored positions, reported at 1, 10 and 100 steps
    (2^18 uniform points, a = 5e-4 as in the 2^22-point orbit).  Gated only by
    the worst case: both sides draw the same offsets and the clamp cannot
    enlarge a difference, so each step adds at most the storage rounding of a
    value in [0, 1] (h: half an ulp below 1, 2^-12 binary16, 2^-9 bfloat16, 0
    FP32) plus the FP32 rounding of p + d and of d (< 2^-23): after T steps
    |delta| <= T (h + 2^-23)."""
    n, a, seed = 1 << 18, 5e-4, 12
    pos0 = inputs.uniform_cloud(n, 41)
    half_ulp = {"f32": 0.0, "f16": 2.0**-12, "bf16": 2.0**-9}
    report = {}
    for dtype in ("f32", "f16", "bf16"):
        stored = inputs.encode(pos0, dtype)
        p64 = oracle.from_storage(stored, dtype).astype(np.float64)
        done, report[dtype] = 0, {}
        for T in (1, 10, 100):
            while done < T:
                oracle.displace_f64(p64, seed, 0, done, float(np.float32(a)))
                done += 1
            g = gpu_run(stored, dtype, 64, 64, seed, a, T, fixed_eye)
            got = oracle.from_storage(g[0], dtype).astype(np.float64)
            d = np.abs(got - p64)
            report[dtype][T] = {"max_abs": float(d.max()), "rms_abs": float(np.sqrt(np.mean(d * d)))}
            assert d.max() <= T * (half_ulp[dtype] + 2.0**-23), (dtype, T, float(d.max()))
    print("storage drift against the FP64 trajectory:", report)


def test_colour_buffer_and_style():
    n = 30_000
    stored = inputs.encode(inputs.uniform_cloud(n, 24), "f32")
    colors = np.random.default_rng(0).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    args = (stored, "f32", 128, 128, 5, 1e-3, 2, fixed_eye)
    kw = dict(colors=colors, background=0x12345678)
    g = gpu_run(*args, **kw)
    _assert_same(g, oracle_run(*args, **kw), "colours")
    kw = dict(color=0xFF00FF00, background=0x0000FF00)
    _assert_same(gpu_run(*args, **kw), oracle_run(*args, **kw), "style")


def test_camera_matrix_matches_oracle():
    from paper_2504_20937_b300.api import Context
    rng = np.random.default_rng(1)
    with Context(1920, 1080) as ctx:
        cams = [((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)]
        for f in range(0, 1000, 37):
            cams.append((inputs.orbit_eye(f, 0.36), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0))
        for _ in range(30):
            eye = tuple(rng.uniform(-3, 3, 3))
            cams.append((eye, tuple(rng.uniform(0, 1, 3)), (0, 1, 0), float(rng.uniform(20, 120)),
                         0.05, 50.0))
        for eye, tgt, up, fov, zn, zf in cams:
            ctx.set_camera(eye, tgt, up, fov, zn, zf)
            got = np.array(ctx.get_matrix(), np.float32)
            want = oracle.camera_f32(eye, tgt, up, fov, 1920 / 1080, zn, zf).reshape(-1)
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_empty_and_degenerate_frames():
    n = 10_000
    stored = inputs.encode(inputs.uniform_cloud(n, 25), "f32")
    # depth range beyond the cloud: nothing drawn, all background
    g = gpu_run(stored, "f32", 64, 48, 1, 1e-3, 1, fixed_eye, znear=50.0, zfar=60.0, background=0xAB)
    assert np.all(g[1] == oracle.EMPTY_KEY) and np.all(g[2] == 0xAB)
    # zero amplitude: positions do not move
    g = gpu_run(stored, "f32", 64, 48, 1, 0.0, 5, fixed_eye)
    assert np.array_equal(g[0], stored)
    # all points clamped at a corner: one pixel wins, smallest id at equal depth
    corner = np.zeros((1000, 3), np.float32)
    args = (corner, "f32", 33, 17, 2, 1e-3, 1, fixed_eye)
    g, o = gpu_run(*args), oracle_run(*args)
    _assert_same(g, o, "corner")


def test_single_pixel_framebuffer_and_tall_frame():
    stored = inputs.encode(inputs.uniform_cloud(5000, 26), "f32")
    for W, H in [(1, 1), (1, 1000), (999, 1)]:
        args = (stored, "f32", W, H, 2, 1e-3, 2, fixed_eye)
        _assert_same(gpu_run(*args), oracle_run(*args), f"{W}x{H}")


@pytest.mark.parametrize("W,H", [(32768, 32), (16384, 4096)])
def test_large_frames_bit_exact(W, H):
    """The widest frame allowed and a 67M-pixel frame (pixel indices past
    2^26, a resolve grid of 16.8M quads), bit for bit."""
    stored = inputs.encode(inputs.gaussian_mixture_cloud(1 << 21, 29, components=8, sigma=0.1), "f32")
    args = (stored, "f32", W, H, 4, 1e-3, 2, orbit(9.0))
    g, o = gpu_run(*args), oracle_run(*args)
    _assert_same(g, o, f"{W}x{H}")
    assert (o[1] != oracle.EMPTY_KEY).sum() > 100       # at 1024:1 the cloud is a few hundred pixels wide


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_pingpong_matches_in_place_and_keeps_previous_state(dtype):
    """Out-of-place stepping into the other buffer (the paper's alternating
    buffers): same positions and frames as the oracle's in-place steps, and
    the buffer that was read still holds the previous state."""
    from paper_2504_20937_b300.api import Context
    n, W, H, frames, seed, a = 40_003, 120, 90, 5, 13, 1e-3
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 28, components=3, sigma=0.05), dtype)
    eye = orbit(4.0)
    tview = np.float32 if dtype == "f32" else np.int16
    with Context(W, H) as ctx:
        bufs = ctx.alloc_pingpong(n, dtype)
        bufs[0].copy_(torch.from_numpy(stored.view(tview)))
        ctx.set_sim(seed, 0, a, 0)
        for f in range(frames):
            before = ctx.points.clone()
            read = ctx.visible
            ctx.set_camera(eye(f), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
            ctx.step_and_render_pingpong()
            torch.cuda.synchronize()
            assert ctx.visible == 1 - read
            assert torch.equal(bufs[read], before)            # the state that was read is untouched
        gpos = ctx.points.cpu().numpy().view(stored.dtype)
        gkeys = ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64)
        grgba = ctx.frame_rgba().cpu().numpy().reshape(-1).view(np.uint32)
        # rendering the other (previous) buffer gives the previous state's frame
        ctx.set_visible(1 - ctx.visible)
        ctx.render()
        torch.cuda.synchronize()
        prev_keys = ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64)
    o = oracle_run(stored, dtype, W, H, seed, a, frames, eye)
    assert np.array_equal(gpos.view(np.uint8), o[0].view(np.uint8))
    assert np.array_equal(gkeys, o[1]) and np.array_equal(grgba, o[2])
    prev = oracle_run(stored, dtype, W, H, seed, a, frames - 1, eye)[0]
    M = oracle.camera_f32(eye(frames - 1), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, W / H, 0.1, 100.0)
    want_prev, _ = oracle.render(prev, dtype, M, W, H, np.float32(0.1), np.float32(100.0))
    assert np.array_equal(prev_keys, want_prev)


def test_indexed_colours():
    """colour = colormap[index[id]] (index >= ncolors takes the default)."""
    from paper_2504_20937_b300.api import Context
    n, W, H, ncolors = 25_000, 100, 80, 9
    stored = inputs.encode(inputs.uniform_cloud(n, 29), "f32")
    rng = np.random.default_rng(3)
    index = rng.integers(0, ncolors + 2, size=n).astype(np.uint32)
    cmap = rng.integers(0, 2**32, size=ncolors, dtype=np.uint64).astype(np.uint32)
    default = 0xFF112233
    with Context(W, H) as ctx:
        ctx.alloc_points(n, "f32").copy_(torch.from_numpy(stored))
        idx, cm = ctx.alloc_indexed_colors(ncolors)
        idx.copy_(torch.from_numpy(index.view(np.int32)))
        cm.copy_(torch.from_numpy(cmap.view(np.int32)))
        ctx.set_sim(5, 0, 1e-3, 0)
        ctx.set_style(default, 0x44)
        for f in range(2):
            ctx.set_camera(fixed_eye(f), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
            ctx.step_and_render()
        torch.cuda.synchronize()
        grgba = ctx.frame_rgba().cpu().numpy().reshape(-1).view(np.uint32)
    per_point = np.where(index < ncolors, cmap[np.minimum(index, ncolors - 1)], default).astype(np.uint32)
    o = oracle_run(stored, "f32", W, H, 5, 1e-3, 2, fixed_eye, colors=per_point, color=default, background=0x44)
    assert np.array_equal(grgba, o[2])
    assert len(np.unique(grgba)) > ncolors // 2


@pytest.mark.parametrize("dtype,radius", [("f32", 0.5), ("f32", 1.0), ("f32", 2.5), ("f32", 4.0), ("f16", 2.0),
                                          ("bf16", 1.5)])
def test_disc_markers_bit_exact(dtype, radius):
    """Disc markers of radius r pixels against the oracle (ragged n, odd
    frame, clustered cloud so discs overlap heavily)."""
    from paper_2504_20937_b300.api import Context
    n, W, H, frames, seed, a = 20_003, 97, 61, 2, 17, 1e-3
    stored = inputs.encode(inputs.gaussian_mixture_cloud(n, 30, components=3, sigma=0.05), dtype)
    eye = orbit(6.0)
    tview = np.float32 if dtype == "f32" else np.int16
    with Context(W, H) as ctx:
        ctx.alloc_points(n, dtype).copy_(torch.from_numpy(stored.view(tview)))
        ctx.set_sim(seed, 0, a, 0)
        ctx.set_marker(radius)
        for f in range(frames):
            ctx.set_camera(eye(f), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
            ctx.step_and_render()
        torch.cuda.synchronize()
        gpos = ctx.points.cpu().numpy().view(stored.dtype)
        gkeys = ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64)
        grgba = ctx.frame_rgba().cpu().numpy().reshape(-1).view(np.uint32)
    pos = stored.copy()
    for f in range(frames):
        oracle.displace(pos, dtype, seed, 0, f, np.float32(a))
    M = oracle.camera_f32(eye(frames - 1), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, W / H, 0.1, 100.0)
    keys, rgba = oracle.render_disc(oracle.from_storage(pos, dtype), M, W, H, np.float32(0.1), np.float32(100.0),
                                    np.float32(radius))
    assert np.array_equal(gpos.view(np.uint8), pos.view(np.uint8))
    assert np.array_equal(gkeys, keys), f"{np.count_nonzero(gkeys != keys)} pixels differ"
    assert np.array_equal(grgba, rgba)
    assert (gkeys != oracle.EMPTY_KEY).sum() > 100          # the discs are really drawn


def test_checkpoint_and_resume_is_bit_exact():
    """State at step s is a pure function of (initial positions, seed, s):
    a positions snapshot plus first_step resumes a run bit for bit."""
    from paper_2504_20937_b300.api import Context
    n, W, H, seed, a = 30_011, 80, 60, 21, 1e-3
    stored = inputs.encode(inputs.uniform_cloud(n, 32), "f32")
    eye = orbit(3.0)

    def run(ctx, frames, first):
        for f in range(first, first + frames):
            ctx.set_camera(eye(f), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
            ctx.step_and_render()
        torch.cuda.synchronize()

    with Context(W, H) as ctx:
        ctx.alloc_points(n, "f32").copy_(torch.from_numpy(stored))
        ctx.set_sim(seed, 0, a, 0)
        run(ctx, 6, 0)
        snapshot, step = ctx.points.clone(), ctx.step
        run(ctx, 5, 6)
        want_pos = ctx.points.cpu().numpy()
        want_rgba = ctx.frame_rgba().cpu().numpy()
    assert step == 6
    with Context(W, H) as ctx:
        ctx.alloc_points(n, "f32").copy_(snapshot)
        ctx.set_sim(seed, 0, a, step)
        run(ctx, 5, 6)
        assert np.array_equal(ctx.points.cpu().numpy(), want_pos)
        assert np.array_equal(ctx.frame_rgba().cpu().numpy(), want_rgba)


@pytest.mark.parametrize("kernel", ["grid", "depth_bound"])
@pytest.mark.parametrize("radius", [0.5, 1.0, 1.5, 2.0, 3.0, 64.0])
@pytest.mark.parametrize("W,H", [(64, 64), (61, 37)])
def test_disc_markers_at_exact_pixel_distances(radius, W, H, kernel):
    """Disc centres exactly on pixel centres and pixel edges and one ulp or
    2^-20 either side of them, so many candidate pixels sit exactly at, or a
    rounding away from, distance r; discs partly off the frame.  With the
    clip matrix x, y -> (x, y, w = 1) the screen position is (x + 1) W/2,
    (1 - y) H/2.  Rendered (no displacement) against the oracle's wide
    candidate box, bit for bit: the kernel's tighter box must hold every
    pixel that passes."""
    from paper_2504_20937_b300.api import Context
    base = np.arange(-110, 111, dtype=np.float64) / 64.0           # screen offsets in half pixels
    vals = set()
    for v in base.astype(np.float32):
        for d in (np.float32(0), np.float32(2.0 ** -20)):
            vals.update({np.float32(v + d), np.float32(v - d)})
        vals.update({np.nextafter(v, np.float32(2)), np.nextafter(v, np.float32(-2))})
    vals = np.array(sorted(vals), dtype=np.float32)
    rng = np.random.default_rng(int(radius * 8) + W)
    xs = rng.choice(vals, 4000)
    ys = rng.choice(vals, 4000)
    pos = np.stack([xs, ys, np.zeros_like(xs)], axis=1).astype(np.float32)
    M = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], dtype=np.float32)
    with Context(W, H) as ctx:
        ctx.alloc_points(len(pos), "f32").copy_(torch.from_numpy(pos))
        ctx.set_matrix(M, 0.5, 2.0)
        ctx.set_marker(radius)
        ctx.set_launch(64, 0, kernel)
        ctx.render()
        torch.cuda.synchronize()
        gkeys = ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64)
    keys, _ = oracle.render_disc(pos, M.reshape(-1), W, H, np.float32(0.5), np.float32(2.0), np.float32(radius))
    assert np.array_equal(gkeys, keys), f"{np.count_nonzero(gkeys != keys)} pixels differ"
    assert (keys != oracle.EMPTY_KEY).sum() > W * H // 4


def test_per_frame_kernel_timing_ring():
    """Frames enqueued back to back keep their own kernel times; reading a
    frame that was not timed, or after timing restarts, is refused."""
    from paper_2504_20937_b300.api import Context, MmrError
    n, W, H = 50_000, 64, 48
    stored = inputs.encode(inputs.uniform_cloud(n, 41), "f32")
    with Context(W, H) as ctx:
        ctx.alloc_points(n, "f32").copy_(torch.from_numpy(stored))
        ctx.set_camera((0.5, 0.5, 2.5), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, 0.1, 100.0)
        with pytest.raises(MmrError, match="STATE"):
            ctx.last_kernel_ms()                      # timing is off
        ctx.set_timing(True)
        for _ in range(10):
            ctx.step_and_render()
        times = [ctx.frame_kernel_ms(k) for k in range(10)]
        assert all(p > 0.0 and r > 0.0 for p, r in times)
        assert ctx.last_kernel_ms() == times[0]
        with pytest.raises(MmrError, match="STATE"):
            ctx.frame_kernel_ms(10)
        ctx.set_timing(True)                          # restarts the count
        with pytest.raises(MmrError, match="STATE"):
            ctx.frame_kernel_ms(0)
