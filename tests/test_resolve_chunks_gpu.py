"""The resolve repaints and clears only the 64-pixel chunks that its frame or
the previous one touched.  These cases make chunks go from covered to empty
and back, change the background between frames, and run the frame numbers
through their wrap; every frame is compared with the oracle whole (keys and
RGBA), so a stale key or a pixel left unpainted would show."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.api import Context

from ._harness import CENTRE, UP, download_frame, upload

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (eye, target) per frame: the cloud in view, then behind the camera (every
# point culled: an empty frame), then in view again from the side, then only
# a corner of it in view
VIEWS = [((0.5, 0.5, 2.5), CENTRE), ((0.5, 0.5, -2.5), (0.5, 0.5, -5.0)), ((2.5, 0.5, 0.5), CENTRE),
         ((0.5, 0.5, 2.5), (1.4, 1.3, 0.5)), ((0.5, 0.5, 2.5), CENTRE)]


def _frames(stored, dtype, W, H, views, styles, seed=5, amplitude=1e-3, launches=None):
    """GPU and oracle frames for a sequence of views and (colour, background)
    styles; launches, if given, is each frame's (kernel, threads, CTAs per SM)."""
    n = stored.shape[0]
    got, want = [], []
    pos = np.array(stored, copy=True)
    with Context(W, H) as ctx:
        ctx.alloc_points(n, dtype)
        upload(ctx, stored)
        ctx.set_sim(seed, 0, amplitude, 0)
        for f, ((eye, target), (color, bg)) in enumerate(zip(views, styles)):
            if launches is not None:
                kernel, threads, ctas = launches[f]
                ctx.set_launch(threads, ctas, kernel)
            ctx.set_style(color, bg)
            ctx.set_camera(eye, target, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render()
            got.append(download_frame(ctx))
            oracle.displace(pos, dtype, seed, 0, f, np.float32(amplitude))
            M = oracle.camera_f32(eye, target, UP, 60.0, W / H, 0.1, 100.0)
            want.append(oracle.render(pos, dtype, M, W, H, np.float32(0.1), np.float32(100.0), None, color, bg))
    return got, want


def _assert_frames(got, want, what):
    for f, ((gk, gr), (ok, orr)) in enumerate(zip(got, want)):
        assert np.array_equal(gk, ok), f"{what}: keys of frame {f}"
        assert np.array_equal(gr, orr), f"{what}: rgba of frame {f}"


@pytest.mark.parametrize("W,H", [(160, 96), (61, 37), (3, 3), (1, 1), (1000, 1)])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_chunks_emptied_and_refilled(W, H, dtype):
    """Chunks covered in one frame, empty in the next (the cloud behind the
    camera), covered again from another side and partly: pixel counts that
    are multiples of 64, ragged ones and frames smaller than a chunk."""
    stored = inputs.encode(inputs.gaussian_mixture_cloud(50_001, 61, components=3, sigma=0.05), dtype)
    styles = [(0xFFFFFFFF, 0)] * len(VIEWS)
    got, want = _frames(stored, dtype, W, H, VIEWS, styles)
    assert (got[1][1] == 0).all() and (got[1][0] == np.uint64(2**64 - 1)).all()
    _assert_frames(got, want, f"{W}x{H} {dtype}")


def test_background_and_colour_changes_repaint():
    """A new background between frames repaints every empty pixel, including
    chunks that stayed empty; a new point colour repaints the covered ones."""
    stored = inputs.encode(inputs.gaussian_mixture_cloud(40_000, 62, components=2, sigma=0.03), "f32")
    views = [VIEWS[0]] * 5 + [VIEWS[1]] * 2
    styles = [(0xFFFFFFFF, 0), (0xFFFFFFFF, 0x11223344), (0xFF00FF00, 0x11223344), (0xFF00FF00, 0x11223344),
              (0xFFFFFFFF, 0), (0xFFFFFFFF, 0x55667788), (0xFFFFFFFF, 0x55667788)]
    got, want = _frames(stored, "f32", 128, 80, views, styles)
    _assert_frames(got, want, "styles")


def test_frame_numbers_wrap():
    """The library numbers frames with 32 bits and clears its chunk tags when
    the numbers would repeat: start three frames before the wrap (a test hook
    read at context creation) and compare six frames with the oracle."""
    code = """
        import sys; sys.path.insert(0, '.')
        import numpy as np
        from tests.test_resolve_chunks_gpu import VIEWS, _frames, _assert_frames
        from paper_2504_20937_b300 import inputs
        stored = inputs.encode(inputs.gaussian_mixture_cloud(30_000, 63, components=2, sigma=0.04), "f32")
        views = [VIEWS[0], VIEWS[1], VIEWS[0], VIEWS[2], VIEWS[1], VIEWS[0]]
        got, want = _frames(stored, "f32", 96, 64, views, [(0xFFFFFFFF, 0)] * 6)
        _assert_frames(got, want, "wrap")
        print("frames equal")
    """
    env = dict(os.environ, MMR_FIRST_FRAME_NUMBER=str(0xFFFFFFFD))
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "frames equal" in r.stdout


def test_frame_ptr_buffers_after_empty_frame():
    """After a frame with every point culled, the depth-id buffer of the
    latest frame is all empty and the framebuffer all background; the next
    frame with points matches the oracle."""
    stored = inputs.encode(inputs.uniform_cloud(20_000, 64), "f32")
    views = [VIEWS[0], VIEWS[1], VIEWS[1], VIEWS[0]]
    got, want = _frames(stored, "f32", 64, 64, views, [(0xFFFFFFFF, 0x01020304)] * 4)
    for f in (1, 2):
        assert (got[f][0] == np.uint64(2**64 - 1)).all() and (got[f][1] == 0x01020304).all()
    _assert_frames(got, want, "empty frames")
    torch.cuda.synchronize()


# per frame: (kernel, threads, CTAs per SM): grid-stride with one thread per
# group and persistent, the two-pass depth bounds, the warp-aggregated splat
# and the TMA-staged kernel, in turn.
SWITCHES = [("grid", 64, 0), ("depth_bound", 64, 0), ("grid", 64, 0), ("warp_agg", 64, 0), ("tma", 256, 1),
            ("grid", 128, 2), ("grid", 64, 0), ("depth_bound", 64, 0), ("grid", 64, 0)]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_kernel_switches_between_frames(dtype):
    """A different point kernel each frame, with views that empty and refill
    chunks: the chunk bookkeeping holds whichever kernel filled the buffer,
    and every frame equals the oracle."""
    stored = inputs.encode(inputs.gaussian_mixture_cloud(60_003, 65, components=3, sigma=0.05), dtype)
    views = [VIEWS[0], VIEWS[2], VIEWS[1], VIEWS[3], VIEWS[0], VIEWS[1], VIEWS[2], VIEWS[0], VIEWS[3]]
    got, want = _frames(stored, dtype, 97, 61, views, [(0xFFFFFFFF, 0x10203040)] * len(views), launches=SWITCHES)
    _assert_frames(got, want, f"kernel switches {dtype}")


@pytest.mark.parametrize("dtype,n", [("f32", 1), ("f32", 3), ("f32", 7), ("f16", 5), ("f16", 13)])
def test_ragged_tail_chunks(dtype, n):
    """Clouds of a few points, all or some of them in the ragged last group
    (fewer than 4 FP32 or 8 16-bit points), which a single thread splats
    outside the vector path: the few chunks those points fill are repainted
    and cleared as they come and go.  Frames of 61x37 and 64x64 pixels."""
    stored = inputs.encode(inputs.uniform_cloud(n, 66 + n), dtype)
    views = [VIEWS[0], VIEWS[0], VIEWS[1], VIEWS[0], VIEWS[2]]
    for W, H in [(61, 37), (64, 64)]:
        got, want = _frames(stored, dtype, W, H, views, [(0xFFFFFFFF, 0x01020304)] * len(views), amplitude=1e-2)
        assert any((gk != np.uint64(2**64 - 1)).any() for gk, _ in got)
        _assert_frames(got, want, f"{n} points {dtype} {W}x{H}")
