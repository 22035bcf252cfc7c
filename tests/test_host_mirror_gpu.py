"""The host mirror of the framebuffer (mmr_alloc_host_mirror /
mmr_mirror_frame): after each update it must equal the device framebuffer of
the latest frame, and so the oracle's frame, although only the 64-pixel runs
that changed cross the host link.  Views turn away from the cloud and back,
the background changes, updates are skipped for some frames, and rendering
and mirroring run on different streams without host synchronisation in
between."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.api import Context, MmrError

from ._harness import CENTRE, UP, upload

pytestmark = pytest.mark.gpu

VIEWS = [((0.5, 0.5, 2.5), CENTRE), ((0.5, 0.5, -2.5), (0.5, 0.5, -5.0)), ((2.5, 0.5, 0.5), CENTRE),
         ((0.5, 0.5, 2.5), (1.4, 1.3, 0.5))]


def _oracle_frames(stored, W, H, views, backgrounds, seed=5, amplitude=1e-3):
    pos = np.array(stored, copy=True)
    out = []
    for f, ((eye, target), bg) in enumerate(zip(views, backgrounds)):
        oracle.displace(pos, "f32", seed, 0, f, np.float32(amplitude))
        M = oracle.camera_f32(eye, target, UP, 60.0, W / H, 0.1, 100.0)
        out.append(oracle.render(pos, "f32", M, W, H, np.float32(0.1), np.float32(100.0), None, 0xFFFFFFFF, bg)[1])
    return out


def _context(stored, W, H, seed=5, amplitude=1e-3):
    ctx = Context(W, H)
    ctx.alloc_points(stored.shape[0], "f32")
    upload(ctx, stored)
    ctx.set_sim(seed, 0, amplitude, 0)
    return ctx


@pytest.mark.parametrize("W,H", [(160, 96), (61, 37), (3, 3), (1, 1), (1001, 333)])
def test_mirror_follows_every_frame(W, H):
    stored = inputs.encode(inputs.gaussian_mixture_cloud(40_003, 71, components=3, sigma=0.05), "f32")
    views = VIEWS * 3
    backgrounds = [0] * 5 + [0x11223344] * 4 + [0] * 3
    want = _oracle_frames(stored, W, H, views, backgrounds)
    side = torch.cuda.Stream()
    with _context(stored, W, H) as ctx:
        mirror = ctx.alloc_host_mirror()
        for f, ((eye, target), bg) in enumerate(zip(views, backgrounds)):
            ctx.set_style(0xFFFFFFFF, bg)
            ctx.set_camera(eye, target, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render()
            ctx.mirror_frame(side)
            side.synchronize()
            got = mirror.reshape(-1).copy()
            dev = ctx.frame_rgba().cpu().numpy().reshape(-1).view(np.uint32)
            assert np.array_equal(dev, want[f]), f"device frame {f}"
            assert np.array_equal(got, want[f]), f"mirror frame {f}"


@pytest.mark.parametrize("side_priority", ["default", "highest"])
def test_mirror_skipped_frames_and_no_host_sync_between(side_priority):
    """Render on one stream and update the mirror on another (of the default
    or the highest priority) every third frame, with no host synchronisation
    until the end of each group of frames; the next frame's resolve waits
    for the update in flight."""
    W, H = 128, 80
    stored = inputs.encode(inputs.gaussian_mixture_cloud(60_000, 72, components=4, sigma=0.04), "f32")
    views = VIEWS * 6
    want = _oracle_frames(stored, W, H, views, [0] * len(views))
    prio = torch.cuda.Stream.priority_range()[1] if side_priority == "highest" else 0
    main, side = torch.cuda.Stream(), torch.cuda.Stream(priority=prio)
    with _context(stored, W, H) as ctx:
        mirror = ctx.alloc_host_mirror()
        for f, (eye, target) in enumerate(views):
            ctx.set_camera(eye, target, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render(main)
            if f % 3 == 2:
                ctx.mirror_frame(side)
            if f % 6 == 5:
                side.synchronize()
                assert np.array_equal(mirror.reshape(-1), want[f]), f"mirror after frame {f}"
        main.synchronize()


def test_mirror_bytes_only_changes_cross():
    """The first update writes the whole frame; an update after a frame that
    moved nothing into or out of any run writes only the runs the frame
    touched; two empty frames in a row write nothing the second time."""
    W, H = 256, 128
    stored = inputs.encode(inputs.gaussian_mixture_cloud(20_000, 73, components=1, sigma=0.01), "f32")
    with _context(stored, W, H, amplitude=0.0) as ctx:
        mirror = ctx.alloc_host_mirror()
        ctx.set_camera(*VIEWS[0], UP, 60.0, 0.1, 100.0)
        ctx.step_and_render()
        ctx.mirror_frame()
        assert ctx.mirror_bytes() == W * H * 4
        keys = ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64)
        touched_runs = len(np.unique(np.nonzero(keys != np.uint64(2**64 - 1))[0] // 64))
        assert 0 < touched_runs < W * H // 64 // 4
        ctx.step_and_render()                      # amplitude 0: the same pixels
        ctx.mirror_frame()
        assert ctx.mirror_bytes() == W * H * 4 + touched_runs * 256
        ctx.set_camera(*VIEWS[1], UP, 60.0, 0.1, 100.0)
        ctx.step_and_render()                      # empty: the runs that held points are written once more
        ctx.mirror_frame()
        assert ctx.mirror_bytes() == W * H * 4 + 2 * touched_runs * 256
        ctx.step_and_render()                      # empty again: nothing to write
        ctx.mirror_frame()
        assert ctx.mirror_bytes() == W * H * 4 + 2 * touched_runs * 256
        torch.cuda.synchronize()
        assert (mirror == 0).all()


def test_mirror_bytes_ragged_frame():
    """On a frame whose pixel count is a multiple of neither 4 nor 64 an
    update writes 16 bytes for every whole quad of each run it copies (runs
    holding a key in a whole quad, plus those the mirror still holds a point
    in) and the last 1-3 pixels every time."""
    W, H = 1001, 333
    npx, quads = W * H, W * H // 4
    stored = inputs.encode(inputs.gaussian_mixture_cloud(30_000, 75, components=2, sigma=0.02), "f32")

    def runs_holding_keys(keys):
        held = (keys[:4 * quads].reshape(quads, 4) != np.uint64(2**64 - 1)).any(axis=1)
        return set(np.unique(np.nonzero(held)[0] // 16).tolist())

    def run_bytes(runs):
        return sum(16 * (min(quads, 16 * (r + 1)) - 16 * r) for r in runs)

    with _context(stored, W, H, amplitude=0.0) as ctx:
        ctx.alloc_host_mirror()
        ctx.set_camera(*VIEWS[0], UP, 60.0, 0.1, 100.0)
        ctx.step_and_render()
        ctx.mirror_frame()
        assert ctx.mirror_bytes() == 16 * quads + 4 * (npx % 4)
        total = ctx.mirror_bytes()
        held = runs_holding_keys(ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64))
        assert held
        for eye_target in (VIEWS[3], VIEWS[1], VIEWS[1], VIEWS[0]):
            ctx.set_camera(*eye_target, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render()
            ctx.mirror_frame()
            now = runs_holding_keys(ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64))
            total += run_bytes(now | held) + 4 * (npx % 4)
            assert ctx.mirror_bytes() == total
            held = now
        torch.cuda.synchronize()


def test_mirror_4k_frame():
    """A 3840x2160 frame of a 16-cluster cloud on an orbit, the mirror brought
    up to date after every frame on a stream of the highest priority: equal to
    the oracle's frame each time, with only the changed runs written after the
    first update."""
    W, H = 3840, 2160
    stored = inputs.encode(inputs.gaussian_mixture_cloud(1 << 20, 76), "f32")
    frames = 4
    eyes = [inputs.orbit_eye(f, 3.0) for f in range(frames)]
    side = torch.cuda.Stream(priority=torch.cuda.Stream.priority_range()[1])
    pos = stored.copy()
    with _context(stored, W, H, amplitude=5e-4) as ctx:
        mirror = ctx.alloc_host_mirror()
        for f, eye in enumerate(eyes):
            ctx.set_camera(eye, CENTRE, UP, 60.0, 0.1, 100.0)
            ctx.step_and_render()
            ctx.mirror_frame(side)
            side.synchronize()
            oracle.displace(pos, "f32", 5, 0, f, np.float32(5e-4))
            M = oracle.camera_f32(eye, CENTRE, UP, 60.0, W / H, 0.1, 100.0)
            _, want = oracle.render(pos, "f32", M, W, H, np.float32(0.1), np.float32(100.0))
            assert np.array_equal(mirror.reshape(-1), want), f"mirror frame {f}"
        assert ctx.mirror_bytes() < W * H * 4 * 2       # the first update writes the frame, the others far less
        torch.cuda.synchronize()


def test_mirror_state_errors():
    stored = inputs.encode(inputs.uniform_cloud(1000, 74), "f32")
    with _context(stored, 32, 32) as ctx:
        with pytest.raises(MmrError, match="STATE"):
            ctx.mirror_frame()                     # no mirror yet
        ctx.alloc_host_mirror()
        with pytest.raises(MmrError, match="STATE"):
            ctx.mirror_frame()                     # no frame yet
        ctx.set_camera(*VIEWS[0], UP, 60.0, 0.1, 100.0)
        ctx.step_and_render()
        ctx.mirror_frame()
        torch.cuda.synchronize()
