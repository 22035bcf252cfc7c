"""Batched clouds: each cloud in the batch must equal the oracle run of that
cloud alone (bit-exact positions, keys and RGBA), whatever the launch shape,
direct or graph-replayed, before or after autotuning."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs

from ._harness import CENTRE, UP, oracle_run

pytestmark = pytest.mark.gpu


def _eye_fn(radius, elevation, start_deg, deg):
    return lambda f: inputs.orbit_eye(f, deg, radius, CENTRE, elevation, start_deg)


def _make(sizes_res, dtype, seed=0):
    rng = np.random.default_rng(seed)
    clouds, stored, eyes = [], [], []
    for i, (n, W, H) in enumerate(sizes_res):
        pos = inputs.uniform_cloud(n, 500 + i) if i % 2 == 0 else \
            inputs.gaussian_mixture_cloud(n, 500 + i, components=4, sigma=0.05)
        stored.append(inputs.encode(pos, dtype))
        clouds.append(dict(n=n, width=W, height=H, seed=1000 + i, cloud=i, amplitude=1e-3 * (1 + i % 3),
                           color=0xFF000000 | i, background=i))
        eyes.append(_eye_fn(float(rng.uniform(1.5, 3.0)), float(rng.uniform(-0.5, 0.5)),
                            float(rng.uniform(0, 360)), 2.0))
    return clouds, stored, eyes


def _upload(batch, stored):
    for i, s in enumerate(stored):
        batch.points(i).copy_(torch.from_numpy(s if s.dtype == np.float32 else s.view(np.int16)))
    torch.cuda.synchronize()


def _set_cameras(batch, eyes, slots, frame0=0):
    for i, e in enumerate(eyes):
        for s in range(slots):
            batch.set_camera(i, s, e(frame0 + s), CENTRE, UP, 60.0, 0.1, 100.0)


def _download(batch, i, dtype):
    torch.cuda.synchronize()
    pos = batch.points(i).cpu().numpy()
    if dtype != "f32":
        pos = pos.view(np.uint16)
    keys = batch.frame_keys(i).cpu().numpy().reshape(-1).view(np.uint64)
    rgba = batch.frame_rgba(i).cpu().numpy().reshape(-1).view(np.uint32)
    return pos, keys, rgba


def _oracle(c, s, eye, dtype, frames):
    return oracle_run(s, dtype, c["width"], c["height"], c["seed"], c["amplitude"], frames, eye,
                      cloud=c["cloud"], color=c.get("color", 0xFFFFFFFF), background=c.get("background", 0))


def _check_all(batch, clouds, stored, eyes, dtype, frames):
    batch.check_device()                    # no pixel item gave up waiting
    for i, c in enumerate(clouds):
        g = _download(batch, i, dtype)
        o = _oracle(c, stored[i], eyes[i], dtype, frames)
        assert np.array_equal(g[0].view(np.uint8), o[0].view(np.uint8)), f"positions of cloud {i}"
        assert np.array_equal(g[1], o[1]), f"keys of cloud {i}"
        assert np.array_equal(g[2], o[2]), f"rgba of cloud {i}"


RAGGED = [(1, 16, 16), (5, 37, 23), (4097, 64, 48), (30_001, 128, 128), (2, 1, 1), (65_536, 256, 256),
          (999, 33, 17), (200_003, 320, 200), (8, 3, 5), (12_345, 100, 60)]


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_batch_direct_matches_oracle_per_cloud(dtype):
    from paper_2504_20937_b300.api import Batch
    clouds, stored, eyes = _make(RAGGED, dtype)
    frames = 3
    with Batch(clouds, dtype, camera_slots=frames) as b:
        _upload(b, stored)
        _set_cameras(b, eyes, frames)
        for _ in range(frames):
            b.step_and_render()
        assert b.frames == frames
        _check_all(b, clouds, stored, eyes, dtype, frames)


@pytest.mark.parametrize("dtype,pinned", [("f32", True), ("f16", False), ("bf16", True)])
def test_batch_roundtrip_matches_oracle_per_cloud(dtype, pinned):
    """The host round trip (displace, positions device -> host -> device,
    render from the copy) mixed with zero-copy frames: every cloud still
    equals its oracle run."""
    from paper_2504_20937_b300.api import Batch
    clouds, stored, eyes = _make(RAGGED, dtype, seed=3)
    frames = 4
    with Batch(clouds, dtype, camera_slots=frames) as b:
        _upload(b, stored)
        _set_cameras(b, eyes, frames)
        b.step_and_render_roundtrip(pinned=pinned)
        b.step_and_render()
        b.step_and_render_roundtrip(pinned=not pinned)       # switching host buffer kinds
        b.step_and_render_roundtrip(pinned=pinned)
        assert b.frames == frames
        _check_all(b, clouds, stored, eyes, dtype, frames)


@pytest.mark.parametrize("launch", [(32, 0, 1), (128, 1, 64), (512, 8, 1024), (512, 2, 7), (64, 0, 65536)])
def test_batch_launch_shapes_and_graph(launch):
    from paper_2504_20937_b300.api import Batch
    clouds, stored, eyes = _make(RAGGED, "f32", seed=1)
    frames = 4
    with Batch(clouds, "f32", camera_slots=frames) as b:
        _upload(b, stored)
        _set_cameras(b, eyes, frames)
        b.set_launch(*launch)
        b.step_and_render()            # frame 0 direct
        b.run_graph(frames - 1)        # frames 1..3 by graph replay
        _check_all(b, clouds, stored, eyes, "f32", frames)


def test_batch_autotune_keeps_state():
    from paper_2504_20937_b300.api import Batch
    clouds, stored, eyes = _make(RAGGED, "f32", seed=2)
    frames = 3
    with Batch(clouds, "f32", camera_slots=frames) as b:
        _upload(b, stored)
        _set_cameras(b, eyes, frames)
        b.step_and_render()
        best = b.autotune(frames_per_config=1)
        assert best["threads"] in (64, 128, 256) and best["ms_per_frame"] > 0
        assert best["chunk_groups"] % best["threads"] == 0
        assert b.frames == 1
        b.run_graph(frames - 1)
        _check_all(b, clouds, stored, eyes, "f32", frames)


def test_batch_requires_cameras_and_validates():
    from paper_2504_20937_b300.api import Batch, MmrError
    clouds, stored, eyes = _make(RAGGED[:3], "f32")
    with Batch(clouds, "f32", camera_slots=2) as b:
        with pytest.raises(MmrError, match="STATE"):
            b.step_and_render()
        _set_cameras(b, eyes, 1)
        b.step_and_render()                      # slot 0 is set
        with pytest.raises(MmrError, match="STATE"):
            b.step_and_render()                  # slot 1 is not
        with pytest.raises(MmrError, match="INVALID"):
            b.set_launch(33, 0, 1)
        with pytest.raises(MmrError, match="INVALID"):
            b.set_launch(1024, 0, 1)
    with pytest.raises(MmrError, match="INVALID"):
        Batch([dict(n=0, width=4, height=4)])
    with pytest.raises(MmrError, match="BUDGET"):
        Batch([dict(n=1000, width=64, height=64)], budget_bytes=1000)


def test_batched_256_clouds_graph_sampled():
    """The 256-cloud benchmark scene (log-uniform sizes 1e3..1e6, uniform or
    4-cluster, own orbit camera and resolution), 100 frames by graph replay
    after autotuning; a spread of clouds is replayed alone by the oracle."""
    from paper_2504_20937_b300.api import Batch
    table = inputs.batched_table()
    frames = 100
    clouds, stored, eyes = [], [], []
    for i, bc in enumerate(table):
        clouds.append(dict(n=bc.n, width=bc.W, height=bc.H, seed=4, cloud=i, amplitude=5e-4))
        stored.append(inputs.encode(inputs.batch_cloud_positions(bc), "f32"))
        eyes.append(_eye_fn(bc.radius, bc.elevation, bc.start_deg, bc.deg_per_frame))
    with Batch(clouds, "f32", camera_slots=frames) as b:
        _upload(b, stored)
        _set_cameras(b, eyes, frames)
        b.autotune(frames_per_config=1)
        b.run_graph(frames)
        order = np.argsort([c["n"] for c in clouds])
        sample = sorted(set(order[[0, 1, 64, 128, 200, 254, 255]].tolist()))
        for i in sample:
            c = clouds[i]
            g = _download(b, i, "f32")
            o = _oracle(c, stored[i], eyes[i], "f32", frames)
            assert np.array_equal(g[0], o[0]), f"positions of cloud {i} (n={c['n']})"
            assert np.array_equal(g[1], o[1]), f"keys of cloud {i}"
            assert np.array_equal(g[2], o[2]), f"rgba of cloud {i}"


# (eye, target): the cloud in view, behind the camera (every point culled), from the side, partly in view
_VIEWS = [((0.5, 0.5, 2.5), CENTRE), ((0.5, 0.5, -2.5), (0.5, 0.5, -5.0)), ((2.5, 0.5, 0.5), CENTRE),
          ((0.5, 0.5, 2.5), (1.4, 1.3, 0.5))]


@pytest.mark.parametrize("mode", ["direct", "graph", "roundtrip"])
def test_batch_chunks_emptied_and_refilled(mode):
    """The batch resolve repaints and clears only 64-pixel chunks that a frame
    or the one before touched.  Each cloud's view turns away from it for a
    frame and back (on different frames for different clouds), with non-zero
    backgrounds and ragged frames; every cloud is compared with the oracle at
    every frame."""
    from paper_2504_20937_b300.api import Batch
    sizes = [(20_000, 96, 64), (5_000, 61, 37), (30_000, 128, 128), (1_000, 7, 5)]
    clouds, stored, _ = _make(sizes, "f32", seed=7)
    frames = 2 * len(_VIEWS)
    views = lambda f, i: _VIEWS[(f + i) % len(_VIEWS)]   # noqa: E731
    with Batch(clouds, "f32", camera_slots=frames) as b:
        _upload(b, stored)
        for i in range(len(clouds)):
            for f in range(frames):
                eye, target = views(f, i)
                b.set_camera(i, f, eye, target, UP, 60.0, 0.1, 100.0)
        pos = [np.array(s, copy=True) for s in stored]
        for f in range(frames):
            if mode == "graph":
                b.run_graph(1)
            elif mode == "roundtrip":
                b.step_and_render_roundtrip()
            else:
                b.step_and_render()
            for i, c in enumerate(clouds):
                oracle.displace(pos[i], "f32", c["seed"], c["cloud"], f, np.float32(c["amplitude"]))
                eye, target = views(f, i)
                M = oracle.camera_f32(eye, target, UP, 60.0, c["width"] / c["height"], 0.1, 100.0)
                keys, rgba = oracle.render(pos[i], "f32", M, c["width"], c["height"], np.float32(0.1),
                                           np.float32(100.0), None, c["color"], c["background"])
                gpos, gk, gr = _download(b, i, "f32")
                assert np.array_equal(gpos, pos[i]), (mode, f, i)
                assert np.array_equal(gk, keys) and np.array_equal(gr, rgba), (mode, f, i)
