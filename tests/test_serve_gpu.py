"""Serving engine: frames against the oracle, the same frame alone and in a
mix of viewers (bit for bit), budget admission, the round-trip baseline,
and the continuous-batching request loop."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.api import MmrError, Server
from paper_2504_20937_b300.serve import ServeConfig, run_trace

pytestmark = pytest.mark.gpu

CEN = (0.5, 0.5, 0.5)
UP = (0.0, 1.0, 0.0)
SHARED_N, SHARED_SEED, AMP = 20_001, 77, np.float32(1e-3)
SHARED_COLOR = 0xFFEEDDCC

# (private n, W, H, join tick, frames)
VIEWERS = [(1, 64, 48, 0, 6), (999, 37, 23, 2, 2), (5000, 128, 96, 3, 3), (12_345, 80, 60, 1, 5)]


def _eye(v, k):
    return inputs.orbit_eye(k, 5.0, 2.0 + 0.1 * v, CEN, 0.1 * v, 40.0 * v)


def _private(v, n):
    return inputs.encode(inputs.uniform_cloud(n, 900 + v), "f32")


def _shared():
    return inputs.encode(inputs.uniform_cloud(SHARED_N, 901), "f32")


def _viewer_args(v, n, W, H):
    return dict(private_n=n, width=W, height=H, seed=3000 + v, cloud=1 + v, amplitude=float(AMP),
                color=0xFF000000 | v, background=0x10 + v)


def _run_mix(viewers, record, roundtrip=False):
    """Drive the engine through `viewers`; returns {(v, k): (keys, rgba)} for
    the requested (viewer, frame) pairs, plus the final shared positions."""
    out = {}
    with Server(SHARED_N, "f32", SHARED_SEED, 0, float(AMP)) as srv:
        srv.shared_points().copy_(torch.from_numpy(_shared()))
        srv.set_shared_color(SHARED_COLOR)
        ids, done = {}, {}
        last_tick = max(j + f for (_, _, _, j, f) in viewers)
        for tick in range(last_tick):
            for v, (n, W, H, join, frames) in enumerate(viewers):
                if join == tick:
                    ids[v] = srv.add_viewer(**_viewer_args(v, n, W, H))
                    srv.viewer_points(ids[v]).copy_(torch.from_numpy(_private(v, n)))
                    done[v] = 0
            for v, vid in ids.items():
                srv.set_camera(vid, _eye(v, done[v]), CEN, UP, 60.0, 0.1, 100.0)
            srv.tick(roundtrip=roundtrip)
            torch.cuda.synchronize()
            for v in list(ids):
                done[v] += 1
                if (v, done[v] - 1) in record:
                    rgba, keys, f = srv.frame(ids[v])
                    assert f == done[v]
                    out[(v, done[v] - 1)] = (keys.cpu().numpy().reshape(-1).view(np.uint64),
                                             rgba.cpu().numpy().reshape(-1).view(np.uint32))
                if done[v] == viewers[v][4]:
                    srv.remove_viewer(ids.pop(v))
        shared = srv.shared_points().cpu().numpy()
    return out, shared


def _oracle_frame(v, k, join):
    n, W, H = VIEWERS[v][0], VIEWERS[v][1], VIEWERS[v][2]
    shared = _shared()
    for t in range(join + k + 1):
        oracle.displace_f32(shared, SHARED_SEED, 0, t, AMP)
    priv = _private(v, n)
    for s in range(k + 1):
        oracle.displace_f32(priv, 3000 + v, 1 + v, s, AMP)
    both = np.concatenate([shared, priv])
    colors = np.concatenate([np.full(SHARED_N, SHARED_COLOR, np.uint32), np.full(n, 0xFF000000 | v, np.uint32)])
    M = oracle.camera_f32(_eye(v, k), CEN, UP, 60.0, W / H, 0.1, 100.0)
    return oracle.render(both, "f32", M, W, H, np.float32(0.1), np.float32(100.0), colors, 0, 0x10 + v)


def test_serve_frames_match_oracle():
    record = {(0, 0), (0, 5), (1, 1), (2, 0), (2, 2), (3, 4)}
    got, shared = _run_mix(VIEWERS, record)
    for (v, k) in sorted(record):
        keys, rgba = _oracle_frame(v, k, VIEWERS[v][3])
        assert np.array_equal(got[(v, k)][0], keys), f"keys of viewer {v} frame {k}"
        assert np.array_equal(got[(v, k)][1], rgba), f"rgba of viewer {v} frame {k}"
    want = _shared()
    for t in range(max(j + f for (_, _, _, j, f) in VIEWERS)):
        oracle.displace_f32(want, SHARED_SEED, 0, t, AMP)
    assert np.array_equal(shared, want)


def test_serve_alone_equals_mix():
    """Each viewer's frames are identical when it is the only viewer (same
    join tick, so the shared cloud is at the same step) and when it is
    served together with the others; tolerance 0."""
    record = {(v, k) for v, vw in enumerate(VIEWERS) for k in range(vw[4])}
    mix, _ = _run_mix(VIEWERS, record)
    for v, vw in enumerate(VIEWERS):
        alone, _ = _run_alone(v)
        for k in range(vw[4]):
            assert np.array_equal(mix[(v, k)][0], alone[(v, k)][0]), f"keys viewer {v} frame {k}"
            assert np.array_equal(mix[(v, k)][1], alone[(v, k)][1]), f"rgba viewer {v} frame {k}"


def _run_alone(v):
    n, W, H, join, frames = VIEWERS[v]
    out = {}
    with Server(SHARED_N, "f32", SHARED_SEED, 0, float(AMP)) as srv:
        srv.shared_points().copy_(torch.from_numpy(_shared()))
        srv.set_shared_color(SHARED_COLOR)
        for _ in range(join):
            srv.tick()                          # no viewers: only the shared cloud moves
        vid = srv.add_viewer(**_viewer_args(v, n, W, H))
        srv.viewer_points(vid).copy_(torch.from_numpy(_private(v, n)))
        for k in range(frames):
            srv.set_camera(vid, _eye(v, k), CEN, UP, 60.0, 0.1, 100.0)
            srv.tick()
            torch.cuda.synchronize()
            rgba, keys, _ = srv.frame(vid)
            out[(v, k)] = (keys.cpu().numpy().reshape(-1).view(np.uint64),
                           rgba.cpu().numpy().reshape(-1).view(np.uint32))
    return out, None


def test_serve_roundtrip_gives_same_frames():
    record = {(v, VIEWERS[v][4] - 1) for v in range(len(VIEWERS))}
    a, sa = _run_mix(VIEWERS, record)
    b, sb = _run_mix(VIEWERS, record, roundtrip=True)
    assert np.array_equal(sa, sb)
    for key in record:
        assert np.array_equal(a[key][0], b[key][0]) and np.array_equal(a[key][1], b[key][1])


def test_serve_budget_admission_and_release():
    shared_bytes = (SHARED_N * 12 + 47) // 48 * 48
    viewer_bytes = (1000 * 12 + 47) // 48 * 48 + 64 * 64 * 20 + 2 * 64 * 64 // 64 * 4   # + chunk tags
    with Server(SHARED_N, "f32", 1, 0, 1e-3, budget_bytes=shared_bytes + viewer_bytes + 100) as srv:
        a = srv.add_viewer(1000, 64, 64)
        assert srv.try_add_viewer(1000, 64, 64) is None          # refused, nothing allocated
        with pytest.raises(MmrError, match="BUDGET"):
            srv.add_viewer(1000, 64, 64)
        with pytest.raises(MmrError, match="STATE"):
            srv.tick()                                            # viewer a has no camera yet
        srv.set_camera(a, (0.5, 0.5, 2.5), CEN, UP, 60.0, 0.1, 100.0)
        srv.tick()
        srv.remove_viewer(a)
        b = srv.add_viewer(1000, 64, 64)                          # fits again
        assert srv.status()["active"] == 1 and b is not None
        with pytest.raises(MmrError, match="INVALID"):
            srv.add_viewer(0, 64, 64)


def test_serve_request_loop_small_trace():
    trace = inputs.serving_trace(requests=200, seed=11, rate_hz=5000.0, frames_per_viewer=5,
                                 private_lo=1e3, private_hi=2e4, resolutions=((64, 48), (160, 90), (320, 240)))
    cfg = ServeConfig(shared_n=50_000, max_viewers=8, tick_hz=0.0)
    stats = run_trace(trace, cfg)
    s = stats.summary()
    assert s["frames"] == sum(r.frames for r in trace)
    assert 0 < s["p50_ms"] <= s["p99_ms"]
    assert 1 <= s["max_active_viewers"] <= 8
    # a budget for the shared cloud plus two of the largest viewers forces queueing on memory
    tight = ServeConfig(shared_n=50_000, max_viewers=8, tick_hz=0.0,
                        budget_bytes=(50_000 * 12 + 47) // 48 * 48 + 2 * (20_000 * 12 + 48 + 320 * 240 * 20))
    s2 = run_trace(trace, tight).summary()
    assert s2["frames"] == s["frames"] and s2["refused_for_budget"] > 0


def test_serve_request_loop_paced_by_a_display_rate():
    """At 200 Hz refreshes, every frame of every viewer is rendered, each
    viewer's frames on consecutive ticks, and a later frame's latency (from
    its refresh) stays below a refresh period when no refresh is dropped."""
    trace = inputs.serving_trace(requests=300, seed=12, rate_hz=100.0, frames_per_viewer=10,
                                 private_lo=1e3, private_hi=2e4, resolutions=((64, 48), (160, 90)))
    cfg = ServeConfig(shared_n=50_000, max_viewers=16, tick_hz=200.0)
    s = run_trace(trace, cfg).summary()
    assert s["frames"] == 300 and s["tick_hz"] == 200.0
    assert s["ticks"] >= 300 // 16
    if s["refreshes_dropped"] == 0:
        assert s["p99_ms_after_first"] < 5.0


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_serve_16bit_storage_matches_oracle(dtype):
    """Shared and private clouds stored as binary16 / bfloat16."""
    n_shared, n_priv, W, H, frames = 9_001, 2_003, 72, 40, 3
    shared = inputs.encode(inputs.uniform_cloud(n_shared, 902), dtype)
    priv = inputs.encode(inputs.uniform_cloud(n_priv, 903), dtype)
    tv = lambda a: torch.from_numpy(a.view(np.int16))  # noqa: E731
    with Server(n_shared, dtype, 55, 0, 1e-3) as srv:
        srv.shared_points().copy_(tv(shared))
        srv.set_shared_color(SHARED_COLOR)
        v = srv.add_viewer(n_priv, W, H, seed=66, cloud=9, amplitude=1e-3, color=0xFF0000AA, background=3)
        srv.viewer_points(v).copy_(tv(priv))
        for k in range(frames):
            srv.set_camera(v, _eye(1, k), CEN, UP, 60.0, 0.1, 100.0)
            srv.tick()
        torch.cuda.synchronize()
        rgba, keys, _ = srv.frame(v)
        gkeys = keys.cpu().numpy().reshape(-1).view(np.uint64)
        grgba = rgba.cpu().numpy().reshape(-1).view(np.uint32)
        gshared = srv.shared_points().cpu().numpy().view(np.uint16)
    for t in range(frames):
        oracle.displace(shared, dtype, 55, 0, t, np.float32(1e-3))
        oracle.displace(priv, dtype, 66, 9, t, np.float32(1e-3))
    assert np.array_equal(gshared, shared)
    both = np.concatenate([shared, priv])
    colors = np.concatenate([np.full(n_shared, SHARED_COLOR, np.uint32), np.full(n_priv, 0xFF0000AA, np.uint32)])
    M = oracle.camera_f32(_eye(1, frames - 1), CEN, UP, 60.0, W / H, 0.1, 100.0)
    keys, rgba = oracle.render(both, dtype, M, W, H, np.float32(0.1), np.float32(100.0), colors, 0, 3)
    assert np.array_equal(gkeys, keys) and np.array_equal(grgba, rgba)


def test_serve_full_size_sampled():
    """The serving configuration at full size: the 2^24-point shared cloud
    and viewers at 3840x2160, 1920x1080 and 640x480 with private clouds of
    1e6, 1e5 and 1e4 points, the third joining one tick later; three ticks.
    Every viewer's last frame and the shared positions against the oracle,
    bit for bit."""
    cfg = ServeConfig()
    amp = np.float32(cfg.amplitude)
    shared0 = inputs.encode(inputs.uniform_cloud(cfg.shared_n, cfg.shared_seed), "f32")
    viewers = [(1_000_000, 3840, 2160, 0), (100_000, 1920, 1080, 0), (10_000, 640, 480, 1)]
    ticks = 3
    got = {}
    with Server(cfg.shared_n, "f32", cfg.shared_seed, 0, cfg.amplitude) as srv:
        srv.shared_points().copy_(torch.from_numpy(shared0))
        srv.set_shared_color(SHARED_COLOR)
        ids, done = {}, {}
        for tick in range(ticks):
            for v, (n, W, H, join) in enumerate(viewers):
                if join == tick:
                    ids[v] = srv.add_viewer(**_viewer_args(v, n, W, H))
                    srv.viewer_points(ids[v]).copy_(torch.from_numpy(_private(v, n)))
                    done[v] = 0
            for v, vid in ids.items():
                srv.set_camera(vid, _eye(v, done[v]), CEN, UP, 60.0, 0.1, 100.0)
            srv.tick()
            for v in ids:
                done[v] += 1
        torch.cuda.synchronize()
        for v, vid in ids.items():
            rgba, keys, f = srv.frame(vid)
            assert f == done[v]
            got[v] = (done[v], keys.cpu().numpy().reshape(-1).view(np.uint64),
                      rgba.cpu().numpy().reshape(-1).view(np.uint32))
        shared_gpu = srv.shared_points().cpu().numpy()
    shared = shared0.copy()
    for t in range(ticks):
        oracle.displace_f32(shared, cfg.shared_seed, 0, t, amp)
    assert np.array_equal(shared_gpu, shared), "shared positions"
    for v, (n, W, H, join) in enumerate(viewers):
        frames, gkeys, grgba = got[v]
        priv = _private(v, n)
        for s in range(frames):
            oracle.displace_f32(priv, 3000 + v, 1 + v, s, AMP)      # the private amplitude of _viewer_args
        both = np.concatenate([shared, priv])
        colors = np.concatenate([np.full(cfg.shared_n, SHARED_COLOR, np.uint32),
                                 np.full(n, 0xFF000000 | v, np.uint32)])
        M = oracle.camera_f32(_eye(v, frames - 1), CEN, UP, 60.0, W / H, 0.1, 100.0)
        keys, rgba = oracle.render(both, "f32", M, W, H, np.float32(0.1), np.float32(100.0), colors, 0, 0x10 + v)
        bad = np.nonzero(gkeys != keys)[0]
        assert bad.size == 0, (f"keys of viewer {v} ({W}x{H}): {bad.size} pixels differ, first {bad[:4]}, "
                               f"gpu {[hex(int(x)) for x in gkeys[bad[:4]]]}, oracle {[hex(int(x)) for x in keys[bad[:4]]]}")
        assert np.array_equal(grgba, rgba), f"rgba of viewer {v} ({W}x{H})"
        assert (keys != oracle.EMPTY_KEY).sum() > W * H // 20


def _oracle_viewer_frame(v, n, W, H, shared_ticks, private_steps, eye):
    shared = _shared()
    for t in range(shared_ticks):
        oracle.displace_f32(shared, SHARED_SEED, 0, t, AMP)
    priv = _private(v, n)
    for s in range(private_steps):
        oracle.displace_f32(priv, 3000 + v, 1 + v, s, AMP)
    both = np.concatenate([shared, priv])
    colors = np.concatenate([np.full(SHARED_N, SHARED_COLOR, np.uint32), np.full(n, 0xFF000000 | v, np.uint32)])
    M = oracle.camera_f32(eye, CEN, UP, 60.0, W / H, 0.1, 100.0)
    return oracle.render(both, "f32", M, W, H, np.float32(0.1), np.float32(100.0), colors, 0, 0x10 + v)


def test_serve_reuses_departed_viewers_buffers():
    """A departed viewer's buffers serve the next join: a join of the same
    frame size takes no new device memory and still renders like the oracle
    (its reused buffers were cleared), and a join that needs larger buffers
    makes the kept ones give way under a budget that holds one viewer."""
    shared_bytes = (SHARED_N * 12 + 47) // 48 * 48
    budget = shared_bytes + (1000 * 12 + 47) // 48 * 48 + 64 * 64 * 20 + 2 * 64 * 64 // 64 * 4 + 100
    with Server(SHARED_N, "f32", SHARED_SEED, 0, float(AMP), budget_bytes=budget) as srv:
        srv.shared_points().copy_(torch.from_numpy(_shared()))
        srv.set_shared_color(SHARED_COLOR)

        def join_and_tick(v, n, W, H):
            vid = srv.add_viewer(**_viewer_args(v, n, W, H))
            srv.viewer_points(vid).copy_(torch.from_numpy(_private(v, n)))
            srv.set_camera(vid, _eye(v, 0), CEN, UP, 60.0, 0.1, 100.0)
            srv.tick()
            torch.cuda.synchronize()
            rgba, keys, f = srv.frame(vid)
            assert f == 1
            return vid, keys.cpu().numpy().reshape(-1).view(np.uint64), rgba.cpu().numpy().reshape(-1).view(np.uint32)

        a, _, _ = join_and_tick(0, 1000, 64, 64)                 # tick 0
        held = srv.status()["device_bytes"]
        srv.remove_viewer(a)
        assert srv.status()["device_bytes"] == held and srv.status()["active"] == 0
        b, keys, rgba = join_and_tick(1, 800, 64, 64)            # tick 1: reused buffers
        assert srv.status()["device_bytes"] == held
        want = _oracle_viewer_frame(1, 800, 64, 64, 2, 1, _eye(1, 0))
        assert np.array_equal(keys, want[0]) and np.array_equal(rgba, want[1])
        srv.remove_viewer(b)
        c, keys, rgba = join_and_tick(2, 1000, 4097, 1)          # tick 2: needs larger buffers
        assert srv.status()["device_bytes"] <= budget and srv.status()["active"] == 1
        want = _oracle_viewer_frame(2, 1000, 4097, 1, 3, 1, _eye(2, 0))
        assert np.array_equal(keys, want[0]) and np.array_equal(rgba, want[1])


# (eye, target): the cloud in view, behind the camera (every point culled), from the side, partly in view
_VIEWS = [((0.5, 0.5, 2.5), CEN), ((0.5, 0.5, -2.5), (0.5, 0.5, -5.0)), ((2.5, 0.5, 0.5), CEN),
          ((0.5, 0.5, 2.5), (1.4, 1.3, 0.5))]


@pytest.mark.parametrize("roundtrip", [False, True])
def test_serve_chunks_emptied_and_refilled(roundtrip):
    """The serving resolve stores only in 64-pixel chunks a view's frame or
    its previous one touched.  Each viewer's view turns away for a tick and
    back (on different ticks for different viewers), with non-zero
    backgrounds and a ragged frame; every frame is compared with the oracle."""
    specs = [(300, 64, 48), (2000, 61, 37), (50, 7, 5)]
    ticks = 2 * len(_VIEWS)
    view = lambda v, k: _VIEWS[(k + v) % len(_VIEWS)]   # noqa: E731
    with Server(SHARED_N, "f32", SHARED_SEED, 0, float(AMP)) as srv:
        srv.shared_points().copy_(torch.from_numpy(_shared()))
        srv.set_shared_color(SHARED_COLOR)
        ids = []
        for v, (n, W, H) in enumerate(specs):
            ids.append(srv.add_viewer(**_viewer_args(v, n, W, H)))
            srv.viewer_points(ids[v]).copy_(torch.from_numpy(_private(v, n)))
        shared = _shared()
        priv = [_private(v, n) for v, (n, _, _) in enumerate(specs)]
        for k in range(ticks):
            for v, vid in enumerate(ids):
                eye, target = view(v, k)
                srv.set_camera(vid, eye, target, UP, 60.0, 0.1, 100.0)
            srv.tick(roundtrip=roundtrip)
            torch.cuda.synchronize()
            oracle.displace_f32(shared, SHARED_SEED, 0, k, AMP)
            for v, (n, W, H) in enumerate(specs):
                oracle.displace_f32(priv[v], 3000 + v, 1 + v, k, AMP)
                rgba, keys, f = srv.frame(ids[v])
                assert f == k + 1
                both = np.concatenate([shared, priv[v]])
                colors = np.concatenate([np.full(SHARED_N, SHARED_COLOR, np.uint32),
                                         np.full(n, 0xFF000000 | v, np.uint32)])
                eye, target = view(v, k)
                M = oracle.camera_f32(eye, target, UP, 60.0, W / H, 0.1, 100.0)
                want = oracle.render(both, "f32", M, W, H, np.float32(0.1), np.float32(100.0), colors, 0, 0x10 + v)
                assert np.array_equal(keys.cpu().numpy().reshape(-1).view(np.uint64), want[0]), (k, v)
                assert np.array_equal(rgba.cpu().numpy().reshape(-1).view(np.uint32), want[1]), (k, v)
