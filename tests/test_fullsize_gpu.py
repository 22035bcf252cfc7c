"""Parity at the benchmark sizes, in the launch configuration the bench
times (the library defaults).

4M-point 1920x1080 orbit: the first frames are compared whole against the
oracle; after 1000 frames, sampled points are followed one by one by the
oracle and the frame is checked through its winners.  64M-point 16-cluster
Gaussian mixture at 3840x2160: one whole frame in FP32, binary16 and
bfloat16 storage against the oracle, plus the accuracy gates of each storage
type against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from oracle import accuracy
from paper_2504_20937_b300 import inputs

from ._harness import CENTRE, UP, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2_start():
    sc = inputs.C2
    return sc, inputs.encode(sc.positions(), "f32")


def test_c2_first_frames_bit_exact(c2_start):
    sc, stored = c2_start
    args = (stored, "f32", sc.W, sc.H, sc.philox_seed, sc.amplitude, 3, sc.eye)
    g = gpu_run(*args)
    o = oracle_run(*args)
    assert np.array_equal(g[0], o[0])
    assert np.array_equal(g[1], o[1])
    assert np.array_equal(g[2], o[2])


def test_c2_1000_frames_sampled(c2_start):
    sc, stored = c2_start
    frames = sc.frames
    gpos, gkeys, grgba, _ = gpu_run(stored, "f32", sc.W, sc.H, sc.philox_seed, sc.amplitude, frames, sc.eye)
    # invariants of the whole state
    assert gpos.shape == stored.shape and np.all(np.isfinite(gpos))
    assert gpos.min() >= 0.0 and gpos.max() <= 1.0
    covered = gkeys != oracle.EMPTY_KEY
    assert np.array_equal(grgba[covered], np.full(covered.sum(), sc.color, np.uint32))
    assert np.all(grgba[~covered] == sc.background)
    ids = (gkeys[covered] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert ids.max() < sc.n
    # sampled points followed one by one through all frames by the oracle
    rng = np.random.default_rng(7)
    sample = np.unique(np.concatenate([rng.choice(sc.n, 3000, replace=False),
                                       rng.choice(ids, 3000, replace=False), [0, sc.n - 1]]))
    sample = sample.astype(np.uint32)
    pos = stored[sample].copy()
    for f in range(frames):
        oracle.displace_ids_f32(pos, sample, sc.philox_seed, 0, f, np.float32(sc.amplitude))
    np.testing.assert_array_equal(gpos[sample], pos)
    # every sampled point: its key at its pixel is >= the stored minimum, and
    # equal exactly when it is that pixel's winner
    M = oracle.camera_f32(sc.eye(frames - 1), CENTRE, UP, sc.fovy_deg, sc.aspect, sc.znear, sc.zfar)
    px, w = oracle.project_f32(M, pos, sc.W, sc.H, np.float32(sc.znear), np.float32(sc.zfar))
    on = px != 0xFFFFFFFF
    key = (w.view(np.uint32).astype(np.uint64) << np.uint64(32)) | sample.astype(np.uint64)
    assert np.all(gkeys[px[on]] <= key[on])
    winner = (gkeys[px[on]] & np.uint64(0xFFFFFFFF)) == sample[on]
    assert np.array_equal(gkeys[px[on]][winner], key[on][winner])
    assert winner.sum() > 1000                 # the sampled winners were checked


@pytest.fixture(scope="module")
def c3_start():
    sc = inputs.C3
    return sc, sc.positions()


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_c3_frame_bit_exact(c3_start, dtype):
    sc, pos64 = c3_start
    stored = inputs.encode(pos64, dtype)
    args = (stored, dtype, sc.W, sc.H, sc.philox_seed, sc.amplitude, 1, sc.eye)
    g = gpu_run(*args)
    o = oracle_run(*args)
    assert np.array_equal(g[0], o[0])
    bad = np.count_nonzero(g[1] != o[1])
    assert bad == 0, f"{bad} pixels differ"
    assert np.array_equal(g[2], o[2])


def _depths(keys, W, H):
    d = (keys >> np.uint64(32)).astype(np.uint32).view(np.float32).astype(np.float64)
    d[keys == oracle.EMPTY_KEY] = np.inf
    return d.reshape(H, W)


def _depth_agreement(keys_a, keys_b, W, H, neighbourhood):
    """Share of pixels where both depth maps are empty or agree within 2^-9
    relative; with `neighbourhood`, each map is first replaced by its 3x3
    minimum (a point may move by up to one pixel)."""
    da, db = _depths(keys_a, W, H), _depths(keys_b, W, H)
    if neighbourhood:
        def mins(d):
            p = np.pad(d, 1, constant_values=np.inf)
            return np.minimum.reduce([p[y:y + H, x:x + W] for y in range(3) for x in range(3)])
        da, db = mins(da), mins(db)
    both_empty = np.isinf(da) & np.isinf(db)
    with np.errstate(invalid="ignore"):
        close = np.abs(da - db) <= 2.0**-9 * db
    return float(np.mean(both_empty | close))


def test_c3_storage_accuracy_gates(c3_start):
    """Each storage type against the FP64 oracle stepped from the same stored
    input (oracle/accuracy.py).

    binary16: after one step every coordinate is within 2^-10 relative
    (floor 2^-14) of FP64, and >= 99.9% of framebuffer pixels (RGBA8) equal
    those of the frame rendered from the FP64 positions.  Over the pixels
    covered in either frame agreement is lower, because binary16 rounding
    moves a point by up to 2^-11 relative per coordinate (about 0.23 px at
    3840x2160 and distance 2) and a sparsely covered pixel can lose its only
    point to a neighbour.  That tolerance is derived from the bound, not
    measured: a pixel can change only if some point's screen box (its FP64
    projection widened by the bound) touches it without containing it, and
    the gate is that no pixel outside that at-risk set differs, which also
    bounds the covered-pixel agreement from below.  FP32 storage passes the
    same checks with its own rounding bound; bfloat16 boxes reach a pixel,
    so its figures are reported only.  Depth-aware agreement is reported
    beside them."""
    sc, pos64 = c3_start
    report = {}
    for dtype in ("f32", "f16", "bf16"):
        stored = inputs.encode(pos64, dtype)
        g = gpu_run(stored, dtype, sc.W, sc.H, sc.philox_seed, sc.amplitude, 1, sc.eye)
        rep = accuracy.step_accuracy(stored, dtype, g[0], g[2], sc.philox_seed, 0, 0, sc.amplitude, sc.eye(0),
                                     CENTRE, UP, sc.fovy_deg, sc.W, sc.H, sc.znear, sc.zfar, sc.color,
                                     sc.background)
        if dtype != "f32":
            p64 = oracle.from_storage(stored, dtype).astype(np.float64)
            oracle.displace_f64(p64, sc.philox_seed, 0, 0, float(np.float32(sc.amplitude)))
            M = oracle.camera_f32(sc.eye(0), CENTRE, UP, sc.fovy_deg, sc.aspect, sc.znear, sc.zfar)
            k64, _ = oracle.render(p64.astype(np.float32), "f32", M, sc.W, sc.H, np.float32(sc.znear),
                                   np.float32(sc.zfar))
            rep["depth_agree_strict"] = _depth_agreement(g[1], k64, sc.W, sc.H, False)
            rep["depth_agree_3x3"] = _depth_agreement(g[1], k64, sc.W, sc.H, True)
        report[dtype] = rep
    print("storage vs FP64 oracle:", report)
    for dtype in ("f32", "f16"):
        r = report[dtype]
        assert r["max_rel"] <= 2.0**-10
        assert r["pixels_all_agree"] >= 0.999
        assert r["differing_outside_risk"] == 0, f"{dtype}: pixels outside the at-risk set differ"
        assert r["pixels_covered_agree"] >= r["covered_agree_bound"]
    # FP32: |error| <= 2^-24 (|x| + |a|), so relative to max(|x|, 2^-14) at most 2^-24 (1 + 5e-4 2^14) < 2^-20
    assert report["f32"]["max_rel"] <= 2.0**-20
    assert report["bf16"]["pixels_at_risk"] is None      # boxes of a pixel or more: reported only
