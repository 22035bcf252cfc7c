"""Pins of oracle/accuracy.py, the FP64 accuracy figures reported for every
storage type: hand cases of the screen-box rule, and brute force on small
clouds (random positions inside the stated rounding bound, rendered by the
oracle, never differ from the reference frame outside the at-risk pixels)."""
import numpy as np

import oracle
from oracle import accuracy
from paper_2504_20937_b300 import inputs

CEN = (0.5, 0.5, 0.5)
UP = (0.0, 1.0, 0.0)


def _masks(points, eps, W=64, H=48, eye=(0.5, 0.5, 2.5)):
    M32 = oracle.camera_f32(eye, CEN, UP, 60.0, W / H, 0.1, 100.0)
    p = np.asarray(points, np.float64)
    return accuracy.at_risk_pixels(p, np.full_like(p, eps), M32.astype(np.float64), W, H, 0.1, 100.0), M32


def test_centre_point_with_tiny_error_covers_one_pixel_for_sure():
    # the cloud centre projects to ndc (0, 0): screen (W/2, H/2), a pixel corner; move it a quarter pixel in
    # so it sits inside pixel (32, 24) with a margin of a quarter pixel on each side
    W, H = 64, 48
    M = oracle.camera_f32((0.5, 0.5, 2.5), CEN, UP, 60.0, W / H, 0.1, 100.0).astype(np.float64)
    # world offset of a quarter pixel at depth 2: d(sx)/dx = W/2 * M[0,0] / w
    q = 0.25 / (0.5 * W * M[0, 0] / 2.0)
    (may, must), _ = _masks([[0.5 + q, 0.5 - q * M[0, 0] / M[1, 1], 0.5]], 1e-9)
    assert must.sum() == 1 and may.sum() == 1
    assert np.flatnonzero(must)[0] == 24 * W + 32


def test_point_on_a_pixel_edge_is_at_risk_on_both_sides():
    (may, must), _ = _masks([[0.5, 0.6, 0.5]], 1e-6)          # x exactly on the vertical edge sx = W/2
    assert must.sum() == 0 and may.sum() == 2


def test_wide_boxes_are_refused():
    # at this size a world unit at depth 2 is about 21 px, so an error of 0.1 gives a box about 2 px wide
    assert _masks([[0.5, 0.5, 0.5]], 1e-1)[0] is None
    assert _masks([[0.5, 0.5, 0.5]], 3e-2)[0] is not None


def test_perturbations_inside_the_bound_differ_only_on_at_risk_pixels():
    """Boxes of a few tenths of a pixel up to more than a pixel (the binary16
    bound scaled up to this small frame), so that many points straddle pixel
    edges."""
    rng = np.random.default_rng(11)
    W, H = 96, 64
    # the last two: a uniform cloud seen from close by, so points reach the frame's edges, where the depth
    # term of the bound (|cx| a_w) matters most
    for trial, scale in enumerate([16.0, 8.0, 1.0, 12.0, 6.0, 3.0, 60.0, 50.0]):
        if trial < 4 or trial >= 6:
            pos = inputs.gaussian_mixture_cloud(3000, 90 + trial, components=2, sigma=0.05)
            eye = inputs.orbit_eye(17 * trial, 1.0)
        else:
            pos = inputs.uniform_cloud(6000, 90 + trial)
            eye = inputs.orbit_eye(17 * trial, 1.0, radius=1.3)
        pos = inputs.encode(pos, "f32").astype(np.float64)
        M32 = oracle.camera_f32(eye, CEN, UP, 60.0, W / H, 0.1, 100.0)
        eps = scale * accuracy.coordinate_bound(pos, "f16", 5e-4)
        masks = accuracy.at_risk_pixels(pos, eps, M32.astype(np.float64), W, H, 0.1, 100.0)
        assert masks is not None
        may, must = masks
        assert not np.any(must & ~may)
        _, ref = oracle.render(pos.astype(np.float32), "f32", M32, W, H, np.float32(0.1), np.float32(100.0))
        changed = 0
        for _ in range(20):
            moved = pos + rng.uniform(-1.0, 1.0, pos.shape) * eps
            # also the extreme corners of the box, where a crossing is most likely
            moved[::3] = pos[::3] + np.sign(rng.standard_normal(pos[::3].shape)) * eps[::3]
            _, got = oracle.render(moved.astype(np.float32), "f32", M32, W, H, np.float32(0.1),
                                   np.float32(100.0))
            differ = got != ref
            changed += int(differ.sum())
            assert not np.any(differ & ~(may & ~must)), "a pixel outside the at-risk set changed"
            assert np.all(got[must] == 0xFFFFFFFF) and np.all(got[~may] == 0)
        if scale > 1.0:
            assert changed > 0          # the perturbations did move points across pixel edges


def test_step_accuracy_of_the_oracle_itself_is_exact_in_fp32():
    # the FP32 oracle step against the FP64 one: within the FP32 rounding bound, frames differ only at risk
    W, H = 80, 60
    stored = inputs.encode(inputs.uniform_cloud(5000, 3), "f32")
    after = stored.copy()
    oracle.displace_f32(after, 7, 0, 0, np.float32(5e-4))
    M32 = oracle.camera_f32((0.5, 0.5, 2.5), CEN, UP, 60.0, W / H, 0.1, 100.0)
    _, rgba = oracle.render(after, "f32", M32, W, H, np.float32(0.1), np.float32(100.0))
    rep = accuracy.step_accuracy(stored, "f32", after, rgba, 7, 0, 0, 5e-4, (0.5, 0.5, 2.5), CEN, UP, 60.0, W, H,
                                 0.1, 100.0)
    # |error| <= 2^-24 (|x| + |a|): relative to max(|x|, 2^-14) at most 2^-24 (1 + 5e-4 * 2^14) < 2^-20
    assert rep["max_rel"] <= 2.0**-20
    assert rep["differing_outside_risk"] == 0
    assert rep["pixels_covered_agree"] >= rep["covered_agree_bound"]
