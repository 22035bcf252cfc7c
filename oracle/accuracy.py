"""Accuracy of a stored GPU result against the FP64 oracle (test
infrastructure, like the rest of this package: only the tests, the smoke
check and the bench's CPU-side legs use it).

The precision pattern of the build stores positions in FP32, binary16 or
bfloat16 and computes in FP32; its accuracy is stated against the same step
taken in FP64 from the same stored input (one Brownian step, Sec. 4.1).  Two
figures come out of it:

- the relative error of every coordinate after one step,
  |x_gpu - x_fp64| / max(|x_fp64|, 2^-14), its maximum and RMS;
- pixel agreement between the GPU frame and the frame the oracle renders
  from the FP64 positions (rounded once to FP32), over all pixels and over
  the pixels covered in either frame.

With one colour for every point (Sec. 4.1), the RGBA frame is the coverage
mask, so two frames differ exactly on pixels that one covers and the other
does not.  A point whose stored coordinates differ from the FP64 ones by at
most eps per coordinate lands somewhere in a small screen box around its
FP64 projection; coverage can differ only on pixels that such a box touches
without containing it whole.  `at_risk_pixels` builds that set from the
stated rounding bound alone, so "every disagreeing pixel is at risk" is a
check derived from the bound, not from the measured frames.
"""
from __future__ import annotations

import numpy as np

from . import EMPTY_KEY, camera_f32, camera_f64, displace_f64, from_storage, render

# Largest relative rounding error of storing the FP32 step in the storage
# type, for values at or above binary16's smallest normal 2^-14: half an ulp,
# 2^-p relative with p significand bits (11 for binary16, 8 for bfloat16);
# FP32 storage keeps the FP32 value, so it adds nothing.  Below the floor the
# bound is absolute, floor * unit (binary16's subnormal half-spacing 2^-25).
UNIT_ROUNDOFF = {"f32": 0.0, "f16": 2.0**-11, "bf16": 2.0**-8}
REL_FLOOR = 2.0**-14

# Screen-space slack (pixels) for evaluating the projection in FP32 rather
# than exactly, in both frames.  For the benchmark cameras every term of the
# clip-space dot products is below 4 in magnitude, so each of about ten
# roundings (at most 2^-24 relative) moves ndc by under 1e-6 in all, and a
# screen coordinate (ndc scaled by at most 1920 px) by under 2e-3 px; 0.01 px
# is a fivefold margin.
FP32_PROJECTION_SLACK_PX = 0.01

# Largest half-width (pixels) of a screen box the at-risk check handles; a box
# narrower than 2h touches at most 2h + 1 pixels per axis, all of which it
# marks.  Binary16 boxes at 3840x2160 reach about 0.7 px; bfloat16 ones are
# eight times wider and fall outside the check.
MAX_HALF_BOX_PX = 1.5


def coordinate_bound(p_ref: np.ndarray, dtype: str, amplitude: float) -> np.ndarray:
    """Bound on |x_gpu - x_ref| per coordinate after one step of the given
    amplitude a.  The FP32 step rounds the offset (at most 2^-24 |a|) and
    the sum (2^-24 |x|); the reference, the FP64 step (exact up to 2^-53),
    is rounded once to FP32 (2^-24 |x|); the GPU value is then stored
    (UNIT_ROUNDOFF[dtype] relative, floored at 2^-14).  Clamping to [0, 1]
    moves no value further apart.  The FP32 terms are doubled as margin for
    the products of small errors:
    eps = u max(|x|, 2^-14) + 2^-22 |x| + 2^-23 |a|."""
    x = np.abs(p_ref)
    return UNIT_ROUNDOFF[dtype] * np.maximum(x, REL_FLOOR) + 2.0**-22 * x + 2.0**-23 * abs(float(amplitude))


def relative_error(got: np.ndarray, ref: np.ndarray) -> dict:
    rel = np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), REL_FLOOR)
    return {"max_rel": float(rel.max()), "rms_rel": float(np.sqrt(np.mean(rel * rel)))}


def at_risk_pixels(p_ref: np.ndarray, eps: np.ndarray, M64: np.ndarray, W: int, H: int, znear: float,
                   zfar: float, chunk: int = 1 << 23):
    """(may, must): boolean W*H masks, or None when some point's screen box
    has a half-width of MAX_HALF_BOX_PX or more (the check then does not
    apply).  `must` marks pixels that a point's
    whole screen box lies in (covered in both frames); `may` marks every
    pixel a box touches.  A pixel outside `may` is empty in both frames.

    For clip coordinates c = M p and a change |dp_k| <= eps_k, the changes of
    cx, cy and cw are bounded by a_r = sum_k |M_rk| eps_k, and
    |d(cx/cw)| <= (a_x |cw| + |cx| a_w) / (|cw| (|cw| - a_w)), exactly (no
    linearisation), whenever |cw| > a_w.  Screen x is (1 + cx/cw) W/2 and
    screen y is (1 - cy/cw) H/2.  Points whose depth interval can reach a
    clipping plane, or whose box reaches outside the frame, only add to
    `may`, never to `must`."""
    may = np.zeros(W * H, bool)
    must = np.zeros(W * H, bool)
    Mabs = np.abs(M64)
    for s in range(0, p_ref.shape[0], chunk):
        p = p_ref[s:s + chunk].astype(np.float64)
        e = eps[s:s + chunk].astype(np.float64)
        cx = p @ M64[0, :3] + M64[0, 3]
        cy = p @ M64[1, :3] + M64[1, 3]
        cw = p @ M64[3, :3] + M64[3, 3]
        ax = e @ Mabs[0, :3]
        ay = e @ Mabs[1, :3]
        aw = e @ Mabs[3, :3]
        ok = (cw - aw > znear) & (cw + aw < zfar)        # drawn in both frames whatever the change
        maybe = (cw + aw > znear) & (cw - aw < zfar)     # drawn in at least one frame
        cwa = np.abs(cw)
        with np.errstate(divide="ignore", invalid="ignore"):
            den = cwa * (cwa - aw)
            dx = 0.5 * W * (ax * cwa + np.abs(cx) * aw) / den + FP32_PROJECTION_SLACK_PX
            dy = 0.5 * H * (ay * cwa + np.abs(cy) * aw) / den + FP32_PROJECTION_SLACK_PX
            sx = 0.5 * W * (1.0 + cx / cw)
            sy = 0.5 * H * (1.0 - cy / cw)
        good = maybe & (cwa > aw) & np.isfinite(dx) & np.isfinite(dy) & (dx < MAX_HALF_BOX_PX) & \
            (dy < MAX_HALF_BOX_PX)
        if np.any(maybe & ~good):
            return None          # a box may span more pixels than this check walks: it does not apply
        x0, x1 = np.floor(sx - dx), np.floor(sx + dx)
        y0, y1 = np.floor(sy - dy), np.floor(sy + dy)
        span = int(2 * MAX_HALF_BOX_PX) + 1          # a box narrower than 2h spans at most 2h + 1 pixels
        for ox in range(span):
            for oy in range(span):
                xs, ys = x0 + ox, y0 + oy
                inside = good & (xs <= x1) & (ys <= y1) & (xs >= 0) & (xs < W) & (ys >= 0) & (ys < H)
                may[(ys[inside] * W + xs[inside]).astype(np.int64)] = True
        whole = good & ok & (x0 == x1) & (y0 == y1) & (x0 >= 0) & (x0 < W) & (y0 >= 0) & (y0 < H)
        must[(y0[whole] * W + x0[whole]).astype(np.int64)] = True
    return may, must


def step_accuracy(stored_before: np.ndarray, dtype: str, got_after: np.ndarray, rgba_gpu: np.ndarray, seed: int,
                  cloud: int, step: int, amplitude: float, eye, target, up, fovy_deg: float, W: int, H: int,
                  znear: float, zfar: float, color: int = 0xFFFFFFFF, background: int = 0,
                  pixels: bool = True) -> dict:
    """Accuracy of one GPU step against the FP64 oracle.

    stored_before: the positions the GPU step started from (storage form);
    got_after: the GPU's positions after the step (storage form); rgba_gpu:
    the GPU frame of that step (W*H uint32, one colour).  The FP64 oracle
    takes the same step from the same stored input; its positions, rounded
    once to FP32, are rendered by the oracle with the FP32 matrix of the same
    camera."""
    seg = {"stored_before": stored_before, "got_after": got_after, "seed": seed, "cloud": cloud, "step": step,
           "amplitude": amplitude}
    return segments_accuracy([seg], dtype, rgba_gpu, eye, target, up, fovy_deg, W, H, znear, zfar, color,
                             background, pixels)


def segments_accuracy(segments, dtype: str, rgba_gpu: np.ndarray, eye, target, up, fovy_deg: float, W: int,
                      H: int, znear: float, zfar: float, color: int = 0xFFFFFFFF, background: int = 0,
                      pixels: bool = True) -> dict:
    """As step_accuracy for a frame drawn from several clouds, each stepped
    with its own Philox key, counter word and step (a viewer's frame: the
    shared cloud, then its private cloud, point ids following on in that
    order).  Each segment is a dict with stored_before, got_after, seed,
    cloud, step and amplitude."""
    refs, gots, eps = [], [], []
    for sg in segments:
        p64 = from_storage(sg["stored_before"], dtype).astype(np.float64)
        displace_f64(p64, sg["seed"], sg["cloud"], sg["step"], float(np.float32(sg["amplitude"])))
        refs.append(p64)
        gots.append(from_storage(sg["got_after"], dtype))
        p32 = p64.astype(np.float32).astype(np.float64)
        eps.append(coordinate_bound(p32, dtype, sg["amplitude"]))
    p64 = np.concatenate(refs)
    out = relative_error(np.concatenate(gots), p64)
    out["gate_2^-10"] = bool(out["max_rel"] <= 2.0**-10)
    if not pixels:
        return out
    M32 = camera_f32(eye, target, up, fovy_deg, W / H, znear, zfar)
    keys64, rgba64 = render(p64.astype(np.float32), "f32", M32, W, H, np.float32(znear), np.float32(zfar),
                            color=color, background=background)
    rgba_gpu = np.asarray(rgba_gpu).reshape(-1)
    cov_ref = keys64 != EMPTY_KEY
    cov_gpu = rgba_gpu != np.uint32(background)
    differ = rgba_gpu != rgba64
    union = cov_ref | cov_gpu
    # the bound is evaluated with the FP32 matrix as exact numbers, the matrix both frames use
    p_ref = p64.astype(np.float32).astype(np.float64)
    masks = at_risk_pixels(p_ref, np.concatenate(eps), M32.astype(np.float64), W, H, float(np.float32(znear)),
                           float(np.float32(zfar)))
    n_union = int(union.sum())
    out.update({
        "pixels_all_agree": float(1.0 - differ.mean()),
        "pixels_covered_either": n_union,
        "pixels_covered_agree": float(1.0 - differ[union].sum() / max(n_union, 1)),
        "pixels_at_risk": None, "covered_agree_bound": None, "differing_outside_risk": None,
    })
    if masks is not None:
        at_risk = masks[0] & ~masks[1]
        out.update({
            "pixels_at_risk": int(at_risk.sum()),
            "covered_agree_bound": float(1.0 - (at_risk & union).sum() / max(n_union, 1)),
            "differing_outside_risk": int((differ & ~at_risk).sum()),
        })
    return out


def camera_pair(eye, target, up, fovy_deg, W, H, znear, zfar):
    """FP64 and FP32 matrices of one camera (for callers that need both)."""
    return (camera_f64(eye, target, up, fovy_deg, W / H, znear, zfar),
            camera_f32(eye, target, up, fovy_deg, W / H, znear, zfar))
