"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle (oracle/mmr_oracle.c) against a published value,
a closed form, a library routine, a brute-force search or an invariant, so a
dropped term, a wrong sign, a wrong index or a transposed operand in the
oracle fails at least one of them.  No GPU is used here.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)
# --------------------------------------------------------------------------
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat_rows())
def test_philox_known_answers(ctr, key, want):
    assert list(oracle.philox4x32_10(ctr, key)) == want


def test_philox_counter_words_all_matter():
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for j in range(4):
        ctr = [1, 2, 3, 4]
        ctr[j] ^= 1
        assert not np.array_equal(oracle.philox4x32_10(ctr, [5, 6]), base)
    for j in range(2):
        key = [5, 6]
        key[j] ^= 1
        assert not np.array_equal(oracle.philox4x32_10([1, 2, 3, 4], key), base)


# --------------------------------------------------------------------------
# Displacement (Sec. 4.1): draw mapping, worked example, statistics,
# invariants, FP64 rounding bound.
# --------------------------------------------------------------------------
def test_displacement_worked_example_from_kat():
    """Seed 0, cloud 0, point 0, step 0 uses counter (0,0,0,0) and key (0,0),
    whose Philox output is the first published known-answer vector.  Its top
    24 bits give u; one step from p = 0.5 with a = 1e-3 moves each axis by
    a (2u - 1), computed here by hand in exact rationals."""
    _, _, want = _kat_rows()[0]
    pos = np.full((1, 3), 0.5, np.float32)
    a = np.float32(1e-3)
    oracle.displace_f32(pos, 0, 0, 0, a)
    for k in range(3):
        u = (want[k] >> 8) / 2.0**24                 # exact in float64
        exact = 0.5 + float(a) * (2.0 * u - 1.0)     # within 1 ulp of the two FP32 roundings
        assert abs(float(pos[0, k]) - exact) <= 2.0**-24 + 2.0**-30
    # axis x: top 24 bits 0x6627e8 < 2^23, so the point moves towards 0
    assert pos[0, 0] < 0.5


def test_displacement_statistics():
    """Offsets t = (p' - p)/a are uniform on [-1, 1): mean 0, variance 1/3,
    axes uncorrelated, consecutive steps uncorrelated."""
    n = 200_000
    a = np.float32(1e-3)
    pos = np.full((n, 3), 0.5, np.float32)
    oracle.displace_f32(pos, 11, 0, 0, a)
    t1 = (pos.astype(np.float64) - 0.5) / float(a)
    start = pos.copy()
    oracle.displace_f32(pos, 11, 0, 1, a)
    t2 = (pos.astype(np.float64) - start) / float(a)
    for t in (t1, t2):
        assert np.all(np.abs(t) <= 1.0 + 1e-3)
        sd = math.sqrt(1 / 3) / math.sqrt(n)
        assert np.all(np.abs(t.mean(axis=0)) < 5 * sd)
        assert np.all(np.abs(t.var(axis=0) - 1 / 3) < 0.01)
        c = np.corrcoef(t.T)
        assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 0.02)
    assert np.all(np.abs([np.corrcoef(t1[:, k], t2[:, k])[0, 1] for k in range(3)]) < 0.02)


def test_displacement_depends_on_point_step_cloud_seed():
    base = np.full((64, 3), 0.5, np.float32)
    outs = []
    for (seed, cloud, step) in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1 << 32, 0, 0)]:
        p = base.copy()
        oracle.displace_f32(p, seed, cloud, step, np.float32(1e-3))
        outs.append(p)
    for i in range(len(outs)):
        for j in range(i + 1, len(outs)):
            assert not np.array_equal(outs[i], outs[j])
    # different points draw different offsets
    assert len(np.unique(outs[0][:, 0])) > 60


def test_displacement_invariants_and_clamp():
    n = 50_000
    pos = inputs.encode(inputs.uniform_cloud(n, 7), "f32")
    pos[:100] = 0.0
    pos[100:200] = 1.0
    a = np.float32(0.05)                 # large steps so the clamp is exercised
    for s in range(20):
        oracle.displace_f32(pos, 3, 0, s, a)
    assert pos.shape == (n, 3)
    assert np.all(np.isfinite(pos))
    assert pos.min() >= 0.0 and pos.max() <= 1.0
    assert (pos == 0.0).sum() > 0 and (pos == 1.0).sum() > 0


def test_displacement_clamps_non_finite_and_out_of_box_inputs():
    """Reading 3 (clamp) on inputs a caller may write: NaN and -inf go to 0,
    +inf and anything that stays above 1 after the step to 1, anything below
    0 to 0; an in-box coordinate moves by at most a.  The same with a = 0:
    the clamp still applies."""
    vals = np.array([np.nan, np.inf, -np.inf, 1e30, -1e30, 2.0, -2.0, 0.5], np.float32)
    want = np.array([0, 1, 0, 1, 0, 1, 0], np.float32)
    for a in (np.float32(0.0), np.float32(1e-3)):
        pos = np.repeat(vals[:, None], 3, axis=1)
        oracle.displace_f32(pos, 9, 0, 0, a)
        assert np.array_equal(pos[:7], np.repeat(want[:, None], 3, axis=1)), a
        assert np.all(np.abs(pos[7] - np.float32(0.5)) <= a), a


def test_displacement_fp32_within_rounding_bound_of_fp64():
    """Each FP32 step rounds twice (a*t and p+d), each at most half an ulp of a
    value below 1 + a, so after s steps |p32 - p64| <= s (1 + a) 2^-24."""
    n = 20_000
    p32 = inputs.encode(inputs.uniform_cloud(n, 8), "f32")
    p64 = p32.astype(np.float64)
    a = np.float32(1e-3)
    steps = 100
    for s in range(steps):
        oracle.displace_f32(p32, 5, 0, s, a)
        oracle.displace_f64(p64, 5, 0, s, float(a))
    err = np.abs(p32.astype(np.float64) - p64).max()
    assert err <= steps * (1 + float(a)) * 2.0**-24
    assert err > 0.0                      # the two do round differently


def test_displacement_ids_matches_full_cloud():
    n = 4096
    pos = inputs.encode(inputs.uniform_cloud(n, 9), "f32")
    ids = np.array([0, 1, 17, 4095, 2048], np.uint32)
    sub = pos[ids].copy()
    for s in range(5):
        oracle.displace_f32(pos, 21, 2, s, np.float32(1e-3))
        oracle.displace_ids_f32(sub, ids, 21, 2, s, np.float32(1e-3))
    assert np.array_equal(sub, pos[ids])


# --------------------------------------------------------------------------
# Storage conversions: every binary32 bit pattern against torch's RNE casts.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_narrowing_exhaustive_against_torch(fmt):
    tdt = torch.float16 if fmt == "f16" else torch.bfloat16
    to = oracle.f32_to_f16 if fmt == "f16" else oracle.f32_to_bf16
    chunk = 1 << 26
    base = np.arange(chunk, dtype=np.uint32)
    for start in range(0, 1 << 32, chunk):
        bits = base + np.uint32(start)
        x = bits.view(np.float32)
        got = to(x)
        want = torch.from_numpy(x).to(tdt).view(torch.int16).numpy().view(np.uint16)
        bad = got != want
        if bad.any():
            # only NaN inputs may differ (payload), and they must stay NaN
            idx = np.nonzero(bad)[0]
            assert np.all(np.isnan(x[idx])), f"{fmt} mismatch at {bits[idx[0]]:#010x}"
            back = oracle.f16_to_f32(got[idx]) if fmt == "f16" else oracle.bf16_to_f32(got[idx])
            assert np.all(np.isnan(back))


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_widening_exhaustive_against_torch(fmt):
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    got = (oracle.f16_to_f32 if fmt == "f16" else oracle.bf16_to_f32)(bits)
    tdt = torch.float16 if fmt == "f16" else torch.bfloat16
    want = torch.from_numpy(bits.view(np.int16)).view(tdt).to(torch.float32).numpy()
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint32), want[~nan].view(np.uint32))


def test_h16_step_within_storage_gate_of_fp64():
    """One step with 16-bit storage against the FP64 step from the same stored
    input: binary16 within 2^-10 relative (floor 2^-14); bfloat16 reported."""
    n = 50_000
    for fmt in ("f16", "bf16"):
        stored = inputs.encode(inputs.uniform_cloud(n, 12), fmt)
        start64 = oracle.from_storage(stored, fmt).astype(np.float64)
        oracle.displace_h16(stored, fmt, 4, 0, 0, np.float32(5e-4))
        p64 = start64.copy()
        oracle.displace_f64(p64, 4, 0, 0, float(np.float32(5e-4)))
        got = oracle.from_storage(stored, fmt).astype(np.float64)
        rel = np.abs(got - p64) / np.maximum(np.abs(p64), 2.0**-14)
        if fmt == "f16":
            assert rel.max() <= 2.0**-10
        else:
            assert rel.max() <= 2.0**-7      # bfloat16: half an ulp of 8 bits


def test_bf16_small_steps_do_not_move_upper_half():
    """bfloat16 spacing on [1/2, 1) is 2^-8; a step of |d| <= 5e-4 is below half
    of it, so coordinates there never move (a finding reported, not hidden)."""
    n = 10_000
    pos64 = 0.5 + 0.49 * inputs.uniform_cloud(n, 13)
    stored = inputs.encode(pos64, "bf16")
    before = stored.copy()
    for s in range(10):
        oracle.displace_h16(stored, "bf16", 1, 0, s, np.float32(5e-4))
    assert np.array_equal(stored, before)


# --------------------------------------------------------------------------
# Camera and projection: closed forms and the FP64 twin.
# --------------------------------------------------------------------------
EYE = (0.5, 0.5, 2.5)
CEN = (0.5, 0.5, 0.5)
UP = (0.0, 1.0, 0.0)


def test_camera_closed_form_default_view():
    aspect = 1920 / 1080
    M = oracle.camera_f64(EYE, CEN, UP, 60.0, aspect, 0.1, 100.0)
    ndc, w, ok = oracle.project_f64(M, np.array([CEN]), 0.1, 100.0)
    assert ok[0] and abs(w[0] - 2.0) < 1e-12 and np.all(np.abs(ndc[0]) < 1e-12)
    half_w = math.tan(math.radians(30.0)) * 2.0 * aspect   # half-width of view at distance 2
    half_h = math.tan(math.radians(30.0)) * 2.0
    pts = np.array([[0.5 + half_w, 0.5, 0.5], [0.5, 0.5 + half_h, 0.5], [0.5, 0.5, 1.5]])
    ndc, w, ok = oracle.project_f64(M, pts, 0.1, 100.0)
    assert abs(ndc[0, 0] - 1.0) < 1e-12 and abs(ndc[0, 1]) < 1e-12
    assert abs(ndc[1, 1] - 1.0) < 1e-12 and abs(ndc[1, 0]) < 1e-12
    assert abs(w[2] - 1.0) < 1e-12                     # w is distance along the view axis
    # view rows are orthonormal; the w row is -(view z row)
    R = M[[0, 1, 3], :3] / np.array([[1 / math.tan(math.radians(30)) / aspect],
                                     [1 / math.tan(math.radians(30))], [1.0]])
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)


def test_camera_side_view_closed_form():
    """Eye on +x looking at the centre: screen right is -z, screen up is +y."""
    M = oracle.camera_f64((2.5, 0.5, 0.5), CEN, UP, 90.0, 1.0, 0.1, 100.0)
    ndc, w, ok = oracle.project_f64(M, np.array([[0.5, 0.5, 0.0], [0.5, 1.0, 0.5], [0.0, 0.5, 0.5]]),
                                    0.1, 100.0)
    # fov 90: ndc = offset / distance
    assert np.allclose(ndc[0], [0.5 / 2.0, 0.0], atol=1e-12)
    assert np.allclose(ndc[1], [0.0, 0.5 / 2.0], atol=1e-12)
    assert np.allclose(w, [2.0, 2.0, 2.5], atol=1e-12)


def test_camera_f32_is_one_rounding():
    M64 = oracle.camera_f64(EYE, CEN, UP, 60.0, 1.0, 0.1, 100.0)
    M32 = oracle.camera_f32(EYE, CEN, UP, 60.0, 1.0, 0.1, 100.0)
    assert np.array_equal(M32, M64.astype(np.float32))


def test_projection_fp32_vs_fp64_ndc():
    pts = inputs.encode(inputs.uniform_cloud(100_000, 14), "f32")
    for f in range(0, 1000, 97):
        eye = inputs.orbit_eye(f, 0.36)
        M64 = oracle.camera_f64(eye, CEN, UP, 60.0, 16 / 9, 0.1, 100.0)
        M32 = M64.astype(np.float32)
        _, w32, nd32 = oracle.project_f32(M32, pts, 1 << 20, 1 << 20, 0.1, 100.0, want_ndc=True)
        nd64, w64, ok = oracle.project_f64(M64, pts.astype(np.float64), 0.1, 100.0)
        assert ok.all()
        assert np.abs(nd32.astype(np.float64) - nd64).max() < 1e-5
        assert np.abs(w32.astype(np.float64) - w64).max() < 1e-5


def _plain_matrix():
    """cx = x, cy = y, w = z: ndc = (x/z, y/z)."""
    M = np.zeros((4, 4), np.float32)
    M[0, 0] = M[1, 1] = M[3, 2] = 1.0
    return M


def test_pixel_mapping_hand_cases():
    W, H = 8, 4
    M = _plain_matrix()
    eps = 1e-6
    pts = np.array([
        [-1.0, 1.0, 1.0],            # top-left corner -> pixel 0
        [1.0 - eps, -1.0 + eps, 1.0],  # bottom-right -> last pixel
        [1.0, 0.0, 1.0],             # sx == W -> outside
        [0.0, -1.0, 1.0],            # sy == H -> outside
        [0.0, 0.0, 1.0],             # centre -> (4, 2)
        [-0.76, 0.49, 1.0],          # sx = 0.96 -> col 0; sy = 1.02 -> row 1
        [0.0, 0.0, 0.1],             # w == near -> culled
        [0.0, 0.0, 100.0],           # w == far -> culled
        [0.0, 0.0, -1.0],            # behind -> culled
        [-2.0, 0.0, 2.0],            # ndc.x = -1 -> col 0
    ], np.float32)
    px, w = oracle.project_f32(M, pts, W, H, 0.1, 100.0)
    none = 0xFFFFFFFF
    assert list(px) == [0, W * H - 1, none, none, 2 * W + 4, 1 * W + 0, none, none, none, 2 * W + 0]
    assert w[0] == 1.0 and w[9] == 2.0


# --------------------------------------------------------------------------
# Splat and resolve: brute-force per-pixel search, order independence.
# --------------------------------------------------------------------------
def _brute_force_keys(pos32, M32, W, H, znear, zfar):
    px, w = oracle.project_f32(M32, pos32, W, H, znear, zfar)
    want = np.full(W * H, 0xFFFFFFFFFFFFFFFF, np.uint64)
    for p in range(W * H):
        hits = np.nonzero(px == p)[0]
        best = None
        for i in hits:                                   # smallest depth, then smallest id
            cand = (float(w[i]), int(i))
            if best is None or cand < best:
                best = cand
        if best is not None:
            dbits = int(np.array([best[0]], np.float32).view(np.uint32)[0])
            want[p] = (dbits << 32) | best[1]
    return want


@pytest.mark.parametrize("kind", ["uniform", "gmm"])
def test_splat_matches_brute_force(kind):
    W, H = 48, 32
    n = 3000
    pos64 = (inputs.uniform_cloud(n, 15) if kind == "uniform"
             else inputs.gaussian_mixture_cloud(n, 15, components=3, sigma=0.05))
    pos = inputs.encode(pos64, "f32")
    # duplicate some points exactly so equal depths meet at one pixel
    pos[2000:2100] = pos[100:200]
    M = oracle.camera_f32(EYE, CEN, UP, 60.0, W / H, 0.1, 100.0)
    keys = oracle.empty_keys(W, H)
    oracle.splat(pos, "f32", M, W, H, 0.1, 100.0, keys)
    assert np.array_equal(keys, _brute_force_keys(pos, M, W, H, 0.1, 100.0))
    # ties broke to the smaller id: none of the duplicates 2000..2099 wins
    ids = (keys[keys != oracle.EMPTY_KEY] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert not np.any((ids >= 2000) & (ids < 2100))


def test_splat_order_independent_and_conserves_points():
    W, H = 64, 64
    n = 4096
    pos = inputs.encode(inputs.gaussian_mixture_cloud(n, 16, components=2, sigma=0.05), "f32")
    M = oracle.camera_f32(EYE, CEN, UP, 60.0, 1.0, 0.1, 100.0)
    keys = oracle.empty_keys(W, H)
    oracle.splat(pos, "f32", M, W, H, 0.1, 100.0, keys)
    # shuffle the points, splat with ids mapped back through id_base per point
    perm = np.random.default_rng(0).permutation(n)
    keys2 = oracle.empty_keys(W, H)
    for j, i in enumerate(perm):
        oracle.splat(pos[i:i + 1], "f32", M, W, H, 0.1, 100.0, keys2, id_base=int(i))
    assert np.array_equal(keys, keys2)
    # every point lands somewhere or is off-frame; covered pixels hold a real
    # point's key and the number of covered pixels equals the distinct pixels hit
    px, w = oracle.project_f32(M, pos, W, H, 0.1, 100.0)
    hit = px[px != 0xFFFFFFFF]
    assert (keys != oracle.EMPTY_KEY).sum() == len(np.unique(hit))
    win = (keys[keys != oracle.EMPTY_KEY] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.array_equal(px[win], np.nonzero(keys != oracle.EMPTY_KEY)[0].astype(np.uint32))
    assert np.array_equal(w[win].view(np.uint32),
                          (keys[keys != oracle.EMPTY_KEY] >> np.uint64(32)).astype(np.uint32))


@pytest.mark.parametrize("scene", ["c2", "c3_quarter"])
def test_splat_full_size_segmented_minimum(scene):
    """At full frame size the oracle's depth-id buffer equals the per-pixel
    minimum of the keys, computed independently of its splat loop: keys
    bits(w) << 32 | id from the oracle's projection, reduced per pixel with
    numpy's unbuffered minimum.  2^22 uniform points at 1920x1080 (orbit
    frame 250), and 2^24 points of the 16-cluster mixture at 3840x2160, where
    thousands of points share a pixel."""
    if scene == "c2":
        sc, pos = inputs.C2, inputs.encode(inputs.C2.positions(), "f32")
        M = oracle.camera_f32(sc.eye(250), CEN, UP, sc.fovy_deg, sc.aspect, sc.znear, sc.zfar)
    else:
        sc = inputs.C3
        pos = inputs.encode(inputs.gaussian_mixture_cloud(1 << 24, 3), "f32")
        M = oracle.camera_f32(sc.eye(0), CEN, UP, sc.fovy_deg, sc.aspect, sc.znear, sc.zfar)
    zn, zf = np.float32(sc.znear), np.float32(sc.zfar)
    keys, _ = oracle.render(pos, "f32", M, sc.W, sc.H, zn, zf)
    px, w = oracle.project_f32(M, pos, sc.W, sc.H, zn, zf)
    hit = np.nonzero(px != 0xFFFFFFFF)[0]
    k = (w[hit].view(np.uint32).astype(np.uint64) << np.uint64(32)) | hit.astype(np.uint64)
    want = np.full(sc.W * sc.H, oracle.EMPTY_KEY, np.uint64)
    np.minimum.at(want, px[hit].astype(np.int64), k)
    assert np.array_equal(keys, want)
    assert (keys != oracle.EMPTY_KEY).sum() > sc.W * sc.H // 50


def test_resolve_hand_cases():
    keys = np.array([0xFFFFFFFFFFFFFFFF, (0x40000000 << 32) | 2, (0x3F800000 << 32) | 0], np.uint64)
    assert list(oracle.resolve(keys, color=0x11223344, background=0x55)) == [0x55, 0x11223344, 0x11223344]
    cols = np.array([7, 8, 9], np.uint32)
    assert list(oracle.resolve(keys, colors=cols, background=0x55)) == [0x55, 9, 7]


def test_h16_splat_uses_widened_positions():
    W, H = 32, 32
    pos64 = inputs.uniform_cloud(2000, 17)
    M = oracle.camera_f32(EYE, CEN, UP, 60.0, 1.0, 0.1, 100.0)
    for fmt in ("f16", "bf16"):
        bits = inputs.encode(pos64, fmt)
        k1 = oracle.empty_keys(W, H)
        oracle.splat(bits, fmt, M, W, H, 0.1, 100.0, k1)
        k2 = oracle.empty_keys(W, H)
        oracle.splat(oracle.from_storage(bits, fmt), "f32", M, W, H, 0.1, 100.0, k2)
        assert np.array_equal(k1, k2)


def test_inputs_module_encoding_agrees_with_oracle_conversions():
    pos64 = inputs.uniform_cloud(10_000, 18)
    p32 = inputs.encode(pos64, "f32")
    for fmt in ("f16", "bf16"):
        assert np.array_equal(inputs.encode(pos64, fmt), oracle.to_storage(p32, fmt))
        assert np.array_equal(inputs.decode(inputs.encode(pos64, fmt), fmt),
                              oracle.from_storage(inputs.encode(pos64, fmt), fmt))


# --------------------------------------------------------------------------
# Disc markers: brute-force per-pixel search and lattice-point counts.
# --------------------------------------------------------------------------
def _brute_force_disc(pos32, M32, W, H, radius):
    """Independent restatement: for every pixel, every point; numpy float32
    arithmetic (IEEE round-to-nearest) in the stated order."""
    f = np.float32
    M = M32.astype(np.float32)
    x, y, z = pos32[:, 0], pos32[:, 1], pos32[:, 2]
    cx = ((M[0, 0] * x + M[0, 1] * y) + M[0, 2] * z) + M[0, 3]
    cy = ((M[1, 0] * x + M[1, 1] * y) + M[1, 2] * z) + M[1, 3]
    cw = ((M[3, 0] * x + M[3, 1] * y) + M[3, 2] * z) + M[3, 3]
    ok = (cw > f(0.1)) & (cw < f(100.0))
    with np.errstate(all="ignore"):
        sx = (cx / cw + f(1.0)) * f(0.5 * W)
        sy = (f(1.0) - cy / cw) * f(0.5 * H)
    r2 = f(radius) * f(radius)
    keys = (cw.view(np.uint32).astype(np.uint64) << np.uint64(32)) | np.arange(len(x), dtype=np.uint64)
    want = np.full(W * H, 0xFFFFFFFFFFFFFFFF, np.uint64)
    for py in range(H):
        dy = (f(py) + f(0.5)) - sy
        for px in range(W):
            dx = (f(px) + f(0.5)) - sx
            cov = ok & ((dx * dx + dy * dy) <= r2)
            if cov.any():
                want[py * W + px] = keys[cov].min()
    return want


@pytest.mark.parametrize("radius", [0.5, 1.0, 2.5, 4.0])
def test_disc_splat_matches_brute_force(radius):
    W, H = 40, 30
    pos = inputs.encode(inputs.gaussian_mixture_cloud(600, 40, components=3, sigma=0.08), "f32")
    M = oracle.camera_f32(EYE, CEN, UP, 60.0, W / H, 0.1, 100.0)
    keys = oracle.empty_keys(W, H)
    oracle.splat_disc(pos, M, W, H, 0.1, 100.0, radius, keys)
    assert np.array_equal(keys, _brute_force_disc(pos, M, W, H, radius))


@pytest.mark.parametrize("radius,count", [(1.0, 5), (2.0, 13), (3.0, 29), (0.5, 1)])
def test_disc_covers_lattice_points_of_circle(radius, count):
    """A point projected exactly onto a pixel centre covers the pixels whose
    centres are within r: the number of integer lattice points in a disc of
    radius r (Gauss circle problem: 5, 13, 29 for r = 1, 2, 3)."""
    W = H = 21
    # plain matrix: sx = (x/z + 1) W/2 with z = w = 1; x chosen so that sx = 10.5 (centre of pixel 10)
    M = np.zeros((4, 4), np.float32)
    M[0, 0] = M[1, 1] = M[3, 2] = 1.0
    xc = np.float32(10.5 / (W / 2) - 1.0)
    pos = np.array([[xc, -xc, 1.0]], np.float32)
    keys = oracle.empty_keys(W, H)
    oracle.splat_disc(pos, M, W, H, 0.1, 100.0, radius, keys)
    assert int((keys != oracle.EMPTY_KEY).sum()) == count


# --------------------------------------------------------------------------
# N-body (second workload): two-body closed form, brute force, conservation.
# --------------------------------------------------------------------------
def test_nbody_two_body_closed_form():
    """Two bodies of mass m at rest, distance d apart on x: each is pulled
    towards the other with a = G m d / (d^2 + eps2)^(3/2)."""
    G, m, d, eps2, dt = 1.0, 2.0, 0.5, 1e-4, 1e-3
    pos = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]], np.float32)
    vel = np.zeros_like(pos)
    out = oracle.nbody_step_f32(pos, vel, np.array([m, m], np.float32), np.float32(G), np.float32(eps2),
                                np.float32(dt))
    a = G * m * d / (d * d + eps2) ** 1.5
    assert vel[0, 0] == pytest.approx(a * dt, rel=1e-6) and vel[1, 0] == pytest.approx(-a * dt, rel=1e-6)
    assert np.all(vel[:, 1:] == 0)
    assert out[0, 0] == pytest.approx(a * dt * dt, rel=1e-5) and out[1, 0] == pytest.approx(d - a * dt * dt, rel=1e-6)


def nbody_velocity_tolerance(S, v_new, v_old, G, dt, n):
    """Largest difference of v' = v + (G acc) dt between two summation orders
    of acc: each order is within gamma_{n-1} S of the exact sum (Higham,
    Sec. 4.2), so the two accelerations differ by at most 2 gamma_{n-1} S; the
    three roundings after the sum add at most u (|x| + |y|) each, taken here
    as 8u (|v_old| + |v_new| + |G dt| S) with margin."""
    u = 2.0**-24
    g = oracle.summation_bound_gamma(n)
    return abs(G * dt) * 2.0 * g * S * (1 + 4 * u) + 8 * u * (np.abs(v_old) + np.abs(v_new) + abs(G * dt) * S)


def test_nbody_summation_bound_catches_a_dropped_term():
    """The tolerance above is tight enough to see a whole term go missing for
    a body that one close neighbour dominates."""
    pos = np.array([[0.5, 0.5, 0.5], [0.5005, 0.5, 0.5], [0.9, 0.1, 0.2], [0.1, 0.8, 0.3]], np.float32)
    mass = np.ones(4, np.float32)
    G, eps2, dt = np.float32(1e-3), np.float32(1e-6), np.float32(1e-2)
    vel = np.zeros_like(pos)
    oracle.nbody_step_f32(pos, vel, mass, G, eps2, dt)
    vel_missing = np.zeros_like(pos)
    oracle.nbody_step_f32(pos[:3], vel_missing[:3], mass[:3], G, eps2, dt)     # body 3's pull dropped
    S = oracle.nbody_abs_term_sums(pos, mass, float(eps2))
    tol = nbody_velocity_tolerance(S, vel, np.zeros_like(vel), float(G), float(dt), 4)
    assert np.any(np.abs(vel_missing[:3].astype(np.float64) - vel[:3]) > tol[:3])


def test_nbody_matches_fp64_brute_force_and_conserves_momentum():
    n = 300
    rng = np.random.default_rng(8)
    pos = inputs.encode(inputs.gaussian_mixture_cloud(n, 41, components=2, sigma=0.1), "f32")
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    G, eps2, dt = np.float32(1e-3), np.float32(1e-3), np.float32(1e-2)
    vel = np.zeros_like(pos)
    oracle.nbody_step_f32(pos, vel, mass, G, eps2, dt)
    acc64 = oracle.nbody_accel_f64(pos.astype(np.float64), mass.astype(np.float64), float(G), float(eps2))
    # independent numpy restatement in float64
    d = pos.astype(np.float64)[None, :, :] - pos.astype(np.float64)[:, None, :]
    r2 = (d ** 2).sum(-1) + float(eps2)
    acc_np = float(G) * (d * (mass.astype(np.float64)[None, :] / r2 ** 1.5)[..., None]).sum(1)
    assert np.allclose(acc64, acc_np, rtol=1e-12, atol=1e-15)
    assert np.allclose(vel / float(dt), acc64, rtol=2e-4, atol=1e-6)
    # one chunk is the sequential sum itself; other chunkings stay within the summation error bound of it
    vel_one = np.zeros_like(pos)
    oracle.nbody_step_f32_chunked(pos, vel_one, mass, G, eps2, dt, chunk=n)
    assert np.array_equal(vel_one, vel)
    S = oracle.nbody_abs_term_sums(pos, mass, float(eps2))
    for chunk in (7, 64, 150):
        vel_chunked = np.zeros_like(pos)
        oracle.nbody_step_f32_chunked(pos, vel_chunked, mass, G, eps2, dt, chunk=chunk)
        assert not np.array_equal(vel_chunked, vel)       # a different, but fixed, rounding order
        tol = nbody_velocity_tolerance(S, vel, np.zeros_like(vel), float(G), float(dt), n)
        assert np.all(np.abs(vel_chunked.astype(np.float64) - vel) <= tol)
    # pairwise forces cancel: total momentum stays at zero up to FP32 rounding
    p_tot = (mass[:, None].astype(np.float64) * vel.astype(np.float64)).sum(0)
    scale = (mass[:, None] * np.abs(vel)).sum(0)
    assert np.all(np.abs(p_tot) <= 1e-4 * scale)
