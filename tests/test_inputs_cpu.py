"""The seeded synthetic workloads (paper_2504_20937_b300/inputs.py) that stand in
for the paper's: their sizes, value ranges and distributions, checked on the CPU
against the recipes they state.  Nothing here touches the method's arithmetic."""
import math

import numpy as np

from paper_2504_20937_b300 import inputs


def test_uniform_cloud_range_mean_and_seeding():
    n = 1_000_000
    p = inputs.uniform_cloud(n, 3)
    assert p.shape == (n, 3) and p.dtype == np.float64
    assert p.min() >= 0.0 and p.max() < 1.0
    sigma_mean = 1.0 / math.sqrt(12.0 * n)
    assert np.all(np.abs(p.mean(axis=0) - 0.5) < 5 * sigma_mean)
    assert np.array_equal(p, inputs.uniform_cloud(n, 3))
    assert not np.array_equal(p[:10], inputs.uniform_cloud(10, 4))


def test_gaussian_mixture_concentrates_around_its_centres():
    """16 components, sigma 0.02, clamped to [0,1]^3: the distance of a point
    to the nearest centre follows sigma * chi_3 (median 1.538 sigma), shrunk
    slightly by the clamp, and no point lies beyond 7 sigma of every centre."""
    n, seed = 200_000, 7
    p = inputs.gaussian_mixture_cloud(n, seed)
    assert p.min() >= 0.0 and p.max() <= 1.0
    centres = np.random.Generator(np.random.PCG64(seed)).random((16, 3))
    d = np.min(np.linalg.norm(p[:, None, :] - centres[None, :, :], axis=2), axis=1)
    assert 0.028 < np.median(d) < 0.032
    assert d.max() < 7 * 0.02


def test_storage_encoding_rounds_to_nearest():
    p = 0.25 + 0.75 * inputs.uniform_cloud(100_000, 5)
    f32 = inputs.encode(p, "f32")
    assert f32.dtype == np.float32 and np.array_equal(f32, p.astype(np.float32))
    for dtype, rel in (("f16", 2.0**-11), ("bf16", 2.0**-8)):
        bits = inputs.encode(p, dtype)
        assert bits.dtype == np.uint16 and bits.shape == p.shape
        back = inputs.decode(bits, dtype).astype(np.float64)
        assert np.all(np.abs(back - p.astype(np.float32)) <= rel * np.abs(p) + 1e-12)


def test_orbit_cameras():
    for f in (0, 1, 250, 999):
        e = np.array(inputs.orbit_eye(f, 0.36))
        assert abs(np.linalg.norm(e - 0.5) - 2.0) < 1e-12 and abs(e[1] - 0.5) < 1e-12
    np.testing.assert_allclose(inputs.orbit_eye(0, 0.36), (0.5, 0.5, 2.5), atol=1e-12)
    np.testing.assert_allclose(inputs.orbit_eye(1000, 0.36), inputs.orbit_eye(0, 0.36), atol=1e-12)
    e = np.array(inputs.orbit_eye(3, 0.36, radius=2.5, elevation=0.3, start_deg=40.0))
    assert abs(np.linalg.norm(e - 0.5) - 2.5) < 1e-12


def test_scene_configurations():
    assert (inputs.PR1.n, inputs.PR1.W, inputs.PR1.H, inputs.PR1.frames, inputs.PR1.amplitude) == \
        (65536, 512, 512, 100, 1e-3)
    assert (inputs.C2.n, inputs.C2.W, inputs.C2.H, inputs.C2.frames, inputs.C2.amplitude) == \
        (1 << 22, 1920, 1080, 1000, 5e-4)
    assert (inputs.C3.n, inputs.C3.W, inputs.C3.H, inputs.C3.frames) == (1 << 26, 3840, 2160, 200)
    np.testing.assert_allclose(inputs.C2.eye(1000), inputs.C2.eye(0), atol=1e-12)   # 0.36 deg per frame


def test_batched_table_recipe():
    """256 clouds, sizes log-uniform in [1e3, 1e6), uniform or 4-cluster at
    random, resolutions from {256^2, 512^2, 1024^2}, orbit radius 1.5..3; the
    scene the bench times holds 45,945,637 points and 123,535,360 pixels."""
    t = inputs.batched_table()
    assert len(t) == 256
    n = np.array([c.n for c in t])
    assert n.min() >= 1000 and n.max() < 1_000_000
    logs = np.log(n)
    centre, spread = (math.log(1e3) + math.log(1e6)) / 2, (math.log(1e6) - math.log(1e3)) / math.sqrt(12 * 256)
    assert abs(logs.mean() - centre) < 5 * spread
    assert {(c.W, c.H) for c in t} == {(256, 256), (512, 512), (1024, 1024)}
    kinds = [c.kind for c in t]
    assert set(kinds) == {"uniform", "gmm4"} and 90 < kinds.count("uniform") < 166
    assert all(1.5 <= c.radius <= 3.0 and -0.5 <= c.elevation <= 0.5 for c in t)
    assert int(n.sum()) == 45_945_637
    assert sum(c.W * c.H for c in t) == 123_535_360
    assert [c.n for c in inputs.batched_table()] == list(n)


def test_serving_trace_recipe():
    """10,000 frame requests as 200 viewers of 50 frames, Poisson arrivals at
    40 viewers/s, private clouds log-uniform in [1e4, 1e6), three resolutions.
    At 60 frames a second per viewer the concurrency (viewers whose 50/60 s
    session covers a moment) stays inside 8..64 once the first sessions have
    filled up, until the last arrival."""
    tr = inputs.serving_trace()
    assert len(tr) == 200 and sum(r.frames for r in tr) == 10_000
    arr = np.array([r.arrival_s for r in tr])
    assert np.all(np.diff(arr) > 0)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1 / 40) < 5 * (1 / 40) / math.sqrt(len(gaps))
    session = 50 / 60.0
    grid = np.arange(arr[0] + session, arr[-1], 1 / 60.0)
    conc = np.array([np.count_nonzero((arr <= t) & (arr + session > t)) for t in grid])
    assert 8 <= conc.min() and conc.max() <= 64 and 25 <= conc.mean() <= 42
    pn = np.array([r.private_n for r in tr])
    assert pn.min() >= 10_000 and pn.max() < 1_000_000
    assert {(r.W, r.H) for r in tr} == {(640, 480), (1920, 1080), (3840, 2160)}
