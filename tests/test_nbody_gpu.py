"""Second workload: gravitational all-pairs N-body feeding the renderer.

The definition sums each body's terms in order of j (the oracle's
nbody_step_f32).  The kernel sums them in chunks of 1024 bodies so that it
can fill the GPU; it is checked two ways: bit for bit against the oracle
replaying that chunked order (positions, velocities, keys, RGBA), and
against the sequential sum within Higham's summation error bound."""
import numpy as np
import pytest
import torch

import oracle
from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.api import Context, MmrError

pytestmark = pytest.mark.gpu

CEN = (0.5, 0.5, 0.5)
UP = (0.0, 1.0, 0.0)


@pytest.mark.parametrize("n", [1, 2, 3, 127, 128, 129, 255, 257, 1023, 1024, 1025, 2049, 3001])
def test_nbody_steps_bit_exact(n):
    W, H, steps = 96, 64, 3
    G, eps2, dt = np.float32(2e-4), np.float32(1e-3), np.float32(5e-2)
    pos = inputs.encode(inputs.gaussian_mixture_cloud(n, 60 + n, components=2, sigma=0.08), "f32")
    mass = np.random.default_rng(n).uniform(0.5, 2.0, n).astype(np.float32)
    vel0 = (np.random.default_rng(n + 1).standard_normal((n, 3)) * 0.01).astype(np.float32)
    eye = lambda f: inputs.orbit_eye(f, 3.0)  # noqa: E731
    with Context(W, H) as ctx:
        bufs = ctx.alloc_pingpong(n, "f32")
        bufs[0].copy_(torch.from_numpy(pos))
        v, m = ctx.alloc_nbody()
        v.copy_(torch.from_numpy(vel0))
        m.copy_(torch.from_numpy(mass))
        for f in range(steps):
            ctx.set_camera(eye(f), CEN, UP, 60.0, 0.1, 100.0)
            ctx.nbody_step_and_render(float(G), float(eps2), float(dt))
        torch.cuda.synchronize()
        gpos = ctx.points.cpu().numpy()
        gvel = v.cpu().numpy()
        gkeys = ctx.frame_keys().cpu().numpy().reshape(-1).view(np.uint64)
        grgba = ctx.frame_rgba().cpu().numpy().reshape(-1).view(np.uint32)
        assert ctx.visible == steps % 2
    p, vel = pos.copy(), vel0.copy()
    for f in range(steps):
        p = oracle.nbody_step_f32_chunked(p, vel, mass, G, eps2, dt)
    M = oracle.camera_f32(eye(steps - 1), CEN, UP, 60.0, W / H, 0.1, 100.0)
    keys, rgba = oracle.render(p, "f32", M, W, H, np.float32(0.1), np.float32(100.0))
    assert np.array_equal(gpos, p)
    assert np.array_equal(gvel, vel)
    assert np.array_equal(gkeys, keys) and np.array_equal(grgba, rgba)
    if n > 1:
        assert not np.array_equal(gpos, pos)           # the bodies did move


@pytest.mark.parametrize("n", [257, 3001, 20000])
def test_nbody_step_within_summation_bound_of_sequential_sum(n):
    """One step from the same state: the kernel's velocities and positions
    against the sequential-sum oracle, within the bound of Higham, Accuracy
    and Stability of Numerical Algorithms (2nd ed.), Sec. 4.2: any order of
    recursive FP32 summation of n terms is within gamma_{n-1} sum |t_j| of
    the exact sum, so two orders differ by at most twice that; the update
    v' = v + (G acc) dt and p' = p + v' dt adds a few roundings of its own."""
    from .test_oracle_pins import nbody_velocity_tolerance
    G, eps2, dt = np.float32(2e-4), np.float32(1e-3), np.float32(5e-2)
    pos = inputs.encode(inputs.gaussian_mixture_cloud(n, 80 + n, components=3, sigma=0.08), "f32")
    mass = np.random.default_rng(n).uniform(0.5, 2.0, n).astype(np.float32)
    vel0 = (np.random.default_rng(n + 1).standard_normal((n, 3)) * 0.01).astype(np.float32)
    with Context(64, 64) as ctx:
        bufs = ctx.alloc_pingpong(n, "f32")
        bufs[0].copy_(torch.from_numpy(pos))
        v, m = ctx.alloc_nbody()
        v.copy_(torch.from_numpy(vel0))
        m.copy_(torch.from_numpy(mass))
        ctx.set_camera((0.5, 0.5, 2.5), CEN, UP, 60.0, 0.1, 100.0)
        ctx.nbody_step_and_render(float(G), float(eps2), float(dt))
        torch.cuda.synchronize()
        gpos = ctx.points.cpu().numpy().astype(np.float64)
        gvel = v.cpu().numpy().astype(np.float64)
    vel = vel0.copy()
    p = oracle.nbody_step_f32(pos, vel, mass, G, eps2, dt)
    S = oracle.nbody_abs_term_sums(pos, mass, float(eps2))
    tol_v = nbody_velocity_tolerance(S, vel, vel0, float(G), float(dt), n)
    assert np.all(np.abs(gvel - vel) <= tol_v)
    u = 2.0**-24
    tol_p = abs(float(dt)) * tol_v * (1 + 2 * u) + 4 * u * (np.abs(p) + np.abs(pos) + np.abs(vel * float(dt)))
    assert np.all(np.abs(gpos - p) <= tol_p)
    if n > 1024:
        assert not np.array_equal(gvel, vel)        # the two orders really differ here


def test_nbody_needs_fp32_pingpong():
    with Context(16, 16) as ctx:
        ctx.alloc_points(10, "f32")
        with pytest.raises(MmrError, match="STATE"):
            ctx.alloc_nbody()
    with Context(16, 16) as ctx:
        ctx.alloc_pingpong(10, "f16")
        with pytest.raises(MmrError, match="STATE"):
            ctx.alloc_nbody()
    with Context(16, 16) as ctx:
        ctx.alloc_pingpong(10, "f32")
        ctx.alloc_nbody()
        ctx.set_camera((0.5, 0.5, 2.5), CEN, UP, 60.0, 0.1, 100.0)
        with pytest.raises(MmrError, match="INVALID"):
            ctx.nbody_step_and_render(1.0, 0.0, 0.01)     # eps2 must be > 0
