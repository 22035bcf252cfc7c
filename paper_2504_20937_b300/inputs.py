"""Seeded synthetic inputs for the displace + render path.

Shared by the tests, the bench and the smoke check.  This module holds none
of the method's arithmetic (no Philox, no displacement, no projection): it
only draws initial clouds with numpy's PCG64 generator, encodes them into the
storage formats with library conversions, and lists the benchmark scenes
(camera paths, resolutions, batched cloud tables, viewer arrival traces).

The workloads follow the paper's benchmark (Mimir, Sec. 4.1): a 3D point
cloud with random initial positions moved by Brownian motion each frame and
drawn as 1-px markers of one colour.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

DTYPES = ("f32", "f16", "bf16")
BYTES_PER_POINT = {"f32": 12, "f16": 6, "bf16": 6}


def uniform_cloud(n: int, seed: int) -> np.ndarray:
    """n points uniform in [0,1)^3, float64[n,3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n, 3), dtype=np.float64)


def gaussian_mixture_cloud(n: int, seed: int, components: int = 16, sigma: float = 0.02) -> np.ndarray:
    """n points from an isotropic Gaussian mixture (centres uniform in [0,1]^3),
    each point drawn from a uniformly chosen component, clamped to [0,1]^3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.random((components, 3), dtype=np.float64)
    comp = rng.integers(0, components, size=n)
    pos = rng.standard_normal((n, 3), dtype=np.float64)
    pos *= sigma
    pos += centres[comp]
    np.clip(pos, 0.0, 1.0, out=pos)
    return pos


def encode(pos64: np.ndarray, dtype: str) -> np.ndarray:
    """float64[n,3] -> storage array: float32[n,3] for 'f32', else the uint16
    bit patterns of binary16 / bfloat16 (FP64 -> FP32 -> 16-bit, both RNE)."""
    p32 = np.ascontiguousarray(pos64, dtype=np.float32)
    if dtype == "f32":
        return p32
    t = torch.from_numpy(p32)
    t = t.to(torch.float16 if dtype == "f16" else torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16).copy()


def decode(bits: np.ndarray, dtype: str) -> np.ndarray:
    """Storage array -> float32 (exact widening), via torch's conversions."""
    if dtype == "f32":
        return np.asarray(bits, np.float32)
    t = torch.from_numpy(np.ascontiguousarray(bits).view(np.int16))
    t = t.view(torch.float16 if dtype == "f16" else torch.bfloat16)
    return t.to(torch.float32).numpy()


def orbit_eye(frame: int, deg_per_frame: float, radius: float = 2.0,
              centre=(0.5, 0.5, 0.5), elevation: float = 0.0, start_deg: float = 0.0):
    """Eye on a circle about `centre` (angle evaluated in FP64)."""
    th = math.radians(start_deg + frame * deg_per_frame)
    return (centre[0] + radius * math.cos(elevation) * math.sin(th),
            centre[1] + radius * math.sin(elevation),
            centre[2] + radius * math.cos(elevation) * math.cos(th))


@dataclass
class Scene:
    """One displace + render workload on one cloud and one view."""
    name: str
    n: int
    W: int
    H: int
    frames: int
    amplitude: float
    cloud: str = "uniform"          # or "gmm16"
    init_seed: int = 0
    philox_seed: int = 0
    deg_per_frame: float = 0.0      # orbit speed; 0 = fixed camera
    radius: float = 2.0
    fovy_deg: float = 60.0
    znear: float = 0.1
    zfar: float = 100.0
    target: tuple = (0.5, 0.5, 0.5)
    up: tuple = (0.0, 1.0, 0.0)
    color: int = 0xFFFFFFFF
    background: int = 0x00000000

    def positions(self) -> np.ndarray:
        if self.cloud == "uniform":
            return uniform_cloud(self.n, self.init_seed)
        return gaussian_mixture_cloud(self.n, self.init_seed)

    def eye(self, frame: int):
        return orbit_eye(frame, self.deg_per_frame, self.radius, self.target)

    @property
    def aspect(self) -> float:
        return self.W / self.H


# The five benchmark scenes.  Eye at (0.5, 0.5, 2.5) looking at the cloud
# centre for frame 0 (radius 2 about the centre), vertical fov 60 degrees.
PR1 = Scene("pr1_65536pts_512x512", n=65536, W=512, H=512, frames=100, amplitude=1e-3,
            init_seed=0, philox_seed=0)
C2 = Scene("c2_4Mpts_1920x1080_orbit", n=1 << 22, W=1920, H=1080, frames=1000, amplitude=5e-4,
           init_seed=2, philox_seed=2, deg_per_frame=0.36)
C3 = Scene("c3_64Mpts_gmm16_3840x2160", n=1 << 26, W=3840, H=2160, frames=200, amplitude=5e-4,
           cloud="gmm16", init_seed=3, philox_seed=3)

SCENES = {s.name: s for s in (PR1, C2, C3)}


@dataclass
class BatchCloud:
    n: int
    kind: str                       # "uniform" or "gmm4"
    W: int
    H: int
    radius: float
    elevation: float
    start_deg: float
    deg_per_frame: float
    init_seed: int


def batched_table(count: int = 256, seed: int = 4, n_lo: float = 1e3, n_hi: float = 1e6,
                  resolutions=((256, 256), (512, 512), (1024, 1024))) -> list[BatchCloud]:
    """Independent clouds of log-uniform size, uniform or 4-cluster Gaussian at
    random, each with its own random orbit camera and resolution."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for c in range(count):
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kind = "uniform" if rng.random() < 0.5 else "gmm4"
        W, H = resolutions[int(rng.integers(0, len(resolutions)))]
        out.append(BatchCloud(n=n, kind=kind, W=W, H=H, radius=float(rng.uniform(1.5, 3.0)),
                              elevation=float(rng.uniform(-0.5, 0.5)),
                              start_deg=float(rng.uniform(0.0, 360.0)),
                              deg_per_frame=0.36, init_seed=1000 * seed + c))
    return out


def batch_cloud_positions(bc: BatchCloud) -> np.ndarray:
    if bc.kind == "uniform":
        return uniform_cloud(bc.n, bc.init_seed)
    return gaussian_mixture_cloud(bc.n, bc.init_seed, components=4)


@dataclass
class ViewerRequest:
    viewer: int
    arrival_s: float
    W: int
    H: int
    frames: int
    private_n: int
    start_deg: float
    init_seed: int


def serving_trace(requests: int = 10_000, seed: int = 5, rate_hz: float = 40.0,
                  frames_per_viewer: int = 50, private_lo: float = 1e4, private_hi: float = 1e6,
                  resolutions=((640, 480), (1920, 1080), (3840, 2160))) -> list[ViewerRequest]:
    """Poisson arrivals of viewers; each viewer asks for `frames_per_viewer`
    frames of its own resolution, with its own private cloud.  Served at a
    60 Hz display rate (one frame per viewer per refresh), a viewer stays
    frames_per_viewer / 60 s, so on average rate_hz * frames_per_viewer / 60
    viewers share the engine: about 33 at the defaults, with Poisson spread
    (a standard deviation near 6) inside the 8-64 range."""
    rng = np.random.Generator(np.random.PCG64(seed))
    viewers = max(1, requests // frames_per_viewer)
    t = 0.0
    out = []
    for v in range(viewers):
        t += float(rng.exponential(1.0 / rate_hz))
        W, H = resolutions[int(rng.integers(0, len(resolutions)))]
        pn = int(math.floor(math.exp(rng.uniform(math.log(private_lo), math.log(private_hi)))))
        out.append(ViewerRequest(viewer=v, arrival_s=t, W=W, H=H, frames=frames_per_viewer,
                                 private_n=pn, start_deg=float(rng.uniform(0, 360)),
                                 init_seed=50_000 + v))
    return out
