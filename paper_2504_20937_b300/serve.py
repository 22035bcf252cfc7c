"""Continuous-batching request loop over the serving engine (mmr_serve_*).

Viewers arrive over time (a trace from inputs.serving_trace), each asking
for a run of frames of its own resolution with its own private cloud.  The
loop admits arrived viewers while there is a free slot and the engine's
device-memory budget allows (a refused viewer waits in FIFO order), runs one
engine tick per iteration (one frame for every active viewer, all of them
batched into the same kernels), and retires viewers when their last frame is
done, which frees memory for the queue.

Two pacings.  With a display rate (tick_hz > 0, the default 60 Hz) every
active viewer asks for a frame at each display refresh, as a viewer whose
display shows one frame per refresh would: ticks start on the refresh grid,
a frame's latency runs from its refresh (from the viewer's arrival for its
first frame) to the completion of the tick that rendered it, and a refresh
that comes while a tick is still running is dropped (counted).  The number
of viewers on the engine is then set by the arrivals and the session length,
not by the engine's speed, so two engines see the same load.  With
tick_hz = 0 ticks run back to back, a frame's request being the completion
of the viewer's previous frame: the engine's saturation throughput.

The scheduling decisions and the bookkeeping live here; all device work is
in the library.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import inputs
from .api import Server

CENTRE = (0.5, 0.5, 0.5)
UP = (0.0, 1.0, 0.0)


@dataclass
class ServeConfig:
    shared_n: int = 1 << 24
    shared_seed: int = 5
    dtype: str = "f32"
    amplitude: float = 5e-4
    budget_bytes: int = 40 << 30
    max_viewers: int = 64
    shared_color: int = 0xFFFFFFFF
    deg_per_frame: float = 0.36
    fovy_deg: float = 60.0
    znear: float = 0.1
    zfar: float = 100.0
    tick_hz: float = 60.0           # display refresh rate; 0 = ticks back to back


@dataclass
class ServeStats:
    frames: int = 0
    ticks: int = 0
    wall_s: float = 0.0
    tick_ms: list = field(default_factory=list)
    latencies_ms: list = field(default_factory=list)
    steady_latencies_ms: list = field(default_factory=list)   # frames after a viewer's first
    active_per_tick: list = field(default_factory=list)
    points_rendered: int = 0
    max_active: int = 0
    refused_for_budget: int = 0
    queue_wait_ms: list = field(default_factory=list)
    tick_start_s: list = field(default_factory=list)
    tick_hz: float = 0.0
    refreshes_dropped: int = 0
    steady_window_s: tuple = (0.0, 0.0)   # ticks starting in it count for the steady-state concurrency

    def summary(self) -> dict:
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        steady = np.asarray(self.steady_latencies_ms) if self.steady_latencies_ms else np.zeros(1)
        t = np.asarray(self.tick_start_s)
        act = np.asarray(self.active_per_tick)
        win = (t >= self.steady_window_s[0]) & (t <= self.steady_window_s[1]) if t.size else t.astype(bool)
        return {"tick_hz": self.tick_hz, "frames": self.frames, "ticks": self.ticks, "wall_s": self.wall_s,
                "refreshes_dropped": self.refreshes_dropped,
                "steady_window_s": list(self.steady_window_s),
                "mean_active_viewers_steady": float(act[win].mean()) if win.any() else 0.0,
                "min_active_viewers_steady": int(act[win].min()) if win.any() else 0,
                "frames_per_s": self.frames / self.wall_s if self.wall_s else 0.0,
                "points_per_s": self.points_rendered / self.wall_s if self.wall_s else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "p50_ms_after_first": float(np.percentile(steady, 50)),
                "p99_ms_after_first": float(np.percentile(steady, 99)),
                "mean_active_viewers": float(np.mean(self.active_per_tick)) if self.active_per_tick else 0.0,
                "min_active_viewers": int(min(self.active_per_tick)) if self.active_per_tick else 0,
                "mean_tick_ms": float(np.mean(self.tick_ms)) if self.tick_ms else 0.0,
                "max_active_viewers": self.max_active, "refused_for_budget": self.refused_for_budget,
                "p99_queue_wait_ms": float(np.percentile(self.queue_wait_ms, 99)) if self.queue_wait_ms else 0.0}


def viewer_eye(req: inputs.ViewerRequest, frame: int, cfg: ServeConfig):
    return inputs.orbit_eye(frame, cfg.deg_per_frame, 2.0, CENTRE, 0.0, req.start_deg)


def private_cloud(req: inputs.ViewerRequest, dtype: str) -> np.ndarray:
    return inputs.encode(inputs.uniform_cloud(req.private_n, req.init_seed), dtype)


def _to_torch(stored: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(stored if stored.dtype == np.float32 else stored.view(np.int16))


class ContinuousBatcher:
    """The scheduling policy of the request loop, free of any device work.

    Viewers arrive (`arrive`), wait in FIFO order, and are admitted while a
    slot is free and the engine accepts them (`admit` asks a callback, which
    returns None when the engine's memory budget refuses the viewer: the
    queue then stops, so arrival order is kept).  Every tick renders one frame
    for each admitted viewer (`tick_done`), which records each frame's
    latency from its request time and retires viewers whose last frame is
    done.
    """

    def __init__(self, max_viewers: int):
        self.max_viewers = max_viewers
        self.pending = collections.deque()
        self.waiting = collections.deque()
        self.active = {}              # engine id -> [request, frames done, request time]
        self.refused = 0

    def load(self, trace):
        self.pending = collections.deque(sorted(trace, key=lambda r: r.arrival_s))

    def arrive(self, now: float) -> None:
        while self.pending and self.pending[0].arrival_s <= now:
            self.waiting.append(self.pending.popleft())

    def admit(self, try_add) -> list:
        """try_add(request) -> engine id or None; returns the admitted (id, request)."""
        admitted = []
        while self.waiting and len(self.active) < self.max_viewers:
            req = self.waiting[0]
            vid = try_add(req)
            if vid is None:
                self.refused += 1
                break
            self.waiting.popleft()
            self.active[vid] = [req, 0, req.arrival_s]
            admitted.append((vid, req))
        return admitted

    def frames_due(self):
        """(engine id, request, frame index) of every frame the next tick renders."""
        return [(vid, st[0], st[1]) for vid, st in self.active.items()]

    def tick_done(self, done: float, refresh: float | None = None):
        """Account one tick finished at time `done`; returns (latencies of
        first frames, latencies of later frames, retired engine ids).  A
        first frame's latency runs from the viewer's arrival; a later frame's
        from `refresh`, the display refresh that asked for it, or without a
        display rate from the completion of the viewer's previous frame."""
        first, later, finished = [], [], []
        for vid, st in self.active.items():
            req, k, req_time = st
            if k == 0:
                first.append(done - req_time)
            else:
                later.append(done - (refresh if refresh is not None else req_time))
            st[1], st[2] = k + 1, done
            if st[1] >= req.frames:
                finished.append(vid)
        for vid in finished:
            del self.active[vid]
        return first, later, finished

    def busy(self) -> bool:
        return bool(self.pending or self.waiting or self.active)

    def next_arrival(self):
        return self.pending[0].arrival_s if self.pending else None


def run_trace(trace, cfg: ServeConfig, roundtrip: bool = False, clouds=None, shared=None) -> ServeStats:
    """Serve every request of `trace`; returns the statistics.

    clouds: optional {viewer: stored private cloud} (generated if missing);
    shared: optional stored shared cloud (generated if missing).  Pacing by
    cfg.tick_hz (see the module docstring).
    """
    if shared is None:
        shared = inputs.encode(inputs.uniform_cloud(cfg.shared_n, cfg.shared_seed), cfg.dtype)
    if clouds is None:
        clouds = {r.viewer: private_cloud(r, cfg.dtype) for r in trace}
    host_clouds = {v: _to_torch(c).pin_memory() for v, c in clouds.items()}
    stats = ServeStats(tick_hz=cfg.tick_hz)
    if trace:
        # steady state: after the first viewer's session could have filled up, until the last arrival
        ramp = max(r.frames for r in trace) / cfg.tick_hz if cfg.tick_hz > 0 else 0.0
        stats.steady_window_s = (min(r.arrival_s for r in trace) + ramp, max(r.arrival_s for r in trace))
    stream = torch.cuda.current_stream()
    sched = ContinuousBatcher(cfg.max_viewers)
    sched.load(trace)
    period = 1.0 / cfg.tick_hz if cfg.tick_hz > 0 else 0.0
    with Server(cfg.shared_n, cfg.dtype, cfg.shared_seed, 0, cfg.amplitude, cfg.budget_bytes) as srv:
        srv.shared_points().copy_(_to_torch(shared))
        srv.set_shared_color(cfg.shared_color)
        srv.set_timing(True)
        torch.cuda.synchronize()

        def try_add(req):
            return srv.try_add_viewer(req.private_n, req.W, req.H, seed=req.init_seed, cloud=1 + req.viewer,
                                      amplitude=cfg.amplitude, color=0xFF000000 | (req.viewer & 0xFFFFFF))

        refresh_k = 0
        t0 = time.perf_counter()
        while sched.busy():
            now = time.perf_counter() - t0
            refresh = None
            if period:
                refresh = refresh_k * period
                if now < refresh:
                    time.sleep(refresh - now)
                    now = time.perf_counter() - t0
                sched.arrive(refresh)
            else:
                sched.arrive(now)
            for vid, req in sched.admit(try_add):
                srv.viewer_points(vid).copy_(host_clouds[req.viewer], non_blocking=True)
                stats.queue_wait_ms.append(1e3 * max(0.0, (time.perf_counter() - t0) - req.arrival_s))
            due = sched.frames_due()
            if not due:
                if period:
                    refresh_k += 1
                else:
                    nxt = sched.next_arrival()
                    if nxt is not None:
                        time.sleep(max(0.0, min(nxt - now, 0.001)))
                continue
            stats.max_active = max(stats.max_active, len(due))
            stats.active_per_tick.append(len(due))
            stats.tick_start_s.append(refresh if period else now)
            for vid, req, k in due:
                srv.set_camera(vid, viewer_eye(req, k, cfg), CENTRE, UP, cfg.fovy_deg, cfg.znear, cfg.zfar)
            srv.tick(stream, roundtrip=roundtrip)
            stats.tick_ms.append(srv.last_tick_ms())      # waits for the tick
            done = time.perf_counter() - t0
            stats.ticks += 1
            first, later, finished = sched.tick_done(done, refresh)
            stats.latencies_ms += [1e3 * x for x in first + later]
            stats.steady_latencies_ms += [1e3 * x for x in later]
            stats.frames += len(due)
            stats.points_rendered += sum(cfg.shared_n + req.private_n for _, req, _ in due)
            for vid in finished:
                srv.remove_viewer(vid)
            if period:
                # the next refresh after this tick; the ones it ran over are dropped
                nxt = max(refresh_k + 1, int(np.ceil(done / period)))
                stats.refreshes_dropped += nxt - refresh_k - 1
                refresh_k = nxt
        stats.refused_for_budget = sched.refused
        stats.wall_s = time.perf_counter() - t0
    return stats
