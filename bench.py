#!/usr/bin/env python
"""Benchmark of the zero-copy displace + render step on one B300.

One step = one frame of the hot path: a fused kernel displaces every point
(Philox-4x32 Brownian offsets), projects it and depth-splats it into the
depth-id buffer, then a resolve kernel writes the RGBA8 framebuffer and
clears the next depth-id buffer.  Inputs are resident in device memory when
the timed region starts.

Default workload (the headline): 2^26 = 67,108,864 FP32 points drawn from a
16-component isotropic Gaussian mixture (sigma 0.02), 3840x2160, fixed
camera, a = 5e-4.  Its 805 MB of positions are larger than L2 (126 MB), so
no flush is needed between frames; each frame is timed with CUDA events on
the launching stream.  Also reported on the same run: the host round-trip
path (positions device -> host -> device every frame), the end-to-end rate
through the public API with each frame read back to host memory, the error
of each storage type against the FP64 oracle, the same frame in binary16 and
bfloat16 storage, the 2^22-point 1920x1080 orbit (L2 flushed before every
frame), and the batched and served forms.

`--impl reference` times the CPU oracle (single-threaded C) on the same
workload instead.  Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_20937_b300 import inputs  # noqa: E402

METRIC = "points/s (displace+render)"
FLUSH_BYTES = 512 << 20
L2_BYTES = 126 << 20
TIMING_RING = 4096          # frames whose kernel times the library keeps (MMR_TIMING_RING)
CENTRE = (0.5, 0.5, 0.5)
UP = (0.0, 1.0, 0.0)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "pr1"])
    ap.add_argument("--no-extra", action="store_true", help="skip the legs beside the main timed region")
    ap.add_argument("--cpu-frames", type=int, default=-1,
                    help="oracle frames for the CPU baseline (0: skip; -1: 6 on the 64M-point workload, else 60)")
    ap.add_argument("--cpu-omp-seconds", type=float, default=8.0,
                    help="seconds of OpenMP CPU-baseline frames on all host cores (0: skip)")
    ap.add_argument("--points", type=int, default=0, help="override the point count (profiling cases)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="position storage of the main timed region (16-bit: profiling cases, with --no-extra)")
    ap.add_argument("--marker", type=float, default=0.0,
                    help="disc marker radius in pixels for the main timed region (profiling cases, with --no-extra)")
    ap.add_argument("--serve-viewers", type=int, default=0,
                    help="with --leg served: that many viewers of --serve-resolution on the engine for --steps "
                         "ticks back to back, instead of the trace (profiling cases)")
    ap.add_argument("--serve-resolution", default="1920x1080", help="WxH of the --serve-viewers viewers")
    ap.add_argument("--leg", default="all", choices=["all", "batched", "served"],
                    help="run one leg alone (profiling cases): batched = the 256-cloud batch for --steps frames, "
                         "served = the zero-copy serving trace of --serve-requests requests")
    ap.add_argument("--serve-requests", type=int, default=10_000, help="frame requests of the serving trace")
    ap.add_argument("--launch", default="",
                    help="threads,ctas_per_sm,kernel for the point kernel, kernel a code or one of grid, tma, "
                         "depth_bound, warp_agg, auto (default: the library's choice)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def scene_for(name, points=0):
    import dataclasses
    sc = {"c2": inputs.C2, "pr1": inputs.PR1, "c3": inputs.C3}[name]
    if points:
        sc = dataclasses.replace(sc, n=points, name=f"{sc.name}_n{points}")
    return sc


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


_POINT_SOURCES = ("mmr_device.cuh", "mmr_kernels.cu", "mmr_launch.cuh", "mmr_points.cuh", "mmr_tiles.cuh")
KERNEL_SOURCES = {
    "points_kernel_f32_fused": _POINT_SOURCES,
    "points_kernel_f32_fused_depth_bound": _POINT_SOURCES,
    "points_kernel_narrow_f16_fused": _POINT_SOURCES,
    "points_kernel_narrow_f16_fused_depth_bound": _POINT_SOURCES,
    "points_kernel_narrow_bf16_fused": _POINT_SOURCES,
    "points_kernel_narrow_bf16_fused_depth_bound": _POINT_SOURCES,
}


def kernel_source_hash(kernel: str) -> str:
    """Hash of the source files that define `kernel` (ties a committed ncu
    traffic figure to the code it was measured on)."""
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2504_20937_b300", "csrc", fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    if kernel not in KERNEL_SOURCES:
        return None
    src = kernel_source_hash(kernel)
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) >= 4 and parts[0] == kernel and parts[1] == workload and parts[2] == src:
                return float(parts[3])
    return None


class Clocks:
    """nvidia-smi sampler run during a timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.file:
            return None
        try:
            text = open(self.file.name).read()
            os.unlink(self.file.name)
        except Exception:
            return None
        return summarize_clock_samples(text)


def summarize_clock_samples(text: str):
    """Median SM clock under load (samples above half the highest), the
    maximum SM clock and the throttle reasons seen Active, from nvidia-smi
    rows of Clocks.FIELDS (csv, no header, no units); None without a sample."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        r = [v.strip() for v in line.split(",")]
        try:
            s, m = float(r[0]), float(r[1])
        except (ValueError, IndexError):
            continue
        sm.append(s)
        mx.append(m)
        for name, v in zip(names, r[3:7]):
            if v == "Active":
                reasons.add(name)
    if not sm:
        return None
    busy = [s for s in sm if s > 0.5 * max(sm)]
    return {"sm_mhz": statistics.median(busy or sm), "sm_max_mhz": max(mx), "samples": len(sm),
            "reasons": sorted(reasons)}


# ----------------------------------------------------------- multi-rank glue

def reduce_max(value: float) -> float:
    """Max of `value` over all ranks (the value itself in a single process).
    Each rank runs an independent replica of the workload, so this timing
    reduction is the only collective."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


# --------------------------------------------------------------------- ours

def needs_flush(sc, storage) -> bool:
    """L2 is flushed before every timed frame unless the positions alone are
    larger than L2 (126 MB), in which case a frame cannot find the previous
    frame's positions there anyway."""
    return sc.n * inputs.BYTES_PER_POINT[storage] < L2_BYTES


def run_ours(args, rank, world, local):
    import torch
    from paper_2504_20937_b300.api import Context

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = scene_for(args.workload, args.points)
    pos64 = sc.positions()
    stored = inputs.encode(pos64, "f32")
    flush = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_sink = torch.zeros((), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def make_ctx(dtype="f32", data=stored, scene=sc):
        ctx = Context(scene.W, scene.H)
        view = ctx.alloc_points(data.shape[0], dtype)
        view.copy_(torch.from_numpy(data if dtype == "f32" else data.view(np.int16)))
        ctx.set_sim(scene.philox_seed, 0, scene.amplitude, 0)
        ctx.set_style(scene.color, scene.background)
        if args.marker:
            ctx.set_marker(args.marker)
        if args.launch:
            t, c, k = args.launch.split(",")
            ctx.set_launch(int(t), int(c), int(k) if k.isdigit() else k)
        torch.cuda.synchronize()
        return ctx

    def timed_frames(ctx, scene, frames, warm, do_flush, roundtrip=None, kernel_times=False):
        """Per-frame device times (ms) of the whole step and, with
        kernel_times (the library's per-kernel events switched on), of the
        point phase and the resolve.  The warm-up frames run and finish
        first; then all timed frames are enqueued back to back, each between
        two CUDA events on the launching stream (after its L2 flush, when
        flushing), and read once the last one has finished, so the GPU is
        never idle waiting for the host between frames.  With kernel_times
        (up to the library's ring of frames, no host round trip) the
        library's own events bracket each frame (before the point phase,
        between it and the resolve, after the resolve), so no other event is
        recorded and a frame's time is its point phase plus its resolve."""
        ctx.set_timing(kernel_times)
        for f in range(warm):
            ctx.set_camera(scene.eye(f), CENTRE, UP, scene.fovy_deg, scene.znear, scene.zfar)
            if do_flush:
                flush_sink.copy_(flush.sum())
            if roundtrip is None:
                ctx.step_and_render(stream)
            else:
                ctx.step_and_render_roundtrip(stream, pinned=roundtrip)
        torch.cuda.synchronize()
        ctx.set_timing(kernel_times)           # restarts the library's count: frames_back below are timed frames
        own_events = kernel_times and frames <= TIMING_RING and roundtrip is None
        marks = []
        for f in range(warm, warm + frames):
            ctx.set_camera(scene.eye(f), CENTRE, UP, scene.fovy_deg, scene.znear, scene.zfar)
            if do_flush:
                flush_sink.copy_(flush.sum())     # reads 512 MB: evicts L2 without dirtying it
            if not own_events:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            if roundtrip is None:
                ctx.step_and_render(stream)
            else:
                ctx.step_and_render_roundtrip(stream, pinned=roundtrip)
            if not own_events:
                b.record(stream)
                marks.append((a, b))
        torch.cuda.synchronize()
        point_ms, resolve_ms = [0.0] * frames, [0.0] * frames
        if kernel_times:
            kept = min(frames, TIMING_RING)
            times = [ctx.frame_kernel_ms(k) for k in range(kept)][::-1]      # oldest kept frame first
            point_ms, resolve_ms = [t[0] for t in times], [t[1] for t in times]
        if own_events:
            return [p + r for p, r in zip(point_ms, resolve_ms)], point_ms, resolve_ms
        return [a.elapsed_time(b) for a, b in marks], point_ms, resolve_ms

    storage = args.storage
    do_flush = needs_flush(sc, storage)
    free_before = torch.cuda.mem_get_info(local)[0]
    ctx = make_ctx(storage, stored if storage == "f32" else inputs.encode(pos64, storage))
    zero_copy_bytes = ctx.device_bytes
    zero_copy_measured = free_before - torch.cuda.mem_get_info(local)[0]   # cudaMemGetInfo delta
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        # the timed region: K frames, each bracketed by CUDA events on the launching stream, with the
        # library's events around the point phase and the resolve of the same frames (the kernel durations
        # of the roofline come from the timed region itself)
        t0 = time.perf_counter()
        step_ms, point_ms, resolve_ms = timed_frames(ctx, sc, args.steps, args.warmup, do_flush, kernel_times=True)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        kernel_frames = min(args.steps, TIMING_RING)
        # four more repeats of the same K frames without the kernel events: the spread between repeats and
        # what the events cost (`value` is the timed region's)
        repeat_ms = [sum(step_ms) / args.steps]
        for _ in range(4):
            r_ms, _, _ = timed_frames(ctx, sc, args.steps, 0, do_flush)
            repeat_ms.append(sum(r_ms) / args.steps)
    launches_per_frame = ctx.last_frame_kernels()
    total_ms = reduce_max(sum(step_ms))
    if world > 1:
        torch.distributed.barrier()
    n = sc.n
    pts_per_s = job_rate(args.steps * n, world, total_ms)
    hbm_gbs, peak_kind = measured_peaks()
    bytes_point = 2 * inputs.BYTES_PER_POINT[storage] * n
    bytes_frame = bytes_point + 20 * sc.W * sc.H
    mean_point_ms = statistics.mean(point_ms)
    achieved = bytes_point / (mean_point_ms / 1e3) / 1e9
    bounded = launches_per_frame == 4
    kernel_name = ("points_kernel_f32_fused" if storage == "f32" else f"points_kernel_narrow_{storage}_fused") + \
        ("_depth_bound" if bounded else "")
    traffic = profiled_traffic(kernel_name, sc.name)
    kernel = "points_kernel<f32, displace, splat>" if storage == "f32" else \
        f"points_kernel_narrow<{storage}, displace, splat>"
    if bounded:
        kernel = f"point phase with screen-tile depth bounds: {kernel} on the first eighth of the points " \
                 f"(marking splat), tile_bound_kernel, {kernel} on the rest (bounded splat)"
    l2_note = (f"flushed before every timed frame ({FLUSH_BYTES >> 20} MB read)" if do_flush else
               f"not flushed: the {n * inputs.BYTES_PER_POINT[storage] / 1e6:.0f} MB of positions are larger "
               f"than L2 ({L2_BYTES >> 20} MB)")

    out = {
        "metric": METRIC, "value": pts_per_s, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": storage,
        "data": f"synthetic ({'16-cluster Gaussian mixture' if sc.cloud == 'gmm16' else 'uniform'} cloud, "
                "numpy PCG64)",
        "config": {"workload": sc.name, "points": n, "width": sc.W, "height": sc.H,
                   "storage": storage, "amplitude": sc.amplitude, "orbit_deg_per_frame": sc.deg_per_frame,
                   "l2": l2_note, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "launch": args.launch or "library default"},
        "roofline": {"bound": "hbm", "kernel": kernel,
                     "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
                     "traffic": traffic, "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_point},
        "gpu_launches": launches_per_frame * args.steps,
        "frames_per_s": job_rate(args.steps, world, total_ms),
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "hbm_gbs_step": bytes_frame / (total_ms / args.steps / 1e3) / 1e9,
        "frac_step": bytes_frame / (total_ms / args.steps / 1e3) / 1e9 / hbm_gbs,
        "kernels_ms": {"point_phase": mean_point_ms, "resolve": statistics.mean(resolve_ms),
                       "launches_per_frame": launches_per_frame,
                       "frames": kernel_frames,
                       "note": "the library's CUDA events before the point phase, between it and the resolve, and "
                               "after the resolve of every frame of the timed region; they are also the frames' "
                               "own brackets there (a frame's time is its point phase plus its resolve)"},
        "repeats": {"ms_per_step": repeat_ms, "median_ms_per_step": float(np.median(repeat_ms)),
                    "note": "the timed region (bracketed by the library's per-kernel events) and four more runs of "
                            "the same K frames bracketed by two events each instead; value is the first"},
        "wall_s_timed_region": wall,
        "device_bytes": {"zero_copy": zero_copy_bytes, "zero_copy_cudaMemGetInfo": zero_copy_measured},
    }
    clocks = clk.summary()
    if clocks:
        out["clocks"] = clocks

    if rank == 0 and not args.no_extra:
        # end to end through the public API: camera in, every frame read back to pinned host memory
        e2e_frames = min(args.steps, 300 if sc.W * sc.H <= 1 << 22 else 100)
        serial_s = e2e_readback(ctx, sc, e2e_frames, stream, pipelined=False)
        full_s = e2e_readback(ctx, sc, e2e_frames, stream, pipelined=True)
        mirror_s, mirror_bytes, mirror_ok = e2e_mirror(ctx, sc, e2e_frames, stream)
        out["e2e"] = {"value": e2e_frames * n / mirror_s, "unit": "points/s", "h2d_bytes_per_step": 64,
                      "d2h_bytes_per_step": mirror_bytes, "frames": e2e_frames,
                      "mirror_equals_device_frame": mirror_ok,
                      "note": "camera matrix in as kernel parameters; every frame delivered to the library's "
                              "host mirror of the framebuffer (mmr_mirror_frame on a second, high-priority stream: only the "
                              "64-pixel runs that changed since the mirror's last update cross the host link, "
                              "overlapping the next frame's point phase); d2h bytes counted by the library; all "
                              "updates complete inside the timed region; the mirror's first, whole-frame fill "
                              "happens before it"}
        out["e2e_full_frame"] = {"value": e2e_frames * n / full_s, "unit": "points/s", "h2d_bytes_per_step": 64,
                                 "d2h_bytes_per_step": 4 * sc.W * sc.H, "frames": e2e_frames,
                                 "note": "every frame's whole RGBA copied to pinned host memory, the copy of "
                                         "frame f overlapping the compute of frame f+1 (two device staging "
                                         "buffers, a copy stream, the host waits for frame f-2 before reusing "
                                         "its buffer)"}
        out["e2e_serial"] = {"value": e2e_frames * n / serial_s, "unit": "points/s", "frames": e2e_frames,
                             "note": "the whole frame copied on the compute stream, synchronised after every "
                                     "frame (no overlap)"}
        # host round trip (pinned), same frames: the paper's RAM-based comparison
        rt_frames = min(args.steps, 200 if n <= 1 << 22 else 20)
        rt_ms, _, _ = timed_frames(ctx, sc, rt_frames, 3, do_flush, roundtrip=True)
        out["device_bytes"]["roundtrip"] = ctx.device_bytes
        out["device_bytes"]["roundtrip_cudaMemGetInfo"] = free_before - torch.cuda.mem_get_info(local)[0]
        out["roundtrip_pinned"] = {"points_per_s": rt_frames * n / (sum(rt_ms) / 1e3),
                                   "frames_per_s": rt_frames / (sum(rt_ms) / 1e3),
                                   "p50_ms": float(np.percentile(rt_ms, 50)),
                                   "p99_ms": float(np.percentile(rt_ms, 99)), "frames": rt_frames,
                                   "host_bytes_per_frame": 2 * inputs.BYTES_PER_POINT[storage] * n}
        pg_frames = 20 if n <= 1 << 22 else 5
        pg_ms, _, _ = timed_frames(ctx, sc, pg_frames, 2, do_flush, roundtrip=False)
        out["roundtrip_pageable"] = {"points_per_s": pg_frames * n / (sum(pg_ms) / 1e3),
                                     "p99_ms": float(np.percentile(pg_ms, 99)), "frames": pg_frames}
        out["zero_copy_vs_roundtrip_pinned"] = out["value"] / world / out["roundtrip_pinned"]["points_per_s"]
        ctx.close()
        # error of one step against the FP64 oracle, for this storage type and the others
        fp64 = {storage: storage_accuracy(make_ctx, sc, pos64, storage)}
        others = [d for d in ("f32", "f16", "bf16") if d != storage]
        legs = run_storage_legs(make_ctx, timed_frames, hbm_gbs, sc, pos64, others, do_flush)
        for d in others:
            fp64[d] = storage_accuracy(make_ctx, sc, pos64, d)
        out["fp64_error"] = fp64
        out[f"{sc.name}_other_storage"] = legs
        if sc is not inputs.C2 and not args.points:
            out[inputs.C2.name] = run_c2_leg(make_ctx, timed_frames, hbm_gbs)
        out["features_c2"] = run_features(inputs.C2, inputs.encode(inputs.C2.positions(), "f32"), hbm_gbs)
        out["nbody"] = run_nbody()
        out["batched_256_clouds"] = run_batched(hbm_gbs)
        out["served"] = run_served(args.serve_requests)
    else:
        ctx.close()
    return out


def storage_accuracy(make_ctx, sc, pos64, dtype):
    """One step of the workload in `dtype` storage on the GPU, against the
    same step taken by the FP64 oracle from the same stored input
    (oracle/accuracy.py, on the host, outside every timed region)."""
    from oracle import accuracy
    stored = inputs.encode(pos64, dtype)
    ctx = make_ctx(dtype, stored, sc)
    ctx.set_camera(sc.eye(0), CENTRE, UP, sc.fovy_deg, sc.znear, sc.zfar)
    ctx.step_and_render()
    got = ctx.points.cpu().numpy()
    rgba = ctx.frame_rgba().cpu().numpy().reshape(-1).view(np.uint32)
    ctx.close()
    got = got if dtype == "f32" else got.view(np.uint16)
    rep = accuracy.step_accuracy(stored, dtype, got, rgba, sc.philox_seed, 0, 0, sc.amplitude, sc.eye(0), CENTRE,
                                 UP, sc.fovy_deg, sc.W, sc.H, sc.znear, sc.zfar, sc.color, sc.background)
    rep["note"] = ("one step from the stored input: relative error |x - x64| / max(|x64|, 2^-14); RGBA agreement "
                   "with the oracle's frame of the FP64 positions, over all pixels and over pixels covered in "
                   "either; at-risk pixels: those the stated rounding bound lets change (None when it reaches "
                   "a pixel)")
    return rep


def e2e_mirror(ctx, sc, frames, stream):
    """Seconds for `frames` frames through the public API, each with its
    camera set and the library's host mirror brought up to it by
    mmr_mirror_frame on a second stream of the highest priority; the loop ends when the last update
    has landed.  Returns (seconds, d2h bytes per frame as counted by the
    library, whether the mirror then equals the device framebuffer)."""
    import torch
    mirror = ctx.alloc_host_mirror()
    # the update's CTAs go ahead of the next frame's point kernel (include/mmr.h)
    copy_stream = torch.cuda.Stream(priority=torch.cuda.Stream.priority_range()[1])
    ctx.set_camera(sc.eye(0), CENTRE, UP, sc.fovy_deg, sc.znear, sc.zfar)
    ctx.step_and_render(stream)
    ctx.mirror_frame(copy_stream)             # the first update fills the whole mirror
    torch.cuda.synchronize()
    b0 = ctx.mirror_bytes()
    t0 = time.perf_counter()
    for f in range(1, frames + 1):
        ctx.set_camera(sc.eye(f), CENTRE, UP, sc.fovy_deg, sc.znear, sc.zfar)
        ctx.step_and_render(stream)
        ctx.mirror_frame(copy_stream)
    copy_stream.synchronize()
    stream.synchronize()
    dt = time.perf_counter() - t0
    per_frame = (ctx.mirror_bytes() - b0) / frames
    dev = ctx.frame_rgba().cpu().numpy().view(np.uint32)
    return dt, per_frame, bool(np.array_equal(mirror, dev))


def e2e_readback(ctx, sc, frames, stream, pipelined):
    """Seconds for `frames` frames through the public API, each with its
    camera set and its RGBA frame delivered to pinned host memory.

    pipelined=False: copy on the compute stream and synchronise every frame.
    pipelined=True: the frame is first copied to one of two device staging
    buffers on the compute stream (so the next frame may overwrite the
    library's framebuffer), then to one of two pinned host buffers on a copy
    stream, overlapping the next frame's compute.  Before a staging or host
    buffer is reused the host waits for the copy that filled it two frames
    earlier (where a caller would take the frame); the loop ends when every
    copy has landed."""
    import torch
    W, H = sc.W, sc.H
    torch.cuda.synchronize()
    if not pipelined:
        host = torch.empty((H, W), dtype=torch.int32, pin_memory=True)
        t0 = time.perf_counter()
        for f in range(frames):
            ctx.set_camera(sc.eye(f), CENTRE, UP, sc.fovy_deg, sc.znear, sc.zfar)
            ctx.step_and_render(stream)
            with torch.cuda.stream(stream):
                host.copy_(ctx.frame_rgba(), non_blocking=True)
            stream.synchronize()
        return time.perf_counter() - t0
    copy_stream = torch.cuda.Stream()
    stage = [torch.empty((H, W), dtype=torch.int32, device="cuda") for _ in range(2)]
    host = [torch.empty((H, W), dtype=torch.int32, pin_memory=True) for _ in range(2)]
    staged = [torch.cuda.Event() for _ in range(2)]
    copied = [None, None]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for f in range(frames):
        slot = f & 1
        ctx.set_camera(sc.eye(f), CENTRE, UP, sc.fovy_deg, sc.znear, sc.zfar)
        ctx.step_and_render(stream)
        if copied[slot] is not None:
            copied[slot].synchronize()          # frame f-2 is on the host: its buffers are free
            stream.wait_event(copied[slot])
        with torch.cuda.stream(stream):
            stage[slot].copy_(ctx.frame_rgba(), non_blocking=True)
        staged[slot].record(stream)
        copy_stream.wait_event(staged[slot])
        with torch.cuda.stream(copy_stream):
            host[slot].copy_(stage[slot], non_blocking=True)
        done = torch.cuda.Event()
        done.record(copy_stream)
        copied[slot] = done
    for ev in copied:
        if ev is not None:
            ev.synchronize()
    dt = time.perf_counter() - t0
    if not torch.equal(host[(frames - 1) & 1], ctx.frame_rgba().cpu()):
        raise RuntimeError("pipelined read-back: the last frame on the host differs from the framebuffer")
    return dt


def run_storage_legs(make_ctx, timed_frames, hbm_gbs, sc, pos64, dtypes, do_flush, frames=20):
    """The same workload in the other storage types (FP32 compute): frame
    times with and without the per-kernel events."""
    res = {}
    for dtype in dtypes:
        data = inputs.encode(pos64, dtype)
        ctx = make_ctx(dtype, data, sc)
        step_ms, _, _ = timed_frames(ctx, sc, frames, 3, do_flush)
        _, point_ms, resolve_ms = timed_frames(ctx, sc, frames, 1, do_flush, kernel_times=True)
        ctx.close()
        bpp = inputs.BYTES_PER_POINT[dtype] * 2
        frame_bytes = bpp * sc.n + 20 * sc.W * sc.H
        mean_step = statistics.mean(step_ms)
        pk = statistics.mean(point_ms)
        res[dtype] = {"ms_per_frame": mean_step, "frames_per_s": 1e3 / mean_step,
                      "points_per_s": sc.n / (mean_step / 1e3),
                      "p99_ms": float(np.percentile(step_ms, 99)),
                      "frac_frame": frame_bytes / (mean_step / 1e3) / 1e9 / hbm_gbs,
                      "points_kernel_ms": pk, "resolve_ms": statistics.mean(resolve_ms),
                      "points_kernel_frac": bpp * sc.n / (pk / 1e3) / 1e9 / hbm_gbs}
        del data
    return res


def run_c2_leg(make_ctx, timed_frames, hbm_gbs, frames=200):
    """The 2^22-point 1920x1080 orbit (L2 flushed before every frame), zero
    copy and host round trip."""
    sc = inputs.C2
    stored = inputs.encode(sc.positions(), "f32")
    ctx = make_ctx("f32", stored, sc)
    step_ms, _, _ = timed_frames(ctx, sc, frames, 5, True)
    _, point_ms, resolve_ms = timed_frames(ctx, sc, frames, 3, True, kernel_times=True)
    rt_ms, _, _ = timed_frames(ctx, sc, 50, 3, True, roundtrip=True)
    ctx.close()
    m = statistics.mean(step_ms)
    pk = statistics.mean(point_ms)
    return {"ms_per_frame": m, "points_per_s": sc.n / (m / 1e3), "p99_ms": float(np.percentile(step_ms, 99)),
            "points_kernel_ms": pk, "resolve_ms": statistics.mean(resolve_ms),
            "points_kernel_frac": 24 * sc.n / (pk / 1e3) / 1e9 / hbm_gbs,
            "roundtrip_pinned_ms_per_frame": statistics.mean(rt_ms),
            "zero_copy_vs_roundtrip_pinned": statistics.mean(rt_ms) / m, "frames": frames,
            "l2": f"flushed before every frame ({FLUSH_BYTES >> 20} MB read)"}


def run_features(sc, stored, hbm_gbs, frames=50):
    """The same 2^22-point 1920x1080 orbit with the paper's other usage
    patterns: ping-pong buffers (step out of place into the other buffer),
    indexed colour (colormap[index[id]]), and disc markers of radius 1, 2,
    4, 8 and 16 pixels (the library's kernel choice: from 64 discs over each
    pixel, two passes around 32x32-tile depth bounds).  Per-frame CUDA
    events, L2 flushed by a 512 MB read."""
    import torch
    from paper_2504_20937_b300.api import Context
    dev = torch.cuda.current_device()
    flush = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sink = torch.zeros((), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    res = {}

    def time_frames(ctx, step):
        marks = []
        for f in range(frames + 3):
            ctx.set_camera(sc.eye(f), CENTRE, UP, sc.fovy_deg, sc.znear, sc.zfar)
            sink.copy_(flush.sum())
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(ctx)
            b.record(stream)
            if f >= 3:
                marks.append((a, b))
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in marks]
        m = statistics.mean(ms)
        return {"ms_per_frame": m, "points_per_s": sc.n / (m / 1e3), "p99_ms": float(np.percentile(ms, 99)),
                "launches_per_frame": ctx.last_frame_kernels()}

    cases = [("pingpong", 0.0, False, True), ("indexed_colour", 0.0, True, False)]
    cases += [(f"disc_r{r:g}", r, False, False) for r in (1.0, 2.0, 4.0, 8.0, 16.0)]
    for name, radius, indexed, pingpong in cases:
        with Context(sc.W, sc.H) as ctx:
            if pingpong:
                ctx.alloc_pingpong(sc.n, "f32")[0].copy_(torch.from_numpy(stored))
            else:
                ctx.alloc_points(sc.n, "f32").copy_(torch.from_numpy(stored))
            if indexed:
                idx, cm = ctx.alloc_indexed_colors(9)
                idx.copy_(torch.arange(sc.n, dtype=torch.int32, device=dev) % 9)
                cm.copy_(torch.arange(9, dtype=torch.int32, device=dev) * 0x1C1C1C)
            ctx.set_sim(sc.philox_seed, 0, sc.amplitude, 0)
            ctx.set_marker(radius)
            torch.cuda.synchronize()
            step = (lambda c: c.step_and_render_pingpong(stream)) if pingpong else (lambda c: c.step_and_render(stream))
            res[name] = time_frames(ctx, step)
    return res


def run_nbody(sizes=(16384, 65536), steps=10):
    """Second workload: all-pairs gravity feeding the renderer (1920x1080),
    one fused step+splat kernel plus resolve per frame.  Compute-bound: the
    roofline is the FP32 issue rate (no FMA contraction on this path), here
    counted as 20 FP32 operations per interaction (sqrt and divide as one
    each) against 148 SMs x 128 lanes x the measured SM clock."""
    import torch
    from paper_2504_20937_b300.api import Context
    out = {}
    stream = torch.cuda.current_stream()
    for n in sizes:
        pos = inputs.encode(inputs.gaussian_mixture_cloud(n, 70, components=4, sigma=0.05), "f32")
        with Context(1920, 1080) as ctx:
            ctx.alloc_pingpong(n, "f32")[0].copy_(torch.from_numpy(pos))
            v, m = ctx.alloc_nbody()
            m.fill_(1.0 / n)
            ctx.set_timing(True)
            ms = []
            for f in range(steps + 2):
                ctx.set_camera(inputs.orbit_eye(f, 0.36), CENTRE, UP, 60.0, 0.1, 100.0)
                ctx.nbody_step_and_render(1e-3, 1e-4, 1e-3, stream)
                pk, rk = ctx.last_kernel_ms()
                if f >= 2:
                    ms.append(pk)
        k = statistics.mean(ms)
        inter = float(n) * n
        out[f"n{n}"] = {"nbody_kernel_ms": k, "interactions_per_s": inter / (k / 1e3),
                        "gflops_20_per_interaction": 20 * inter / (k / 1e3) / 1e9}
    return out


def run_batched(hbm_gbs, frames=100):
    """256 clouds of log-uniform size 1e3..1e6 (uniform or 4-cluster), each
    with its own orbit camera and resolution from {256^2, 512^2, 1024^2}:
    autotuned, then `frames` frames replayed from a one-frame CUDA graph."""
    import torch
    from paper_2504_20937_b300.api import Batch
    table = inputs.batched_table()
    clouds = [dict(n=bc.n, width=bc.W, height=bc.H, seed=4, cloud=i, amplitude=5e-4) for i, bc in enumerate(table)]
    stream = torch.cuda.current_stream()
    starts = {}
    with Batch(clouds, "f32", camera_slots=frames) as b:
        for i, bc in enumerate(table):
            stored = inputs.encode(inputs.batch_cloud_positions(bc), "f32")
            if i in BATCH_ACCURACY_CLOUDS:
                starts[i] = stored
            b.points(i).copy_(torch.from_numpy(stored))
            for f in range(frames):
                eye = inputs.orbit_eye(f, bc.deg_per_frame, bc.radius, CENTRE, bc.elevation, bc.start_deg)
                b.set_camera(i, f, eye, CENTRE, UP, 60.0, 0.1, 100.0)
        torch.cuda.synchronize()
        # the first frame of a sample of clouds against the FP64 oracle (host side, before any timing)
        b.step_and_render(stream)
        torch.cuda.synchronize()
        fp64 = batch_accuracy(b, table, clouds, starts)
        tuned = b.autotune(frames_per_config=2, stream=stream)
        b.run_graph(3, stream)                                   # warm-up frames
        per_frame = []
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for f in range(frames):
            a = torch.cuda.Event(enable_timing=True)
            z = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.run_graph(1, stream)
            z.record(stream)
            per_frame.append((a, z))
        t1.record(stream)
        torch.cuda.synchronize()
        total_ms = t0.elapsed_time(t1)
        frame_ms = [a.elapsed_time(z) for a, z in per_frame]
        # the same frames by the host round trip: displace, all positions device -> pinned host -> device, render
        rt_frames = max(3, min(frames // 10, 10))
        b.step_and_render_roundtrip(stream, pinned=True)          # allocates the host and device copies
        rt_ms = []
        for f in range(rt_frames):
            a = torch.cuda.Event(enable_timing=True)
            z = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.step_and_render_roundtrip(stream, pinned=True)
            z.record(stream)
            z.synchronize()
            rt_ms.append(a.elapsed_time(z))
        b.check_device()
    n_pts = sum(c["n"] for c in clouds)
    n_px = sum(c["width"] * c["height"] for c in clouds)
    bytes_frame = 24 * n_pts + 20 * n_px
    ms = total_ms / frames
    return {"clouds": len(clouds), "points": n_pts, "pixels": n_px, "frames": frames, "autotuned": tuned,
            "ms_per_frame": ms, "p50_ms": float(np.percentile(frame_ms, 50)),
            "p99_ms": float(np.percentile(frame_ms, 99)), "points_per_s": n_pts / (ms / 1e3),
            "cloud_frames_per_s": len(clouds) / (ms / 1e3),
            "hbm_gbs_frame": bytes_frame / (ms / 1e3) / 1e9, "frac_frame": bytes_frame / (ms / 1e3) / 1e9 / hbm_gbs,
            "roundtrip_pinned": {"ms_per_frame": statistics.mean(rt_ms), "p50_ms": float(np.percentile(rt_ms, 50)),
                                 "p99_ms": float(np.percentile(rt_ms, 99)), "frames": rt_frames,
                                 "points_per_s": n_pts / (statistics.mean(rt_ms) / 1e3),
                                 "host_bytes_per_frame": 2 * 12 * n_pts},
            "zero_copy_vs_roundtrip": statistics.mean(rt_ms) / ms, "fp64_error": fp64,
            "launch": "counter resets + one persistent launch (point items, then each cloud's pixel items one resident grid later) + frame counter, replayed as a CUDA graph"}


BATCH_ACCURACY_CLOUDS = (0, 1, 2, 3, 64, 128, 192, 255)


def batch_accuracy(b, table, clouds, starts):
    """First batched frame of a sample of clouds against the FP64 oracle:
    the worst figures over the sample (oracle/accuracy.py)."""
    from oracle import accuracy
    reps = {}
    for i, stored in starts.items():
        bc, c = table[i], clouds[i]
        eye = inputs.orbit_eye(0, bc.deg_per_frame, bc.radius, CENTRE, bc.elevation, bc.start_deg)
        got = b.points(i).cpu().numpy().reshape(-1, 3)
        rgba = b.frame_rgba(i).cpu().numpy().reshape(-1).view(np.uint32)
        reps[i] = accuracy.step_accuracy(stored, "f32", got, rgba, c["seed"], c["cloud"], 0, c["amplitude"], eye,
                                         CENTRE, UP, 60.0, bc.W, bc.H, 0.1, 100.0)
    vals = list(reps.values())
    return {"clouds": sorted(reps), "max_rel": max(r["max_rel"] for r in vals),
            "rms_rel_max": max(r["rms_rel"] for r in vals),
            "pixels_all_agree_min": min(r["pixels_all_agree"] for r in vals),
            "pixels_covered_agree_min": min(r["pixels_covered_agree"] for r in vals),
            "differing_outside_risk": sum(r["differing_outside_risk"] or 0 for r in vals)}


def served_accuracy(cfg, shared):
    """One tick of the serving engine with one 1920x1080 viewer against the
    FP64 oracle: the shared cloud (step = tick 0) and the viewer's private
    cloud (step = its frame 0) in one frame, point ids in that order.  Both
    clouds are drawn in one colour so the frame is the coverage mask."""
    import torch
    from oracle import accuracy
    from paper_2504_20937_b300 import serve
    from paper_2504_20937_b300.api import Server
    req = inputs.ViewerRequest(viewer=0, arrival_s=0.0, W=1920, H=1080, frames=1, private_n=200_000,
                               start_deg=30.0, init_seed=77)
    private = serve.private_cloud(req, cfg.dtype)
    with Server(cfg.shared_n, cfg.dtype, cfg.shared_seed, 0, cfg.amplitude, cfg.budget_bytes) as srv:
        srv.shared_points().copy_(torch.from_numpy(shared))
        srv.set_shared_color(0xFFFFFFFF)
        v = srv.add_viewer(req.private_n, req.W, req.H, seed=req.init_seed, cloud=1, amplitude=cfg.amplitude,
                           color=0xFFFFFFFF)
        srv.viewer_points(v).copy_(torch.from_numpy(private))
        eye = serve.viewer_eye(req, 0, cfg)
        srv.set_camera(v, eye, CENTRE, UP, cfg.fovy_deg, cfg.znear, cfg.zfar)
        srv.tick()
        torch.cuda.synchronize()
        got_shared = srv.shared_points().cpu().numpy().reshape(-1, 3)
        got_private = srv.viewer_points(v).cpu().numpy().reshape(-1, 3)
        rgba = srv.frame(v)[0].cpu().numpy().reshape(-1).view(np.uint32)
    segs = [{"stored_before": shared, "got_after": got_shared, "seed": cfg.shared_seed, "cloud": 0, "step": 0,
             "amplitude": cfg.amplitude},
            {"stored_before": private, "got_after": got_private, "seed": req.init_seed, "cloud": 1, "step": 0,
             "amplitude": cfg.amplitude}]
    rep = accuracy.segments_accuracy(segs, cfg.dtype, rgba, eye, CENTRE, UP, cfg.fovy_deg, req.W, req.H,
                                     cfg.znear, cfg.zfar)
    rep["case"] = f"shared {cfg.shared_n} + private {req.private_n} points, one viewer at {req.W}x{req.H}"
    return rep


def run_served(requests=10_000, roundtrip=True):
    """Continuous batching: shared 2^24-point cloud, Poisson viewer arrivals,
    private clouds 1e4..1e6 points, 640x480 / 1920x1080 / 3840x2160, at most
    64 viewers under a 40 GB budget.  Viewers are paced by a 60 Hz display
    (one frame per viewer per refresh), so the zero-copy engine and the host
    round trip (the shared cloud device -> host -> device every tick) serve
    the same trace at the same concurrency; their latencies compare at equal
    load.  Saturation throughput is measured apart: ticks back to back with
    the paced run's mean number of viewers always on the engine."""
    import dataclasses
    from paper_2504_20937_b300 import serve
    trace = inputs.serving_trace(requests=requests)
    cfg = serve.ServeConfig()
    shared = inputs.encode(inputs.uniform_cloud(cfg.shared_n, cfg.shared_seed), cfg.dtype)
    clouds = {r.viewer: serve.private_cloud(r, cfg.dtype) for r in trace}
    fp64 = served_accuracy(cfg, shared) if roundtrip else None
    zero = serve.run_trace(trace, cfg, clouds=clouds, shared=shared).summary()
    out = {"requests": requests, "viewers": len(trace), "shared_points": cfg.shared_n,
           "max_concurrent": cfg.max_viewers, "budget_gb": cfg.budget_bytes / 2**30, "display_hz": cfg.tick_hz,
           "zero_copy": zero}
    if roundtrip:
        out["roundtrip"] = serve.run_trace(trace, cfg, roundtrip=True, clouds=clouds, shared=shared).summary()
        # saturation: the same viewers all waiting at the start, as many on the engine as the paced mean
        v = max(1, round(zero["mean_active_viewers_steady"]))
        sat_trace = [dataclasses.replace(r, arrival_s=0.0) for r in trace[:2 * v]]
        sat_cfg = dataclasses.replace(cfg, tick_hz=0.0, max_viewers=v)
        sat = {"viewers_on_engine": v, "frames": sum(r.frames for r in sat_trace)}
        for name, rt in (("zero_copy", False), ("roundtrip", True)):
            r = serve.run_trace(sat_trace, sat_cfg, roundtrip=rt, clouds=clouds, shared=shared).summary()
            sat[name] = {"frames_per_s": r["frames_per_s"], "points_per_s": r["points_per_s"],
                         "mean_tick_ms": r["mean_tick_ms"], "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"]}
        out["saturation"] = sat
        out["fp64_error"] = fp64
    out["latency_note"] = ("paced runs: a frame's latency runs from the display refresh that asked for it (from "
                           "the viewer's arrival for its first frame) to the completion of the tick that rendered "
                           "it; wall clock, host overheads included; refreshes a running tick overlaps are dropped "
                           "and counted")
    return out


def run_served_fixed(viewers, W, H, ticks, warm):
    """`viewers` viewers of W x H (private clouds of 10^5 points) on the
    serving engine with the 2^24-point shared cloud, `ticks` ticks back to
    back after `warm` untimed ones: a small, steady case for profilers."""
    import torch
    from paper_2504_20937_b300 import serve
    from paper_2504_20937_b300.api import Server
    cfg = serve.ServeConfig()
    shared = inputs.encode(inputs.uniform_cloud(cfg.shared_n, cfg.shared_seed), cfg.dtype)
    stream = torch.cuda.current_stream()
    with Server(cfg.shared_n, cfg.dtype, cfg.shared_seed, 0, cfg.amplitude, cfg.budget_bytes) as srv:
        srv.shared_points().copy_(torch.from_numpy(shared))
        vids = []
        for v in range(viewers):
            vid = srv.add_viewer(100_000, W, H, seed=100 + v, cloud=1 + v, amplitude=cfg.amplitude)
            srv.viewer_points(vid).copy_(torch.from_numpy(inputs.encode(inputs.uniform_cloud(100_000, 100 + v),
                                                                         cfg.dtype)))
            vids.append(vid)
        srv.set_timing(True)
        ms = []
        for t in range(warm + ticks):
            for k, vid in enumerate(vids):
                srv.set_camera(vid, inputs.orbit_eye(t, 0.36, 2.0, CENTRE, 0.0, 360.0 * k / viewers), CENTRE, UP,
                               cfg.fovy_deg, cfg.znear, cfg.zfar)
            srv.tick(stream)
            tick_ms = srv.last_tick_ms()
            if t >= warm:
                ms.append(tick_ms)
    return {"viewers": viewers, "resolution": f"{W}x{H}", "ticks": ticks, "mean_tick_ms": statistics.mean(ms),
            "frames_per_s": viewers / (statistics.mean(ms) / 1e3)}


# ---------------------------------------------------------------- reference

def cpu_oracle_rate(sc, stored, frames, points):
    """The oracle as it stands (single-threaded C) on `frames` frames of a
    `points`-point slice of the workload, full-size framebuffer."""
    import oracle
    pos = stored[:points].copy()
    t0 = time.perf_counter()
    for f in range(frames):
        oracle.displace_f32(pos, sc.philox_seed, 0, f, np.float32(sc.amplitude))
        M = oracle.camera_f32(sc.eye(f), CENTRE, UP, sc.fovy_deg, sc.aspect, sc.znear, sc.zfar)
        oracle.render(pos, "f32", M, sc.W, sc.H, np.float32(sc.znear), np.float32(sc.zfar))
    dt = time.perf_counter() - t0
    return frames * points / dt, dt


def cpu_omp_rate(sc, stored, seconds):
    """The oracle's frame over all host cores (OpenMP, oracle/mmr_cpu_omp.c):
    whole frames of the full workload, one untimed, then as many as fit in
    `seconds` (at least 3).  The frames equal the oracle's bit for bit."""
    import oracle
    pos = stored.copy()
    keys = np.empty(sc.W * sc.H, np.uint64)
    rgba = np.empty(sc.W * sc.H, np.uint32)

    def frame(f):
        M = oracle.camera_f32(sc.eye(f), CENTRE, UP, sc.fovy_deg, sc.aspect, sc.znear, sc.zfar)
        return oracle.cpu_omp_frame_f32(pos, sc.philox_seed, 0, f, sc.amplitude, M, sc.W, sc.H, sc.znear,
                                        sc.zfar, keys=keys, rgba=rgba)[2]

    threads = frame(0)
    t0 = time.perf_counter()
    frames = 0
    while frames < 3 or time.perf_counter() - t0 < seconds:
        frame(1 + frames)
        frames += 1
    dt = time.perf_counter() - t0
    return frames * sc.n / dt, dt, frames, threads


def run_reference(args, rank, world):
    if rank != 0:
        return None
    sc = scene_for(args.workload, args.points)
    stored = inputs.encode(sc.positions(), "f32")
    sample = min(sc.n, 1 << 20)
    cpu_oracle_rate(sc, stored, args.warmup, sample)     # warm-up steps, untimed
    rate, dt = cpu_oracle_rate(sc, stored, args.steps, sample)
    desc = (f"{args.steps} frames, each displacing and rendering the first {sample} of {sc.n} points "
            f"into the full {sc.W}x{sc.H} frame")
    return {"metric": METRIC, "value": rate, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": sc.name, "points": sc.n, "width": sc.W, "height": sc.H, "storage": "f32"},
            "cpu_baseline": {"value": rate, "unit": "points/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": rate, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if (args.storage != "f32" or args.marker) and not args.no_extra:
        raise SystemExit("--storage f16/bf16 and --marker time the main region only: add --no-extra")
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.leg != "all":
        # one leg alone, on one GPU: a small, self-contained command for profilers
        hbm_gbs, _ = measured_peaks()
        if args.leg == "batched":
            res = run_batched(hbm_gbs, frames=args.steps)
        elif args.serve_viewers:
            W, H = (int(v) for v in args.serve_resolution.split("x"))
            res = run_served_fixed(args.serve_viewers, W, H, args.steps, args.warmup)
        else:
            res = run_served(args.serve_requests, roundtrip=False)
        print(json.dumps({"leg": args.leg, args.leg: res}), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    out = run_ours(args, rank, world, local)
    if rank == 0:
        sc = scene_for(args.workload, args.points)
        frames = args.cpu_frames if args.cpu_frames >= 0 else (6 if sc.n > 1 << 24 else 60)
        stored = inputs.encode(sc.positions(), "f32") if frames > 0 or args.cpu_omp_seconds > 0 else None
        if frames > 0:
            rate, dt = cpu_oracle_rate(sc, stored, frames, sc.n)
            out["cpu_baseline"] = {"value": rate, "unit": "points/s", "cores": 1, "kind": "oracle",
                                   "sample": f"{frames} full frames ({sc.n} points, {sc.W}x{sc.H}) of the "
                                             f"workload on one host core, {dt:.1f} s"}
        if frames > 0 and not args.no_extra:
            # the oracle on one core for the other single-cloud configurations: the whole 100-step
            # reference run, and 20 frames of the other one (per-frame time)
            cfgs = {}
            pr1 = inputs.PR1
            rate, dt = cpu_oracle_rate(pr1, inputs.encode(pr1.positions(), "f32"), pr1.frames, pr1.n)
            cfgs[pr1.name] = {"points_per_s": rate, "seconds": dt, "frames": pr1.frames, "cores": 1}
            other, of = (inputs.C2, 20) if sc.name != inputs.C2.name else (inputs.C3, 3)
            rate, dt = cpu_oracle_rate(other, inputs.encode(other.positions(), "f32"), of, other.n)
            cfgs[other.name] = {"points_per_s": rate, "ms_per_frame": dt / of * 1e3, "frames": of, "cores": 1}
            out["cpu_baseline_configs"] = cfgs
        if args.cpu_omp_seconds > 0:
            rate, dt, omp_frames, threads = cpu_omp_rate(sc, stored, args.cpu_omp_seconds)
            out["cpu_baseline_openmp"] = {
                "value": rate, "unit": "points/s", "cores": threads, "kind": "oracle routines over OpenMP threads",
                "sample": f"{omp_frames} full frames ({sc.n} points, {sc.W}x{sc.H}) of the workload, {dt:.1f} s; "
                          f"host reports {os.cpu_count()} logical CPUs"}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
