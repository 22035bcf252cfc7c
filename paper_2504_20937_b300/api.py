"""Python face of libmmr: a thin object wrapper over the C ABI.

    ctx = Context(1920, 1080)
    pos = ctx.alloc_points(n, "f32")        # torch view of library-owned device memory
    pos.copy_(initial_positions)            # the simulation writes it directly
    ctx.set_camera(eye, target, up, 60.0, 0.1, 100.0)
    ctx.set_sim(seed, cloud=0, amplitude=5e-4)
    ctx.step_and_render()                    # enqueued on torch's current stream
    rgba = ctx.frame_rgba()                  # torch view of the device framebuffer

Mirrors the paper's usage model (Mimir, Listing 1 and Table 2): the
visualised allocation comes from the library and is written in place.
Every view handed out (points, framebuffer, keys, host mirror) aliases
memory the context owns: it must not be used after close().
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import DTYPE_CODE, MmrError, check, stream_handle

_TORCH_VIEW = {"f32": (torch.float32, "<f4"), "f16": (torch.int16, "<i2"), "bf16": (torch.int16, "<i2")}


class _DeviceArray:
    """Minimal __cuda_array_interface__ holder for a library-owned pointer."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2, "strides": None}


def device_view(ptr: int, shape, typestr: str) -> torch.Tensor:
    """A torch tensor aliasing device memory at ptr (no copy, no ownership)."""
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")


class Context:
    """One framebuffer, one point cloud, one camera (include/mmr.h)."""

    def __init__(self, width: int, height: int, budget_bytes: int = 0):
        lib = _lib.load()
        h = C.c_void_p()
        check(lib.mmr_create_ex(width, height, budget_bytes, C.byref(h)), None)
        self._lib = lib
        self._h = h
        self.W, self.H = width, height
        self.n = 0
        self.dtype = None
        self._points = None

    # -- lifetime
    def close(self):
        if self._h:
            self._lib.mmr_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        check(status, self._h)

    # -- data
    def alloc_points(self, n: int, dtype: str = "f32") -> torch.Tensor:
        p = C.c_void_p()
        self._check(self._lib.mmr_alloc_points(self._h, n, DTYPE_CODE[dtype], C.byref(p)))
        self.n, self.dtype = n, dtype
        tdt, typestr = _TORCH_VIEW[dtype]
        self._points = device_view(p.value, (n, 3), typestr)
        return self._points

    def alloc_pingpong(self, n: int, dtype: str = "f32"):
        """Two point buffers (views) for read-one / write-the-other simulations."""
        a, b = C.c_void_p(), C.c_void_p()
        self._check(self._lib.mmr_alloc_pingpong(self._h, n, DTYPE_CODE[dtype], C.byref(a), C.byref(b)))
        self.n, self.dtype = n, dtype
        typestr = _TORCH_VIEW[dtype][1]
        self._pp = (device_view(a.value, (n, 3), typestr), device_view(b.value, (n, 3), typestr))
        self._points = self._pp[0]
        return self._pp

    def set_visible(self, which: int):
        self._check(self._lib.mmr_set_visible(self._h, which))

    @property
    def visible(self) -> int:
        w = C.c_int()
        self._check(self._lib.mmr_get_visible(self._h, C.byref(w)))
        return w.value

    def step_and_render_pingpong(self, stream=None):
        self._check(self._lib.mmr_step_and_render_pingpong(self._h, stream_handle(stream)))

    def alloc_nbody(self):
        """(velocities float32[n,3] view, masses float32[n] view) for the
        N-body workload (needs FP32 ping-pong buffers)."""
        v, m = C.c_void_p(), C.c_void_p()
        self._check(self._lib.mmr_alloc_nbody(self._h, C.byref(v), C.byref(m)))
        return device_view(v.value, (self.n, 3), "<f4"), device_view(m.value, (self.n,), "<f4")

    def nbody_step_and_render(self, G: float, eps2: float, dt: float, stream=None):
        self._check(self._lib.mmr_nbody_step_and_render(self._h, G, eps2, dt, stream_handle(stream)))

    def alloc_indexed_colors(self, ncolors: int):
        """(index int32[n] view, colormap int32[ncolors] view)."""
        i, m = C.c_void_p(), C.c_void_p()
        self._check(self._lib.mmr_alloc_indexed_colors(self._h, ncolors, C.byref(i), C.byref(m)))
        return device_view(i.value, (self.n,), "<i4"), device_view(m.value, (ncolors,), "<i4")

    @property
    def points(self) -> torch.Tensor:
        """The visible point buffer."""
        if getattr(self, "_pp", None) is not None:
            return self._pp[self.visible]
        return self._points

    def alloc_colors(self) -> torch.Tensor:
        p = C.c_void_p()
        self._check(self._lib.mmr_alloc_colors(self._h, C.byref(p)))
        return device_view(p.value, (self.n,), "<i4")

    # -- parameters
    def set_camera(self, eye, target, up, fovy_deg, znear, zfar):
        d3 = C.c_double * 3
        self._check(self._lib.mmr_set_camera(self._h, d3(*eye), d3(*target), d3(*up), fovy_deg, znear, zfar))

    def set_matrix(self, m, znear, zfar):
        vals = [float(v) for v in torch.as_tensor(m, dtype=torch.float32).reshape(-1).tolist()]
        self._check(self._lib.mmr_set_matrix(self._h, (C.c_float * 16)(*vals), znear, zfar))

    def get_matrix(self):
        out = (C.c_float * 16)()
        self._check(self._lib.mmr_get_matrix(self._h, out))
        return list(out)

    def set_sim(self, seed: int, cloud: int = 0, amplitude: float = 1e-3, first_step: int = 0):
        self._check(self._lib.mmr_set_sim(self._h, seed, cloud, amplitude, first_step))

    def set_style(self, color: int = 0xFFFFFFFF, background: int = 0):
        self._check(self._lib.mmr_set_style(self._h, color, background))

    def set_marker(self, radius_px: float = 0.0):
        """0: 1-px points; 0.5..64: disc markers of that radius in pixels."""
        self._check(self._lib.mmr_set_marker(self._h, radius_px))

    def set_launch(self, threads: int = 64, ctas_per_sm: int = 0, kernel=0):
        """kernel (a code or a name of _lib.KERNEL_CODE): 0 "grid" grid-stride
        (ctas_per_sm 0 = one thread per group, else persistent with
        prefetch); 1 "tma" TMA-staged persistent; 2 "depth_bound" two passes
        with screen-tile depth bounds; 3 "warp_agg" warp-aggregated splat;
        4 "auto" depth bounds for dense clouds, else grid-stride."""
        code = _lib.KERNEL_CODE[kernel] if isinstance(kernel, str) else int(kernel)
        self._check(self._lib.mmr_set_launch(self._h, threads, ctas_per_sm, code))

    # -- frames
    def step_and_render(self, stream=None):
        self._check(self._lib.mmr_step_and_render(self._h, stream_handle(stream)))

    def displace(self, stream=None):
        self._check(self._lib.mmr_displace(self._h, stream_handle(stream)))

    def render(self, stream=None):
        self._check(self._lib.mmr_render(self._h, stream_handle(stream)))

    def step_and_render_roundtrip(self, stream=None, pinned: bool = True):
        self._check(self._lib.mmr_step_and_render_roundtrip(self._h, stream_handle(stream), int(pinned)))

    def frame_ptrs(self):
        r, k = C.c_void_p(), C.c_void_p()
        self._check(self._lib.mmr_frame_ptr(self._h, C.byref(r), C.byref(k)))
        return r.value, k.value

    def frame_rgba(self) -> torch.Tensor:
        """int32[H, W] view of the RGBA8 framebuffer (reinterpret as uint32)."""
        r, _ = self.frame_ptrs()
        return device_view(r, (self.H, self.W), "<i4")

    def frame_keys(self) -> torch.Tensor:
        """int64[H, W] view of the latest depth-id keys (reinterpret as uint64)."""
        _, k = self.frame_ptrs()
        return device_view(k, (self.H, self.W), "<i8")

    def check_device(self):
        """Raise MmrError(MMR_ERR_TIMEOUT) if a kernel gave up a bounded wait."""
        self._check(self._lib.mmr_check_device(self._h))

    def selftest_bounded_wait(self, max_cycles: int = 1_000_000, stream=None):
        """Run the bounded-wait self-test kernel (see include/mmr.h)."""
        self._check(self._lib.mmr_selftest_bounded_wait(self._h, max_cycles, stream_handle(stream)))

    def set_timing(self, enable: bool = True):
        self._check(self._lib.mmr_set_timing(self._h, int(enable)))

    def last_kernel_ms(self):
        """(point phase ms, resolve ms) of the latest timed frame."""
        a, b = C.c_float(), C.c_float()
        self._check(self._lib.mmr_last_kernel_ms(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def frame_kernel_ms(self, frames_back: int):
        """(point phase ms, resolve ms) of the timed frame `frames_back`
        frames before the latest (waits for it)."""
        a, b = C.c_float(), C.c_float()
        self._check(self._lib.mmr_frame_kernel_ms(self._h, frames_back, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_depth_bound_split(self, first_pass_shift: int = 3):
        """Depth-bound kernels: the first pass takes 2^-shift of the points."""
        self._check(self._lib.mmr_set_depth_bound_split(self._h, first_pass_shift))

    def last_frame_kernels(self) -> int:
        """Kernels the latest frame launched (point phase and resolve)."""
        k = C.c_int()
        self._check(self._lib.mmr_last_frame_kernels(self._h, C.byref(k)))
        return k.value

    @property
    def step(self) -> int:
        s = C.c_uint32()
        self._check(self._lib.mmr_get_step(self._h, C.byref(s)))
        return s.value

    @property
    def device_bytes(self) -> int:
        b = C.c_uint64()
        self._check(self._lib.mmr_device_bytes(self._h, C.byref(b)))
        return b.value

    def alloc_host_mirror(self):
        """numpy uint32[H, W] view of the library's host mirror of the
        framebuffer (pinned host memory); mirror_frame keeps it current."""
        import numpy as np
        p = C.c_void_p()
        self._check(self._lib.mmr_alloc_host_mirror(self._h, C.byref(p)))
        buf = (C.c_uint32 * (self.W * self.H)).from_address(p.value)
        self._mirror = np.ctypeslib.as_array(buf).reshape(self.H, self.W)
        return self._mirror

    def mirror_frame(self, stream=None):
        """Enqueue the update of the host mirror to the latest frame on
        `stream` (only the 64-pixel runs that changed cross the host link)."""
        self._check(self._lib.mmr_mirror_frame(self._h, stream_handle(stream)))

    def mirror_bytes(self) -> int:
        """Bytes written to the host mirror since it was allocated."""
        b = C.c_uint64()
        self._check(self._lib.mmr_mirror_bytes(self._h, C.byref(b)))
        return b.value


class Batch:
    """Many independent clouds advanced and rendered together (mmr_batch_*).

    clouds: list of dicts with n, width, height, seed, cloud, amplitude and
    optional color / background.
    """

    def __init__(self, clouds, dtype: str = "f32", camera_slots: int = 1, budget_bytes: int = 0):
        lib = _lib.load()
        arr = (_lib.CloudDesc * len(clouds))()
        for i, c in enumerate(clouds):
            arr[i] = _lib.CloudDesc(int(c["n"]), int(c["width"]), int(c["height"]), int(c.get("seed", 0)),
                                    int(c.get("cloud", i)), float(c.get("amplitude", 1e-3)),
                                    int(c.get("color", 0xFFFFFFFF)), int(c.get("background", 0)))
        h = C.c_void_p()
        check(lib.mmr_batch_create(len(clouds), arr, DTYPE_CODE[dtype], camera_slots, budget_bytes,
                                   C.byref(h)), None, batch=True)
        self._lib, self._h = lib, h
        self.clouds = [dict(c) for c in clouds]
        self.dtype = dtype
        self.slots = camera_slots

    def close(self):
        if self._h:
            self._lib.mmr_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        check(status, self._h, batch=True)

    def points(self, i: int) -> torch.Tensor:
        p = C.c_void_p()
        self._check(self._lib.mmr_batch_points(self._h, i, C.byref(p)))
        return device_view(p.value, (int(self.clouds[i]["n"]), 3), _TORCH_VIEW[self.dtype][1])

    def set_camera(self, i: int, slot: int, eye, target, up, fovy_deg, znear, zfar):
        d3 = C.c_double * 3
        self._check(self._lib.mmr_batch_set_camera(self._h, i, slot, d3(*eye), d3(*target), d3(*up), fovy_deg,
                                                   znear, zfar))

    def set_launch(self, threads: int, ctas_per_sm: int, chunk_groups: int):
        self._check(self._lib.mmr_batch_set_launch(self._h, threads, ctas_per_sm, chunk_groups))

    def step_and_render(self, stream=None):
        self._check(self._lib.mmr_batch_step_and_render(self._h, stream_handle(stream)))

    def step_and_render_roundtrip(self, stream=None, pinned: bool = True):
        """One frame through a device -> host -> device copy of all positions (see include/mmr.h)."""
        self._check(self._lib.mmr_batch_step_and_render_roundtrip(self._h, stream_handle(stream), int(pinned)))

    def run_graph(self, frames: int, stream=None):
        self._check(self._lib.mmr_batch_run_graph(self._h, frames, stream_handle(stream)))

    def autotune(self, frames_per_config: int = 3, stream=None):
        t, c, g, ms = C.c_int(), C.c_int(), C.c_int(), C.c_float()
        self._check(self._lib.mmr_batch_autotune(self._h, stream_handle(stream), frames_per_config, C.byref(t),
                                                 C.byref(c), C.byref(g), C.byref(ms)))
        return {"threads": t.value, "ctas_per_sm": c.value, "chunk_groups": g.value, "ms_per_frame": ms.value}

    def check_device(self):
        """Raise MmrError(MMR_ERR_TIMEOUT) if a pixel item gave up its bounded wait."""
        self._check(self._lib.mmr_batch_check_device(self._h))

    def selftest_bounded_wait(self, max_polls: int = 1000, stream=None):
        """Run the pixel items' bounded wait on a count that never reaches zero (see include/mmr.h)."""
        self._check(self._lib.mmr_batch_selftest_bounded_wait(self._h, max_polls, stream_handle(stream)))

    def frame_rgba(self, i: int) -> torch.Tensor:
        r, k = C.c_void_p(), C.c_void_p()
        self._check(self._lib.mmr_batch_frame_ptr(self._h, i, C.byref(r), C.byref(k)))
        c = self.clouds[i]
        return device_view(r.value, (int(c["height"]), int(c["width"])), "<i4")

    def frame_keys(self, i: int) -> torch.Tensor:
        r, k = C.c_void_p(), C.c_void_p()
        self._check(self._lib.mmr_batch_frame_ptr(self._h, i, C.byref(r), C.byref(k)))
        c = self.clouds[i]
        return device_view(k.value, (int(c["height"]), int(c["width"])), "<i8")

    @property
    def frames(self) -> int:
        f = C.c_uint32()
        self._check(self._lib.mmr_batch_frames(self._h, C.byref(f)))
        return f.value

    @property
    def device_bytes(self) -> int:
        b = C.c_uint64()
        self._check(self._lib.mmr_batch_device_bytes(self._h, C.byref(b)))
        return b.value


class Server:
    """Serving engine (mmr_serve_*): a shared cloud plus per-viewer private
    clouds, one frame per active viewer per tick."""

    def __init__(self, shared_n: int, dtype: str = "f32", seed: int = 0, cloud: int = 0, amplitude: float = 5e-4,
                 budget_bytes: int = 0):
        lib = _lib.load()
        h = C.c_void_p()
        check(lib.mmr_serve_create(shared_n, DTYPE_CODE[dtype], seed, cloud, amplitude, budget_bytes, C.byref(h)),
              None, serve=True)
        self._lib, self._h = lib, h
        self.shared_n, self.dtype = shared_n, dtype
        self.viewers = {}

    def close(self):
        if self._h:
            self._lib.mmr_serve_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        check(status, self._h, serve=True)

    def shared_points(self) -> torch.Tensor:
        p = C.c_void_p()
        self._check(self._lib.mmr_serve_shared_points(self._h, C.byref(p)))
        return device_view(p.value, (self.shared_n, 3), _TORCH_VIEW[self.dtype][1])

    def set_shared_color(self, color: int):
        self._check(self._lib.mmr_serve_set_shared_color(self._h, color))

    def add_viewer(self, private_n: int, width: int, height: int, seed: int = 0, cloud: int = 1,
                   amplitude: float = 5e-4, color: int = 0xFFFFFFFF, background: int = 0) -> int:
        """Viewer id; raises MmrError (MMR_ERR_BUDGET) when it does not fit."""
        v = C.c_int()
        self._check(self._lib.mmr_serve_add_viewer(self._h, private_n, width, height, seed, cloud, amplitude,
                                                   color, background, C.byref(v)))
        self.viewers[v.value] = (private_n, width, height)
        return v.value

    def try_add_viewer(self, *args, **kw):
        """As add_viewer, but None instead of an exception when over budget."""
        try:
            return self.add_viewer(*args, **kw)
        except MmrError as e:
            if e.status == -3:
                return None
            raise

    def viewer_points(self, v: int) -> torch.Tensor:
        p = C.c_void_p()
        self._check(self._lib.mmr_serve_viewer_points(self._h, v, C.byref(p)))
        return device_view(p.value, (self.viewers[v][0], 3), _TORCH_VIEW[self.dtype][1])

    def set_camera(self, v: int, eye, target, up, fovy_deg, znear, zfar):
        d3 = C.c_double * 3
        self._check(self._lib.mmr_serve_set_camera(self._h, v, d3(*eye), d3(*target), d3(*up), fovy_deg, znear, zfar))

    def remove_viewer(self, v: int):
        self._check(self._lib.mmr_serve_remove_viewer(self._h, v))
        self.viewers.pop(v, None)

    def tick(self, stream=None, roundtrip: bool = False):
        fn = self._lib.mmr_serve_tick_roundtrip if roundtrip else self._lib.mmr_serve_tick
        self._check(fn(self._h, stream_handle(stream)))

    def frame(self, v: int):
        """(rgba int32[H,W] view, keys int64[H,W] view, frames rendered so far)."""
        r, k, f = C.c_void_p(), C.c_void_p(), C.c_uint32()
        self._check(self._lib.mmr_serve_frame_ptr(self._h, v, C.byref(r), C.byref(k), C.byref(f)))
        _, W, H = self.viewers[v]
        return device_view(r.value, (H, W), "<i4"), device_view(k.value, (H, W), "<i8"), f.value

    def status(self):
        t, a, b = C.c_uint32(), C.c_int(), C.c_uint64()
        self._check(self._lib.mmr_serve_status(self._h, C.byref(t), C.byref(a), C.byref(b)))
        return {"tick": t.value, "active": a.value, "device_bytes": b.value}

    def set_timing(self, enable: bool = True):
        self._check(self._lib.mmr_serve_set_timing(self._h, int(enable)))

    def last_tick_ms(self) -> float:
        ms = C.c_float()
        self._check(self._lib.mmr_serve_last_tick_ms(self._h, C.byref(ms)))
        return ms.value


__all__ = ["Batch", "Context", "MmrError", "Server", "device_view"]
