"""CPU oracle for the displace + render path (test infrastructure only).

Only tests/, the smoke check and the bench's CPU-baseline leg may import this
package.  The product library never calls it; it shares no code with the CUDA
path.  The arithmetic lives in mmr_oracle.c (plain single-threaded C); this
module only marshals numpy arrays into it.  Each function cites the part of
the paper it follows (Mimir, arXiv 2504.20937).
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = C.CDLL(_build.build())

_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")


def _sig(name, res, *args):
    fn = getattr(_lib, name)
    fn.restype = res
    fn.argtypes = list(args)
    return fn


_sig("orc_philox4x32_10", None, _u32p, _u32p, _u32p)
_sig("orc_philox4x32_10_many", None, _u32p, _u32p, _u32p, C.c_uint64)
_sig("orc_displace_f32", None, _f32p, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_float)
_sig("orc_displace_ids_f32", None, _f32p, _u32p, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
     C.c_float)
_sig("orc_displace_f64", None, _f64p, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_double)
_sig("orc_displace_h16", None, _u16p, C.c_int, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
     C.c_float)
_sig("orc_f32_to_f16_array", None, _f32p, _u16p, C.c_uint64)
_sig("orc_f16_to_f32_array", None, _u16p, _f32p, C.c_uint64)
_sig("orc_f32_to_bf16_array", None, _f32p, _u16p, C.c_uint64)
_sig("orc_bf16_to_f32_array", None, _u16p, _f32p, C.c_uint64)
_sig("orc_camera_f64", None, _f64p, _f64p, _f64p, C.c_double, C.c_double, C.c_double, C.c_double,
     _f64p)
_sig("orc_camera_f32", None, _f64p, _f64p, _f64p, C.c_double, C.c_double, C.c_double, C.c_double,
     _f32p)
_sig("orc_project_many_f32", None, _f32p, _f32p, C.c_uint64, C.c_int, C.c_int, C.c_float, C.c_float,
     _u32p, _f32p, C.c_void_p)
_sig("orc_project_many_f64", None, _f64p, _f64p, C.c_uint64, C.c_double, C.c_double, _f64p, _f64p,
     _i32p)
_sig("orc_splat_f32", None, _f32p, C.c_uint64, _f32p, C.c_int, C.c_int, C.c_float, C.c_float,
     C.c_uint32, _u64p)
_sig("orc_splat_h16", None, _u16p, C.c_int, C.c_uint64, _f32p, C.c_int, C.c_int, C.c_float, C.c_float,
     C.c_uint32, _u64p)
_sig("orc_splat_disc_f32", None, _f32p, C.c_uint64, _f32p, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float,
     C.c_uint32, _u64p)
_sig("orc_nbody_step_f32", None, _f32p, _f32p, _f32p, _f32p, C.c_uint64, C.c_float, C.c_float, C.c_float)
_sig("orc_nbody_step_f32_chunked", None, _f32p, _f32p, _f32p, _f32p, C.c_uint64, C.c_float, C.c_float, C.c_float,
     C.c_uint64)
_sig("orc_nbody_abs_term_sums", None, _f32p, _f32p, C.c_uint64, C.c_float, _f64p)
_sig("orc_nbody_accel_f64", None, _f64p, _f64p, C.c_uint64, C.c_double, C.c_double, _f64p)
_sig("orc_resolve", None, _u64p, C.c_uint64, C.c_void_p, C.c_uint32, C.c_uint32, _u32p)

EMPTY_KEY = np.uint64(0xFFFFFFFFFFFFFFFF)
KIND = {"f16": 1, "bf16": 2}


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one counter (Salmon et al., SC'11)."""
    out = np.zeros(4, np.uint32)
    _lib.orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def philox4x32_10_many(ctr, key):
    """Philox4x32-10 of uint32[n,4] counters with uint32[n,2] keys."""
    ctr = np.ascontiguousarray(ctr, np.uint32)
    key = np.ascontiguousarray(key, np.uint32)
    out = np.empty_like(ctr)
    _lib.orc_philox4x32_10_many(ctr.reshape(-1), key.reshape(-1), out.reshape(-1), ctr.shape[0])
    return out


def displace_f32(pos, seed, cloud, step, a):
    """One Brownian step in FP32, in place on float32[n,3] (Sec. 4.1)."""
    assert pos.dtype == np.float32 and pos.flags.c_contiguous
    _lib.orc_displace_f32(pos.reshape(-1), pos.shape[0], seed, cloud, step, a)


def displace_ids_f32(pos, ids, seed, cloud, step, a):
    """One FP32 step for the listed point ids only (pos[j] belongs to ids[j])."""
    ids = np.ascontiguousarray(ids, np.uint32)
    _lib.orc_displace_ids_f32(pos.reshape(-1), ids, ids.size, seed, cloud, step, a)


def displace_f64(pos, seed, cloud, step, a):
    """The FP64 twin of displace_f32 (same draws, double arithmetic)."""
    assert pos.dtype == np.float64 and pos.flags.c_contiguous
    _lib.orc_displace_f64(pos.reshape(-1), pos.shape[0], seed, cloud, step, a)


def displace_h16(pos_bits, kind, seed, cloud, step, a):
    """One step with binary16 ('f16') or bfloat16 ('bf16') storage, FP32 compute."""
    assert pos_bits.dtype == np.uint16 and pos_bits.flags.c_contiguous
    _lib.orc_displace_h16(pos_bits.reshape(-1), KIND[kind], pos_bits.shape[0], seed, cloud, step, a)


def f32_to_f16(x):
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    _lib.orc_f32_to_f16_array(x.reshape(-1), out.reshape(-1), x.size)
    return out


def f16_to_f32(h):
    h = np.ascontiguousarray(h, np.uint16)
    out = np.empty(h.shape, np.float32)
    _lib.orc_f16_to_f32_array(h.reshape(-1), out.reshape(-1), h.size)
    return out


def f32_to_bf16(x):
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    _lib.orc_f32_to_bf16_array(x.reshape(-1), out.reshape(-1), x.size)
    return out


def bf16_to_f32(h):
    h = np.ascontiguousarray(h, np.uint16)
    out = np.empty(h.shape, np.float32)
    _lib.orc_bf16_to_f32_array(h.reshape(-1), out.reshape(-1), h.size)
    return out


def to_storage(pos_f32, dtype):
    """FP32 positions -> the storage encoding of `dtype` ('f32', 'f16', 'bf16')."""
    if dtype == "f32":
        return np.ascontiguousarray(pos_f32, np.float32).copy()
    return (f32_to_f16 if dtype == "f16" else f32_to_bf16)(pos_f32)


def from_storage(pos_bits, dtype):
    if dtype == "f32":
        return np.asarray(pos_bits, np.float32)
    return (f16_to_f32 if dtype == "f16" else bf16_to_f32)(pos_bits)


def displace(pos, dtype, seed, cloud, step, a):
    """One step in the given storage dtype, in place."""
    if dtype == "f32":
        displace_f32(pos, seed, cloud, step, a)
    else:
        displace_h16(pos, dtype, seed, cloud, step, a)


def camera_f64(eye, target, up, fovy_deg, aspect, znear, zfar):
    """Look-at times perspective in FP64, row-major 4x4."""
    M = np.zeros(16, np.float64)
    _lib.orc_camera_f64(np.asarray(eye, np.float64), np.asarray(target, np.float64),
                        np.asarray(up, np.float64), fovy_deg, aspect, znear, zfar, M)
    return M.reshape(4, 4)


def camera_f32(eye, target, up, fovy_deg, aspect, znear, zfar):
    """camera_f64 rounded once to FP32."""
    M = np.zeros(16, np.float32)
    _lib.orc_camera_f32(np.asarray(eye, np.float64), np.asarray(target, np.float64),
                        np.asarray(up, np.float64), fovy_deg, aspect, znear, zfar, M)
    return M.reshape(4, 4)


def project_f32(M32, pos, W, H, znear, zfar, want_ndc=False):
    """FP32 projection of float32[n,3]; px = 0xffffffff when culled/off-frame."""
    pos = np.ascontiguousarray(pos, np.float32)
    n = pos.shape[0]
    px = np.empty(n, np.uint32)
    w = np.empty(n, np.float32)
    ndc = np.zeros((n, 2), np.float32) if want_ndc else None
    _lib.orc_project_many_f32(np.ascontiguousarray(M32, np.float32).reshape(-1), pos.reshape(-1), n,
                              W, H, znear, zfar, px, w,
                              ndc.ctypes.data if want_ndc else None)
    return (px, w, ndc) if want_ndc else (px, w)


def project_f64(M64, pos, znear, zfar):
    pos = np.ascontiguousarray(pos, np.float64)
    n = pos.shape[0]
    ndc = np.zeros((n, 2), np.float64)
    w = np.zeros(n, np.float64)
    valid = np.zeros(n, np.int32)
    _lib.orc_project_many_f64(np.ascontiguousarray(M64, np.float64).reshape(-1), pos.reshape(-1), n,
                              znear, zfar, ndc, w, valid)
    return ndc, w, valid.astype(bool)


def empty_keys(W, H):
    return np.full(W * H, EMPTY_KEY, np.uint64)


def splat(pos, dtype, M32, W, H, znear, zfar, keybuf, id_base=0):
    """Per-pixel min of bits(w) << 32 | id into keybuf (uint64[W*H])."""
    M = np.ascontiguousarray(M32, np.float32).reshape(-1)
    if dtype == "f32":
        _lib.orc_splat_f32(np.ascontiguousarray(pos, np.float32).reshape(-1), pos.shape[0], M, W, H,
                           znear, zfar, id_base, keybuf)
    else:
        _lib.orc_splat_h16(np.ascontiguousarray(pos, np.uint16).reshape(-1), KIND[dtype], pos.shape[0],
                           M, W, H, znear, zfar, id_base, keybuf)


def splat_disc(pos, M32, W, H, znear, zfar, radius, keybuf, id_base=0):
    """Disc markers of `radius` pixels (FP32 positions): per-pixel min of the
    keys of all points whose disc covers the pixel centre."""
    _lib.orc_splat_disc_f32(np.ascontiguousarray(pos, np.float32).reshape(-1), pos.shape[0],
                            np.ascontiguousarray(M32, np.float32).reshape(-1), W, H, znear, zfar, radius, id_base,
                            keybuf)


def render_disc(pos, M32, W, H, znear, zfar, radius, colors=None, color=0xFFFFFFFF, background=0):
    keys = empty_keys(W, H)
    splat_disc(pos, M32, W, H, znear, zfar, radius, keys)
    return keys, resolve(keys, colors, color, background)


NBODY_CHUNK = 1024


def nbody_step_f32(pos, vel, mass, G, eps2, dt):
    """One all-pairs gravity step (Sec. 4.2.3), the terms summed in order of
    j (the definition); returns the new positions, updates vel in place."""
    out = np.empty_like(pos)
    _lib.orc_nbody_step_f32(np.ascontiguousarray(pos, np.float32).reshape(-1), out.reshape(-1), vel.reshape(-1),
                            np.ascontiguousarray(mass, np.float32), pos.shape[0], G, eps2, dt)
    return out


def nbody_step_f32_chunked(pos, vel, mass, G, eps2, dt, chunk=NBODY_CHUNK):
    """The same step with the terms summed in chunks of `chunk` bodies (each
    chunk in order, then the chunk sums in order): the rounding order of the
    GPU kernel, for its bit-for-bit check."""
    out = np.empty_like(pos)
    _lib.orc_nbody_step_f32_chunked(np.ascontiguousarray(pos, np.float32).reshape(-1), out.reshape(-1),
                                    vel.reshape(-1), np.ascontiguousarray(mass, np.float32), pos.shape[0], G, eps2,
                                    dt, chunk)
    return out


def nbody_abs_term_sums(pos, mass, eps2):
    """float64[n,3]: sum over j of |t_j| per component of body i's terms."""
    out = np.zeros((pos.shape[0], 3), np.float64)
    _lib.orc_nbody_abs_term_sums(np.ascontiguousarray(pos, np.float32).reshape(-1),
                                 np.ascontiguousarray(mass, np.float32), pos.shape[0], eps2, out.reshape(-1))
    return out


def summation_bound_gamma(n):
    """Higham's gamma_{n-1} = (n-1)u / (1 - (n-1)u), u = 2^-24: recursive FP32
    summation of n terms in any order is within gamma_{n-1} sum |t_j| of the
    exact sum (N. J. Higham, Accuracy and Stability of Numerical Algorithms,
    2nd ed., SIAM 2002, Sec. 4.2)."""
    k = max(n - 1, 0) * 2.0**-24
    return k / (1.0 - k)


def nbody_accel_f64(pos, mass, G, eps2):
    acc = np.zeros((pos.shape[0], 3), np.float64)
    _lib.orc_nbody_accel_f64(np.ascontiguousarray(pos, np.float64).reshape(-1), np.ascontiguousarray(mass, np.float64),
                             pos.shape[0], G, eps2, acc.reshape(-1))
    return acc


def resolve(keybuf, colors=None, color=0xFFFFFFFF, background=0):
    """Key buffer -> RGBA8 (uint32 per pixel)."""
    rgba = np.empty(keybuf.size, np.uint32)
    cptr = None
    if colors is not None:
        colors = np.ascontiguousarray(colors, np.uint32)
        cptr = colors.ctypes.data
    _lib.orc_resolve(keybuf, keybuf.size, cptr, color, background, rgba)
    return rgba


def render(pos, dtype, M32, W, H, znear, zfar, colors=None, color=0xFFFFFFFF, background=0):
    """Clear + splat + resolve of one frame; returns (keys, rgba)."""
    keys = empty_keys(W, H)
    splat(pos, dtype, M32, W, H, znear, zfar, keys)
    return keys, resolve(keys, colors, color, background)


def run_frames(pos, dtype, seed, cloud, a, first_step, frames, cam_for_frame, W, H, znear, zfar,
               colors=None, color=0xFFFFFFFF, background=0):
    """`frames` displace+render frames; cam_for_frame(f) -> FP32 matrix.

    Returns the keys and rgba of the last frame; pos is updated in place.
    """
    keys = rgba = None
    for f in range(frames):
        displace(pos, dtype, seed, cloud, first_step + f, a)
        keys, rgba = render(pos, dtype, cam_for_frame(f), W, H, znear, zfar, colors, color, background)
    return keys, rgba


# -- OpenMP CPU baseline (mmr_cpu_omp.c): the oracle's routines over all host
# cores, for bench.py's multi-core CPU figure.  Loaded on first use.
_omp = None


def _omp_lib():
    global _omp
    if _omp is None:
        lib = C.CDLL(_build.build_omp())
        lib.cpu_omp_frame_f32.restype = C.c_int
        lib.cpu_omp_frame_f32.argtypes = [_f32p, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_float,
                                          _f32p, C.c_int, C.c_int, C.c_float, C.c_float, C.c_uint32, C.c_uint32,
                                          _u64p, _u32p, C.c_int]
        lib.cpu_omp_threads.restype = C.c_int
        lib.cpu_omp_threads.argtypes = [C.c_int]
        _omp = lib
    return _omp


def cpu_omp_threads(threads=0):
    """Threads cpu_omp_frame_f32 uses for `threads` (0: OpenMP's default)."""
    return _omp_lib().cpu_omp_threads(threads)


def cpu_omp_frame_f32(pos, seed, cloud, step, a, M32, W, H, znear, zfar, color=0xFFFFFFFF, background=0,
                      threads=0, keys=None, rgba=None):
    """One FP32 frame (displace at `step`, clear, splat, resolve with one
    colour) on `threads` host threads; pos is updated in place.  Returns
    (keys, rgba, threads used); equal to the oracle's frame bit for bit."""
    assert pos.dtype == np.float32 and pos.flags.c_contiguous
    if keys is None:
        keys = np.empty(W * H, np.uint64)
    if rgba is None:
        rgba = np.empty(W * H, np.uint32)
    used = _omp_lib().cpu_omp_frame_f32(pos.reshape(-1), pos.shape[0], seed, cloud, step, np.float32(a),
                                        np.ascontiguousarray(M32, np.float32).reshape(-1), W, H,
                                        np.float32(znear), np.float32(zfar), color, background, keys, rgba,
                                        threads)
    return keys, rgba, used
