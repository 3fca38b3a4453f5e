"""CPU oracle for the bricked multi-resolution raycaster -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does, and fails loudly when its own extension is missing.

``oracle.c`` holds the arithmetic (a decision layer in IEEE binary32 without
contraction, a value layer in float64); this module compiles it with gcc and
marshals numpy arrays.  Every function cites the passage of Drees & Risse,
"Palace" (arXiv 2509.26213) that it follows in ``oracle.c``.

Parity status: every exported function is pinned by tests in
``tests/test_oracle_*.py`` (closed forms, brute force, independent
formulations, finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

U8, U16, F16, F32 = 0, 1, 2, 3
MAX_LEVELS = 16
_NP = {U8: np.uint8, U16: np.uint16, F16: np.uint16, F32: np.float32}
DTYPES = {"u8": U8, "u16": U16, "f16": F16, "f32": F32}

# float32 semantics of the decision layer require no FMA contraction and no
# fast-math; -fexcess-precision=standard keeps every float op in binary32.
CFLAGS = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
          "-fexcess-precision=standard"]


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("fwd", ctypes.c_float * 3),
                ("tan_half_fov", ctypes.c_float), ("aspect", ctypes.c_float),
                ("w", ctypes.c_int32), ("h", ctypes.c_int32)]


class _Params(ctypes.Structure):
    _fields_ = [("step", ctypes.c_float), ("et", ctypes.c_float), ("bg", ctypes.c_float * 4),
                ("lod_mode", ctypes.c_int32), ("lod_bias", ctypes.c_int32), ("level_step", ctypes.c_int32)]


class _Volume(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int32), ("dtype", ctypes.c_int32), ("brick", ctypes.c_int32),
                ("dims", (ctypes.c_int64 * 3) * MAX_LEVELS),
                ("data", ctypes.c_void_p * MAX_LEVELS)]


class TraceRec(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("t_bits", ctypes.c_uint32), ("level", ctypes.c_int32),
                ("i0", ctypes.c_int32 * 3), ("local", ctypes.c_int32 * 3),
                ("brick_id", ctypes.c_int64)]


TRACE_DTYPE = np.dtype([("k", np.int32), ("t_bits", np.uint32), ("level", np.int32),
                        ("i0", np.int32, 3), ("local", np.int32, 3), ("brick_id", np.int64)],
                       align=True)
assert TRACE_DTYPE.itemsize == ctypes.sizeof(TraceRec)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
            lib.orc_level_dims.argtypes = [i64p, ctypes.c_int, vp]
            lib.orc_half_to_double.argtypes = [ctypes.c_uint16]
            lib.orc_half_to_double.restype = ctypes.c_double
            lib.orc_float_to_half.argtypes = [ctypes.c_float]
            lib.orc_float_to_half.restype = ctypes.c_uint16
            lib.orc_u16_to_f16.argtypes = [ctypes.c_int64, vp, vp]
            lib.orc_u8_to_f32.argtypes = [ctypes.c_int64, vp, vp]
            lib.orc_u16_to_f32.argtypes = [ctypes.c_int64, vp, vp]
            lib.orc_downsample.argtypes = [ctypes.c_int, i64p, vp, vp]
            lib.orc_downsample.restype = ctypes.c_int
            lib.orc_trace.argtypes = [ctypes.POINTER(_Volume), ctypes.POINTER(_Camera),
                                      ctypes.POINTER(_Params), ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int64, vp]
            lib.orc_trace.restype = ctypes.c_int64
            lib.orc_render.argtypes = [ctypes.POINTER(_Volume), ctypes.POINTER(_Camera), vp,
                                       ctypes.POINTER(_Params), vp, ctypes.c_int64, ctypes.c_double,
                                       vp, vp, vp, vp, vp, ctypes.c_int]
            lib.orc_render.restype = ctypes.c_int
            lib.orc_render_preview.argtypes = [ctypes.POINTER(_Volume), ctypes.POINTER(_Camera), vp,
                                               ctypes.POINTER(_Params), vp, vp, ctypes.c_int64, ctypes.c_double,
                                               vp, vp, vp, vp, vp, ctypes.c_int]
            lib.orc_render_preview.restype = ctypes.c_int
            lib.orc_render_max.argtypes = [ctypes.POINTER(_Volume), ctypes.POINTER(_Camera), vp,
                                           ctypes.POINTER(_Params), ctypes.c_int, vp, vp, ctypes.c_int64,
                                           ctypes.c_double, vp, vp, vp, vp, ctypes.c_int]
            lib.orc_render_max.restype = ctypes.c_int
            lib.orc_downsample_transpose.argtypes = [i64p, vp, vp]
            lib.orc_render_grad.argtypes = [ctypes.POINTER(_Volume), ctypes.POINTER(_Camera), vp,
                                            ctypes.POINTER(_Params), vp, ctypes.c_int64,
                                            ctypes.c_double, vp, vp, vp, vp, ctypes.c_int]
            lib.orc_render_grad.restype = ctypes.c_int
            lib.orc_ray_info.argtypes = [ctypes.POINTER(_Camera), i64p, ctypes.c_int32,
                                         ctypes.c_int32, vp, ctypes.POINTER(ctypes.c_int32)]
            lib.orc_lod_level.argtypes = [ctypes.POINTER(_Camera), ctypes.c_float, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int]
            lib.orc_lod_level.restype = ctypes.c_int
            lib.orc_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def threads() -> int:
    return _load().orc_threads()


def _dims(D):
    return (ctypes.c_int64 * 3)(*[int(v) for v in D])


def _cam(c: dict) -> _Camera:
    s = _Camera()
    for k in ("eye", "right", "up", "fwd"):
        getattr(s, k)[:] = [float(np.float32(v)) for v in c[k]]
    s.tan_half_fov = float(np.float32(c["tan_half_fov"]))
    s.aspect = float(np.float32(c["aspect"]))
    s.w, s.h = int(c["w"]), int(c["h"])
    return s


def _params(step=0.5, et=0.99, bg=(0, 0, 0, 0), lod_mode=0, lod_bias=0, flags=0, level_step=False,
            **_ignored) -> _Params:
    """``flags`` is read for its level-step bit (16), as the library's render flags carry it."""
    p = _Params()
    p.step, p.et = float(np.float32(step)), float(np.float32(et))
    p.bg[:] = [float(np.float32(b)) for b in bg]
    p.lod_mode, p.lod_bias = int(lod_mode), int(lod_bias)
    p.level_step = int(bool(level_step) or bool(int(flags) & 16))
    return p


def level_dims(D0, nlevels) -> list:
    out = np.zeros((nlevels, 3), dtype=np.int64)
    _load().orc_level_dims(_dims(D0), nlevels, out.ctypes.data)
    return [tuple(int(v) for v in row) for row in out]


def half_to_double(h: int) -> float:
    return _load().orc_half_to_double(int(h))


def float_to_half(f: float) -> int:
    return _load().orc_float_to_half(float(np.float32(f)))


def u16_to_f16(a: np.ndarray) -> np.ndarray:
    """Reduced-precision storage of a uint16 volume: binary16 bits of float32(u / 65535)."""
    a = np.ascontiguousarray(a, dtype=np.uint16)
    out = np.empty_like(a)
    _load().orc_u16_to_f16(a.size, a.ctypes.data, out.ctypes.data)
    return out


def u8_to_f32(a: np.ndarray) -> np.ndarray:
    """Float32 storage of a uint8 volume: u / 255 rounded once to binary32."""
    a = np.ascontiguousarray(a, dtype=np.uint8)
    out = np.empty(a.shape, dtype=np.float32)
    _load().orc_u8_to_f32(a.size, a.ctypes.data, out.ctypes.data)
    return out


def u16_to_f32(a: np.ndarray) -> np.ndarray:
    """Float32 storage of a uint16 volume: u / 65535 rounded once to binary32."""
    a = np.ascontiguousarray(a, dtype=np.uint16)
    out = np.empty(a.shape, dtype=np.float32)
    _load().orc_u16_to_f32(a.size, a.ctypes.data, out.ctypes.data)
    return out


def downsample(a: np.ndarray, dtype: str) -> np.ndarray:
    """One 2x2x2 box-filter level (Sec. III-D).  ``a`` has shape (Dz, Dy, Dx)."""
    code = DTYPES[dtype]
    a = np.ascontiguousarray(a, dtype=_NP[code])
    Dz, Dy, Dx = a.shape
    out = np.empty(((Dz + 1) // 2, (Dy + 1) // 2, (Dx + 1) // 2), dtype=_NP[code])
    rc = _load().orc_downsample(code, _dims((Dx, Dy, Dz)), a.ctypes.data, out.ctypes.data)
    if rc:
        raise RuntimeError("orc_downsample failed")
    return out


def downsample_transpose(g_coarse: np.ndarray, fine_shape) -> np.ndarray:
    """Adjoint of one box-filter level: float64 gradient on the finer level (Dz, Dy, Dx)."""
    g_coarse = np.ascontiguousarray(g_coarse, dtype=np.float64)
    Dz, Dy, Dx = fine_shape
    assert g_coarse.shape == ((Dz + 1) // 2, (Dy + 1) // 2, (Dx + 1) // 2)
    out = np.zeros(fine_shape)
    _load().orc_downsample_transpose(_dims((Dx, Dy, Dz)), g_coarse.ctypes.data, out.ctypes.data)
    return out


def pyramid(a0: np.ndarray, nlevels: int, dtype: str) -> list:
    levels = [np.ascontiguousarray(a0)]
    for _ in range(1, nlevels):
        levels.append(downsample(levels[-1], dtype))
    return levels


class Volume:
    """A dense multi-level volume as the oracle sees it (no bricks, no page table)."""

    def __init__(self, levels: list, dtype: str, brick: int):
        self.levels = [np.ascontiguousarray(l, dtype=_NP[DTYPES[dtype]]) for l in levels]
        if not 1 <= len(self.levels) <= MAX_LEVELS:
            raise ValueError("1..16 levels")
        self.dtype = dtype
        self.brick = int(brick)
        s = _Volume()
        s.nlevels, s.dtype, s.brick = len(self.levels), DTYPES[dtype], self.brick
        for l, arr in enumerate(self.levels):
            Dz, Dy, Dx = arr.shape
            s.dims[l][:] = [Dx, Dy, Dz]
            s.data[l] = arr.ctypes.data
        self._s = s

    @property
    def dims0(self):
        Dz, Dy, Dx = self.levels[0].shape
        return (Dx, Dy, Dz)


class VirtualVolume(Volume):
    """Level dims only, no voxels: for decision-layer traces (``trace``) of volumes too large to
    hold, e.g. the virtual volumes a procedural source serves.  Rendering one is an error."""

    def __init__(self, D0, nlevels: int, dtype: str, brick: int):
        if not 1 <= nlevels <= MAX_LEVELS:
            raise ValueError("1..16 levels")
        self.levels = []
        self.dtype = dtype
        self.brick = int(brick)
        s = _Volume()
        s.nlevels, s.dtype, s.brick = nlevels, DTYPES[dtype], self.brick
        for l, (Dx, Dy, Dz) in enumerate(level_dims(D0, nlevels)):
            s.dims[l][:] = [Dx, Dy, Dz]
            s.data[l] = None
        self._s = s
        self._D0 = tuple(int(v) for v in D0)

    @property
    def dims0(self):
        return self._D0


def ray_info(cam: dict, D0, px: int, py: int):
    out = np.zeros(8, dtype=np.float32)
    hit = ctypes.c_int32()
    _load().orc_ray_info(ctypes.byref(_cam(cam)), _dims(D0), px, py, out.ctypes.data,
                         ctypes.byref(hit))
    return {"o": out[0:3], "d": out[3:6], "t0": out[6], "t1": out[7], "hit": bool(hit.value)}


def lod_level(cam: dict, t: float, bias: int, nlevels: int, mode: int = 1) -> int:
    return _load().orc_lod_level(ctypes.byref(_cam(cam)), float(np.float32(t)), bias, nlevels, mode)


def trace(vol: Volume, cam: dict, params: dict, px: int, py: int, max_samples: int = 1 << 16):
    """Decision-layer records (level, clamped voxel, brick id, local position) per sample."""
    buf = np.zeros(max_samples, dtype=TRACE_DTYPE)
    n = _load().orc_trace(ctypes.byref(vol._s), ctypes.byref(_cam(cam)),
                          ctypes.byref(_params(**params)), px, py, max_samples, buf.ctypes.data)
    return buf[:min(n, max_samples)], int(n)


def render(vol: Volume, cam: dict, tf: np.ndarray, params: dict, pixels=None, amb=1e-5,
           nthreads=0) -> dict:
    """FP64 render of the given pixels ([n,2] int32 px,py; None = whole image, row-major).

    Returns rgba [n,4] float64, n (samples composited), and the alternate result for pixels
    whose early-termination decision lies within ``amb`` of the threshold."""
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    assert tf.shape == (256, 4)
    if pixels is None:
        npix, pp = int(cam["w"]) * int(cam["h"]), None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int32)
        npix, pp = pixels.shape[0], pixels.ctypes.data
    rgba = np.zeros((npix, 4)); n = np.zeros(npix, dtype=np.int32)
    alt = np.zeros((npix, 4)); alt_n = np.zeros(npix, dtype=np.int32)
    flag = np.zeros(npix, dtype=np.int32)
    rc = _load().orc_render(ctypes.byref(vol._s), ctypes.byref(_cam(cam)), tf.ctypes.data,
                            ctypes.byref(_params(**params)), pp, npix, float(amb), rgba.ctypes.data,
                            n.ctypes.data, alt.ctypes.data, alt_n.ctypes.data, flag.ctypes.data,
                            int(nthreads))
    if rc:
        raise RuntimeError("orc_render failed")
    return {"rgba": rgba, "n": n, "alt_rgba": alt, "alt_n": alt_n, "amb": flag.astype(bool)}


def page_table_size(vol: Volume) -> int:
    """Entries of the levels' page tables laid end to end (ceil(D_l / B) bricks per axis)."""
    n = 0
    for arr in vol.levels:
        Dz, Dy, Dx = arr.shape
        n += -(-Dx // vol.brick) * -(-Dy // vol.brick) * -(-Dz // vol.brick)
    return n


def render_preview(vol: Volume, cam: dict, tf: np.ndarray, params: dict, resident: np.ndarray, pixels=None,
                   amb=1e-5, nthreads=0) -> dict:
    """``render`` under a residency map (uint8 per page-table index, levels end to end, brick id
    x fastest): a sample whose brick is absent uses the finest coarser resident level, or
    composites nothing (progressive preview, Sec. III-H)."""
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    resident = np.ascontiguousarray(resident, dtype=np.uint8)
    assert resident.shape == (page_table_size(vol),)
    if pixels is None:
        npix, pp = int(cam["w"]) * int(cam["h"]), None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int32)
        npix, pp = pixels.shape[0], pixels.ctypes.data
    rgba = np.zeros((npix, 4)); n = np.zeros(npix, dtype=np.int32)
    alt = np.zeros((npix, 4)); alt_n = np.zeros(npix, dtype=np.int32)
    flag = np.zeros(npix, dtype=np.int32)
    rc = _load().orc_render_preview(ctypes.byref(vol._s), ctypes.byref(_cam(cam)), tf.ctypes.data,
                                    ctypes.byref(_params(**params)), resident.ctypes.data, pp, npix, float(amb),
                                    rgba.ctypes.data, n.ctypes.data, alt.ctypes.data, alt_n.ctypes.data,
                                    flag.ctypes.data, int(nthreads))
    if rc:
        raise RuntimeError("orc_render_preview failed")
    return {"rgba": rgba, "n": n, "alt_rgba": alt, "alt_n": alt_n, "amb": flag.astype(bool)}


PROJECTIONS = {"mop": 1, "mip": 2}


def render_max(vol: Volume, cam: dict, tf: np.ndarray, params: dict, mode: str, pixels=None, amb=1e-5,
               nthreads=0, resident=None) -> dict:
    """FP64 maximum-opacity ("mop") or maximum-intensity ("mip") projection (Sec. V-A).

    Returns rgba [n,4], n (samples on the ray) and lo/hi [n,4]: per channel the range of the
    outputs over the samples whose opacity lies within ``amb`` of the maximum (MOP).  With a
    residency map, the progressive preview of ``render_preview``."""
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    assert tf.shape == (256, 4)
    res_ptr = None
    if resident is not None:
        resident = np.ascontiguousarray(resident, dtype=np.uint8)
        assert resident.shape == (page_table_size(vol),)
        res_ptr = resident.ctypes.data
    if pixels is None:
        npix, pp = int(cam["w"]) * int(cam["h"]), None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int32)
        npix, pp = pixels.shape[0], pixels.ctypes.data
    rgba = np.zeros((npix, 4)); lo = np.zeros((npix, 4)); hi = np.zeros((npix, 4))
    n = np.zeros(npix, dtype=np.int32)
    rc = _load().orc_render_max(ctypes.byref(vol._s), ctypes.byref(_cam(cam)), tf.ctypes.data,
                                ctypes.byref(_params(**params)), PROJECTIONS[mode], res_ptr, pp, npix, float(amb),
                                rgba.ctypes.data, lo.ctypes.data, hi.ctypes.data, n.ctypes.data,
                                int(nthreads))
    if rc:
        raise RuntimeError("orc_render_max failed")
    return {"rgba": rgba, "lo": lo, "hi": hi, "n": n}


def render_grad(vol: Volume, cam: dict, tf: np.ndarray, params: dict, dI: np.ndarray, pixels=None,
                alt_select=None, amb=1e-5, nthreads=0):
    """FP64 gradients (dL/dtf [256,4], dL/dvoxel level-0 shaped (Dz,Dy,Dx)) for dL/dI [n,4]; with
    footprint LOD the coarser levels' gradients reach level 0 through the box filter's adjoint."""
    tf = np.ascontiguousarray(tf, dtype=np.float32)
    if pixels is None:
        npix, pp = int(cam["w"]) * int(cam["h"]), None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int32)
        npix, pp = pixels.shape[0], pixels.ctypes.data
    dI = np.ascontiguousarray(dI, dtype=np.float64).reshape(npix, 4)
    sel = None
    if alt_select is not None:
        sel = np.ascontiguousarray(alt_select, dtype=np.int32)
    dtf = np.zeros((256, 4)); dvox = np.zeros(vol.levels[0].shape)
    rc = _load().orc_render_grad(ctypes.byref(vol._s), ctypes.byref(_cam(cam)), tf.ctypes.data,
                                 ctypes.byref(_params(**params)), pp, npix, float(amb), dI.ctypes.data,
                                 None if sel is None else sel.ctypes.data, dtf.ctypes.data,
                                 dvox.ctypes.data, int(nthreads))
    if rc:
        raise RuntimeError(f"orc_render_grad failed ({rc})")
    return dtf, dvox
