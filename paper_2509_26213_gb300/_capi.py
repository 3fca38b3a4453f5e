"""ctypes declarations of the C ABI in include/vol.h (argument marshalling only).

Loading fails loudly (ImportError) when the compiled library is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvolrc.so")

VOL_OK = 0
VOL_ERR_INVALID_ARG = -1
VOL_ERR_OOM = -2
VOL_ERR_INCOMPLETE = -3
VOL_ERR_PROVIDER = -4
VOL_ERR_CUDA = -5
VOL_ERR_NO_FORWARD_STATE = -6
VOL_ERR_UNSUPPORTED = -7
VOL_ERR_DEVICE = -8
VOL_ERR_CACHE_FULL = -9
ERROR_NAMES = {v: k for k, v in dict(globals()).items() if k.startswith("VOL_ERR_")}

VOL_U8, VOL_U16, VOL_F16, VOL_F32 = 0, 1, 2, 3
DTYPES = {"u8": VOL_U8, "u16": VOL_U16, "f16": VOL_F16, "f32": VOL_F32}
MAX_LEVELS = 16
VOL_RENDER_GRAD = 1
VOL_RENDER_SKIP_EMPTY = 2
VOL_RENDER_SERIAL_LOADS = 4
VOL_RENDER_PREVIEW = 8
VOL_RENDER_LEVEL_STEP = 16
VOL_RENDER_NO_PREFETCH = 32
VOL_RENDER_CKPT_ALL = 64
VOL_RENDER_GRAD_RECOMPUTE = 128
VOL_COMPOSITE_DVR, VOL_COMPOSITE_MOP, VOL_COMPOSITE_MIP = 0, 1, 2
COMPOSITES = {"dvr": VOL_COMPOSITE_DVR, "mop": VOL_COMPOSITE_MOP, "mip": VOL_COMPOSITE_MIP}
VOL_LAYOUT_COMPACT = 1
LAYOUTS = {"quad": 0, "compact": VOL_LAYOUT_COMPACT}
VOL_LAYOUT_SPARSE_PT = 2

# every entry point include/vol.h declares
EXPORTS = ["vol_plan", "vol_create", "vol_destroy", "vol_last_error", "vol_set_stream", "vol_get_layout",
           "vol_get_stats", "vol_upload_level", "vol_upload_brick", "vol_build_lod", "vol_download_brick",
           "vol_evict_all", "vol_set_provider", "vol_render", "vol_render_resume", "vol_poll_requests",
           "vol_render_backward", "vol_trace", "vol_render_noalloc", "vol_set_provider_batch"]
VOL_NOALLOC_SCRATCH_BYTES = 8192
VOL_NOALLOC_MAX_VIEWS = 64


class vol_camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("right", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fwd", ctypes.c_float * 3), ("tan_half_fov", ctypes.c_float), ("aspect", ctypes.c_float),
                ("w", ctypes.c_int32), ("h", ctypes.c_int32)]


class vol_params(ctypes.Structure):
    _fields_ = [("step", ctypes.c_float), ("et_threshold", ctypes.c_float), ("bg", ctypes.c_float * 4),
                ("lod_mode", ctypes.c_int32), ("lod_bias", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("max_passes", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("refill", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("composite", ctypes.c_int32)]


class vol_layout(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int64 * 3), ("dtype", ctypes.c_int32), ("brick", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("bytes_per_voxel", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("entry_voxels", ctypes.c_int32),
                ("level_dims", (ctypes.c_int64 * 3) * MAX_LEVELS),
                ("level_bricks", (ctypes.c_int64 * 3) * MAX_LEVELS),
                ("level_pt_offset", ctypes.c_int64 * MAX_LEVELS), ("total_bricks", ctypes.c_int64),
                ("slot_bytes", ctypes.c_int64), ("nslots", ctypes.c_int64), ("atlas_bytes", ctypes.c_int64),
                ("sparse_pt", ctypes.c_int64), ("pt_top_entries", ctypes.c_int64)]


class vol_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("passes", "rays", "suspended", "requests", "request_overflow",
                                               "bricks_loaded", "bytes_loaded", "evicted", "resident", "frame",
                                               "device_error", "touched", "load_wait_us", "launches",
                                               "preview_samples", "allocations",
                                               "skipped_samples")]


class vol_trace_rec(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("t_bits", ctypes.c_uint32), ("level", ctypes.c_int32),
                ("i0", ctypes.c_int32 * 3), ("local", ctypes.c_int32 * 3), ("pad", ctypes.c_int32),
                ("brick_id", ctypes.c_int64), ("slot", ctypes.c_uint32), ("pad2", ctypes.c_uint32)]


PROVIDER_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                               ctypes.c_void_p)

_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2509_26213_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    sig = {
        "vol_plan": (i32, [i64p, i32, i32, i32, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(vol_layout)]),
        "vol_create": (i32, [i64p, i32, i32, i32, ctypes.c_uint64, ctypes.c_uint32, vp, ctypes.POINTER(vp)]),
        "vol_destroy": (None, [vp]),
        "vol_last_error": (ctypes.c_char_p, [vp]),
        "vol_set_stream": (i32, [vp, vp]),
        "vol_get_layout": (i32, [vp, ctypes.POINTER(vol_layout)]),
        "vol_get_stats": (i32, [vp, ctypes.POINTER(vol_stats)]),
        "vol_upload_level": (i32, [vp, i32, vp, i32, i32]),
        "vol_upload_brick": (i32, [vp, i32, i32p, vp, i32, i32]),
        "vol_build_lod": (i32, [vp, i32]),
        "vol_download_brick": (i32, [vp, i32, i32p, vp]),
        "vol_evict_all": (i32, [vp]),
        "vol_set_provider": (i32, [vp, PROVIDER_FN, vp, i32]),
        "vol_render": (i32, [vp, ctypes.POINTER(vol_camera), i32, vp, ctypes.POINTER(vol_params), vp, vp]),
        "vol_render_resume": (i32, [vp]),
        "vol_poll_requests": (i32, [vp, i32p, i32, ctypes.POINTER(ctypes.c_int)]),
        "vol_render_backward": (i32, [vp, vp, vp, vp]),
        "vol_trace": (i32, [vp, ctypes.POINTER(vol_camera), ctypes.POINTER(vol_params), i32p, i32, i32,
                            ctypes.POINTER(vol_trace_rec), i32p]),
        "vol_render_noalloc": (i32, [vp, ctypes.POINTER(vol_camera), i32, vp, ctypes.POINTER(vol_params), vp, vp]),
        "vol_set_provider_batch": (i32, [vp, vp, vp, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class VolError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(rc: int, handle=None):
    if rc != VOL_OK:
        msg = load().vol_last_error(handle)
        raise VolError(rc, msg.decode() if msg else "")
    return rc
