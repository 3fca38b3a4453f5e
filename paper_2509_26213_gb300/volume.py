"""Python binding of the bricked volume raycaster (argument marshalling only).

Every computation runs in the CUDA library (libvolrc.so) through its C ABI; PyTorch only
provides device memory and the current CUDA stream.  ``RaycastFn`` wraps render +
adjoint as a ``torch.autograd.Function`` (gradients with respect to the transfer function
and the level-0 density).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _capi as C

_TORCH_DT = {"u8": torch.uint8, "u16": torch.uint16 if hasattr(torch, "uint16") else None,
             "f16": torch.float16, "f32": torch.float32}
_NP_DT = {"u8": np.uint8, "u16": np.uint16, "f16": np.float16, "f32": np.float32}


def camera_struct(cam: dict) -> C.vol_camera:
    # (a ctypes float field rounds the value it is given to binary32 to nearest, as numpy does)
    s = C.vol_camera()
    s.eye[:], s.right[:], s.up[:], s.fwd[:] = cam["eye"], cam["right"], cam["up"], cam["fwd"]
    s.tan_half_fov = cam["tan_half_fov"]
    s.aspect = cam["aspect"]
    s.w, s.h = int(cam["w"]), int(cam["h"])
    return s


def params_struct(step=0.5, et=0.99, bg=(0.0, 0.0, 0.0, 0.0), lod_mode=0, lod_bias=0, tile_w=0, tile_h=0,
                  max_passes=0, flags=0, refill=0, ctas_per_sm=0, composite="dvr", grad=False) -> C.vol_params:
    p = C.vol_params()
    p.step, p.et_threshold = step, et
    p.bg[:] = bg
    p.lod_mode, p.lod_bias = int(lod_mode), int(lod_bias)
    p.tile_w, p.tile_h, p.max_passes = int(tile_w), int(tile_h), int(max_passes)
    p.flags = int(flags) | (C.VOL_RENDER_GRAD if grad else 0)
    p.refill, p.ctas_per_sm = int(refill), int(ctas_per_sm)
    p.composite = C.COMPOSITES[composite] if isinstance(composite, str) else int(composite)
    return p


def plan(dims, dtype: str, brick: int, levels: int, cache_bytes: int = 0, layout: str = "quad",
         sparse_pt: bool = False) -> C.vol_layout:
    lay = C.vol_layout()
    d = (ctypes.c_int64 * 3)(*[int(x) for x in dims])
    C.check(C.load().vol_plan(d, C.DTYPES[dtype], int(brick), int(levels), int(cache_bytes),
                              C.LAYOUTS[layout] | (C.VOL_LAYOUT_SPARSE_PT if sparse_pt else 0),
                              ctypes.byref(lay)))
    return lay


def _stream_ptr():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Volume:
    """A bricked multi-resolution volume resident (or cached) on the current CUDA device.

    dims = (Dx, Dy, Dz) level-0 voxels; dtype in {"u8", "u16", "f16", "f32"} (storage);
    brick = brick edge B (power of two); levels = LOD levels; cache_bytes = atlas size
    (0 = room for every brick of every level); layout = "quad" (four-voxel entries, two
    loads per sample, about 4x memory) or "compact" ((B+1)^3 voxels per brick); sparse_pt =
    three-level sparse page table (bricks beyond what a flat table can index; needs
    cache_bytes > 0 and bricks from vol_upload_brick or a provider)."""

    def __init__(self, dims, dtype: str, brick: int, levels: int, cache_bytes: int = 0, layout: str = "quad",
                 sparse_pt: bool = False):
        self.lib = C.load()
        self.dims = tuple(int(x) for x in dims)
        self.dtype = dtype
        self.brick = int(brick)
        self.levels = int(levels)
        h = ctypes.c_void_p()
        d = (ctypes.c_int64 * 3)(*self.dims)
        C.check(self.lib.vol_create(d, C.DTYPES[dtype], self.brick, self.levels, int(cache_bytes),
                                    C.LAYOUTS[layout] | (C.VOL_LAYOUT_SPARSE_PT if sparse_pt else 0), _stream_ptr(),
                                    ctypes.byref(h)))
        self.h = h
        self._provider = None
        lay = C.vol_layout()
        C.check(self.lib.vol_get_layout(self.h, ctypes.byref(lay)), self.h)
        self.layout = lay
        self.level_dims = [tuple(lay.level_dims[l][a] for a in range(3)) for l in range(self.levels)]
        self.level_bricks = [tuple(lay.level_bricks[l][a] for a in range(3)) for l in range(self.levels)]

    def close(self):
        if getattr(self, "h", None):
            self.lib.vol_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        st = torch.cuda.current_stream().cuda_stream
        if st != getattr(self, "_stream", None):
            C.check(self.lib.vol_set_stream(self.h, ctypes.c_void_p(st)), self.h)
            self._stream = st

    # ------------------------------------------------------------ bricks
    def upload_level(self, level: int, src, src_dtype: str | None = None):
        """Dense level array (shape (Dz, Dy, Dx)) from a CUDA tensor or a host numpy array."""
        self._sync_stream()
        if isinstance(src, torch.Tensor):
            src_dtype = src_dtype or {torch.uint8: "u8", torch.float16: "f16", torch.float32: "f32"}.get(src.dtype, "u16")
            src = src.contiguous()
            on_dev = 1 if src.is_cuda else 0
            ptr = src.data_ptr()
        else:
            src = np.ascontiguousarray(src)
            src_dtype = src_dtype or {np.dtype(np.uint8): "u8", np.dtype(np.uint16): "u16",
                                      np.dtype(np.float16): "f16", np.dtype(np.float32): "f32"}[src.dtype]
            on_dev, ptr = 0, src.ctypes.data
        Dx, Dy, Dz = self.level_dims[level]
        if tuple(src.shape) != (Dz, Dy, Dx):
            raise ValueError(f"level {level} needs shape {(Dz, Dy, Dx)}, got {tuple(src.shape)}")
        C.check(self.lib.vol_upload_level(self.h, int(level), ctypes.c_void_p(ptr), C.DTYPES[src_dtype], on_dev), self.h)
        self._keep = src  # host copies are synchronous; device sources must outlive the enqueued copy

    def upload_brick(self, level: int, brick, src: np.ndarray, src_dtype: str):
        self._sync_stream()
        src = np.ascontiguousarray(src)
        b = (ctypes.c_int32 * 3)(*[int(x) for x in brick])
        C.check(self.lib.vol_upload_brick(self.h, int(level), b, ctypes.c_void_p(src.ctypes.data), C.DTYPES[src_dtype], 0),
                self.h)

    def build_lod(self, from_level: int = 0):
        self._sync_stream()
        C.check(self.lib.vol_build_lod(self.h, int(from_level)), self.h)

    def download_brick(self, level: int, brick) -> np.ndarray:
        B1 = self.brick + 1
        out = np.empty((B1, B1, B1), dtype=_NP_DT[self.dtype])
        b = (ctypes.c_int32 * 3)(*[int(x) for x in brick])
        C.check(self.lib.vol_download_brick(self.h, int(level), b, ctypes.c_void_p(out.ctypes.data)), self.h)
        return out

    def evict_all(self):
        C.check(self.lib.vol_evict_all(self.h), self.h)

    def set_provider(self, fn, src_dtype: str):
        """fn(level, (bx, by, bz)) -> numpy array of (B+1)^3 voxels (apron included) of src_dtype."""
        if fn is None:
            self._provider = None
            C.check(self.lib.vol_set_provider(self.h, C.PROVIDER_FN(), None, 0), self.h)
            return
        B1 = self.brick + 1
        npdt = _NP_DT[src_dtype]
        nbytes = B1 ** 3 * np.dtype(npdt).itemsize

        def tramp(_user, level, brick, dst):
            try:
                arr = np.ascontiguousarray(fn(int(level), (brick[0], brick[1], brick[2])), dtype=npdt)
                if arr.nbytes != nbytes:
                    return 1
                ctypes.memmove(dst, arr.ctypes.data, nbytes)
                return 0
            except Exception:  # reported as VOL_ERR_PROVIDER
                return 1

        self._provider = C.PROVIDER_FN(tramp)
        C.check(self.lib.vol_set_provider(self.h, self._provider, None, C.DTYPES[src_dtype]), self.h)

    def set_provider_batch(self, fn_address: int, user, src_dtype: str):
        """Install a native batch provider: fn_address is the address of a C function
        int fn(void* user, int n, const int32_t* reqs, void* dst); `user` (a ctypes object) is
        passed by reference and kept alive by this volume."""
        self._provider = user
        C.check(self.lib.vol_set_provider_batch(self.h, ctypes.c_void_p(fn_address), ctypes.byref(user),
                                                C.DTYPES[src_dtype]), self.h)

    # ------------------------------------------------------------ render
    def render(self, cams, tf: torch.Tensor, params: dict | None = None, out: torch.Tensor | None = None,
               nsamples: bool = False, grad: bool = False, check_incomplete: bool = True):
        """Render views (list of camera dicts) -> float32 tensor [sum(w*h), 4] (views packed): a new
        CUDA tensor, or ``out`` (CUDA, or pinned host memory that the kernel writes directly)."""
        if isinstance(cams, dict):
            cams = [cams]
        params = dict(params or {})
        self._sync_stream()
        arr = (C.vol_camera * len(cams))(*[camera_struct(c) for c in cams])
        npx = sum(int(c["w"]) * int(c["h"]) for c in cams)
        if not (tf.is_cuda and tf.dtype == torch.float32 and tuple(tf.shape) == (256, 4)):
            raise ValueError("tf must be a float32 CUDA tensor of shape (256, 4)")
        tf = tf.contiguous()
        dev = tf.device
        if out is None:
            out = torch.empty((npx, 4), dtype=torch.float32, device=dev)
        elif not (out.dtype == torch.float32 and out.is_contiguous() and out.numel() >= 4 * npx
                  and (out.is_cuda or out.is_pinned())):
            # a pinned host tensor receives the image across the host link, with no copy
            raise ValueError("out must be a contiguous float32 CUDA or pinned host tensor of sum(w*h) x 4")
        ns = torch.empty(npx, dtype=torch.int32, device=dev) if nsamples else None
        p = params_struct(**params, grad=grad)
        rc = self.lib.vol_render(self.h, arr, len(cams), ctypes.c_void_p(tf.data_ptr()), ctypes.byref(p),
                                 ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(ns.data_ptr() if ns is not None else 0))
        self._last = (tf, out, ns)
        if rc != C.VOL_OK and not (rc == C.VOL_ERR_INCOMPLETE and not check_incomplete):
            C.check(rc, self.h)
        self.last_rc = rc
        return (out, ns) if nsamples else out

    def resume(self) -> int:
        self._sync_stream()
        rc = self.lib.vol_render_resume(self.h)
        if rc not in (C.VOL_OK, C.VOL_ERR_INCOMPLETE):
            C.check(rc, self.h)
        return rc

    def poll_requests(self) -> np.ndarray:
        n = ctypes.c_int()
        C.check(self.lib.vol_poll_requests(self.h, None, 0, ctypes.byref(n)), self.h)
        out = np.zeros((max(n.value, 1), 4), dtype=np.int32)
        C.check(self.lib.vol_poll_requests(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value,
                                           ctypes.byref(n)), self.h)
        return out[:n.value]

    def render_backward(self, drgba: torch.Tensor, dtf: torch.Tensor | None = None, dvox: torch.Tensor | None = None):
        self._sync_stream()
        drgba = drgba.contiguous()
        C.check(self.lib.vol_render_backward(self.h, ctypes.c_void_p(drgba.data_ptr()),
                                             ctypes.c_void_p(dtf.data_ptr() if dtf is not None else 0),
                                             ctypes.c_void_p(dvox.data_ptr() if dvox is not None else 0)), self.h)
        self._keep_bwd = drgba

    def trace(self, cam: dict, params: dict, pixels: np.ndarray, max_samples: int):
        pixels = np.ascontiguousarray(pixels, dtype=np.int32)
        n = pixels.shape[0]
        recs = (C.vol_trace_rec * max(1, n * max_samples))()
        counts = np.zeros(n, dtype=np.int32)
        c = camera_struct(cam)
        p = params_struct(**params)
        self._sync_stream()
        C.check(self.lib.vol_trace(self.h, ctypes.byref(c), ctypes.byref(p),
                                   pixels.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n, int(max_samples), recs,
                                   counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), self.h)
        dt = np.dtype([("k", np.int32), ("t_bits", np.uint32), ("level", np.int32), ("i0", np.int32, 3),
                       ("local", np.int32, 3), ("pad", np.int32), ("brick_id", np.int64), ("slot", np.uint32),
                       ("pad2", np.uint32)])
        assert dt.itemsize == ctypes.sizeof(C.vol_trace_rec)
        arr = np.frombuffer(recs, dtype=dt, count=n * max_samples).reshape(n, max_samples).copy()
        return arr, counts

    def stats(self) -> dict:
        s = C.vol_stats()
        C.check(self.lib.vol_get_stats(self.h, ctypes.byref(s)), self.h)
        return {k: getattr(s, k) for k, _ in s._fields_}


class RaycastFn(torch.autograd.Function):
    """rgba = RaycastFn.apply(density, tf, volume, cams, params).

    density: float32 CUDA tensor (Dz, Dy, Dx) of normalised level-0 values, uploaded into
    ``volume`` (an f32 Volume) on every forward, its coarser levels rebuilt when the render
    uses footprint LOD; tf: float32 CUDA (256, 4).  Backward gives dL/d(density) (through the
    box filter's adjoint for samples on coarser levels) and dL/d(tf) through the adjoint
    kernel.  The backward must run before the next render on the same volume."""

    @staticmethod
    def forward(ctx, density, tf, volume, cams, params):
        volume.upload_level(0, density.detach(), "f32")
        if (params or {}).get("lod_mode") and volume.levels > 1:
            volume.build_lod(0)
        out = volume.render(cams, tf.detach(), params, grad=True)
        ctx.volume = volume
        ctx.frame = volume.stats()["frame"]
        ctx.shapes = (density.shape, tf.shape)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        vol = ctx.volume
        if vol.stats()["frame"] != ctx.frame:
            raise RuntimeError("the volume rendered again between forward and backward")
        dvox = torch.zeros(ctx.shapes[0], dtype=torch.float32, device=grad_out.device) if ctx.needs_input_grad[0] else None
        dtf = torch.zeros(ctx.shapes[1], dtype=torch.float32, device=grad_out.device) if ctx.needs_input_grad[1] else None
        vol.render_backward(grad_out.float(), dtf, dvox)
        return dvox, dtf, None, None, None
