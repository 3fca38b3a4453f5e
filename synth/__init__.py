"""Seeded synthetic inputs: volumes, orbit / fly-through cameras, transfer functions.

This module makes inputs only; it holds none of the rendering arithmetic.  The
CUDA path and the CPU oracle both consume what it produces and never import
each other.  Volumes are generated by ``synth.c`` (compiled on first use with
gcc + OpenMP); cameras and transfer functions are small and built here with
numpy in float64, then rounded once to float32 -- the form both consumers take.

Workload recipes (the paper's datasets -- Sec. IV-A, Table I -- are not
available, so these stand in for them; each is seeded and reproducible):

* ``blobs_u8``   sum of isotropic Gaussian blobs plus U[0,16) noise, clamped to 255
* ``blobs_f32``  the same shape as a float32 density in [0, 1]
* ``noise_spheres_u16``  5-octave fractal value noise with embedded spheres
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into _synth.so (gcc, OpenMP, no ISA-specific flags)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.synth_blobs.argtypes = [ctypes.c_int, i64p, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_int]
            lib.synth_blobs.restype = ctypes.c_int
            lib.synth_noise_spheres_region.argtypes = [
                i64p, ctypes.c_int, i64p, i64p, i64p, ctypes.c_uint64, ctypes.c_int,
                ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_int]
            lib.synth_noise_spheres_region.restype = ctypes.c_int
            lib.synth_draw01.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_draw01.restype = ctypes.c_double
            _lib = lib
    return _lib


def _dims(D):
    return (ctypes.c_int64 * 3)(*[int(v) for v in D])


def _threads(nthreads):
    if nthreads:
        return int(nthreads)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def draw01(seed: int, stream: int, ctr: int) -> float:
    return _load().synth_draw01(seed, stream, ctr)


def blobs(D, seed, *, dtype="u8", nblobs=8, sigma=(6.0, 20.0), amp=(60.0, 200.0),
          noise=16.0, vmax=None, nthreads=0) -> np.ndarray:
    """Gaussian blobs + uniform noise.  Returns an array of shape (Dz, Dy, Dx)."""
    Dx, Dy, Dz = (int(v) for v in D)
    if dtype == "u8":
        code, npdt, vmax = 0, np.uint8, 255.0 if vmax is None else vmax
    elif dtype == "f32":
        code, npdt, vmax = 3, np.float32, 1.0 if vmax is None else vmax
    else:
        raise ValueError(dtype)
    out = np.empty((Dz, Dy, Dx), dtype=npdt)
    rc = _load().synth_blobs(code, _dims(D), seed, nblobs, sigma[0], sigma[1], amp[0], amp[1],
                             noise, vmax, out.ctypes.data, _threads(nthreads))
    if rc != 0:
        raise RuntimeError(f"synth_blobs failed: {rc}")
    return out


def noise_spheres_region(D0, level, Dl, origin, extent, seed, *, octaves=5, period0=128.0,
                         nspheres=200, radius=(4.0, 60.0), value=(0.3, 1.0),
                         nthreads=0, out=None) -> np.ndarray:
    """Fractal value noise + spheres over a (clamped) region of level ``level``.

    Returns uint16 of shape (ez, ey, ex)."""
    ex, ey, ez = (int(v) for v in extent)
    if out is None:
        out = np.empty((ez, ey, ex), dtype=np.uint16)
    assert out.dtype == np.uint16 and out.shape == (ez, ey, ex) and out.flags.c_contiguous
    rc = _load().synth_noise_spheres_region(_dims(D0), level, _dims(Dl), _dims(origin), _dims(extent),
                                            seed, octaves, period0, nspheres, radius[0], radius[1],
                                            value[0], value[1], out.ctypes.data, _threads(nthreads))
    if rc != 0:
        raise RuntimeError(f"synth_noise_spheres_region failed: {rc}")
    return out


def noise_spheres(D, seed, **kw) -> np.ndarray:
    """Level-0 noise + spheres volume, shape (Dz, Dy, Dx), uint16."""
    return noise_spheres_region(D, 0, D, (0, 0, 0), D, seed, **kw)


# ---------------------------------------------------------------- cameras

def _normalize(v):
    return v / math.sqrt(float(np.dot(v, v)))


def look_at(eye, target, w, h, fov_deg=45.0, world_up=(0.0, 0.0, 1.0)) -> dict:
    """Pinhole camera looking from ``eye`` at ``target``; vectors computed in float64, then
    rounded once to float32 (the form both consumers take)."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = _normalize(np.asarray(target, dtype=np.float64) - eye)
    right = np.cross(fwd, np.asarray(world_up, dtype=np.float64))
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right = _normalize(right)
    up = np.cross(right, fwd)
    return {
        "eye": np.float32(eye), "right": np.float32(right), "up": np.float32(up),
        "fwd": np.float32(fwd),
        "tan_half_fov": np.float32(math.tan(math.radians(fov_deg) / 2.0)),
        "aspect": np.float32(float(w) / float(h)), "w": int(w), "h": int(h),
    }


def orbit_camera(D, w, h, theta, phi, fov_deg=45.0, fit=1.1) -> dict:
    """Camera on a sphere around the volume centre, far enough that the bounding sphere fits
    the vertical field of view times ``fit``.  theta: azimuth, phi: elevation (radians)."""
    D = np.asarray(D, dtype=np.float64)
    centre = D / 2.0
    radius = float(np.linalg.norm(D)) / 2.0
    dist = radius / math.sin(math.radians(fov_deg) / 2.0) * fit
    eye = centre + dist * np.array([math.cos(phi) * math.cos(theta),
                                    math.cos(phi) * math.sin(theta), math.sin(phi)])
    return look_at(eye, centre, w, h, fov_deg)


def seeded_orbit(D, w, h, seed, view=0, fov_deg=45.0, fit=1.1) -> dict:
    """Orbit camera at a seeded angle: theta ~ U[0, 2pi), phi ~ U[-30deg, 30deg]."""
    theta = 2.0 * math.pi * draw01(seed, 100, 2 * view)
    phi = math.radians(-30.0 + 60.0 * draw01(seed, 100, 2 * view + 1))
    return orbit_camera(D, w, h, theta, phi, fov_deg, fit)


def batched_views(D, nviews, seed, sizes=(256, 512, 768, 1024), fov_deg=45.0) -> list:
    """Views for the batched workload: square side drawn from ``sizes`` per view, seeded poses."""
    cams = []
    for v in range(nviews):
        s = sizes[int(draw01(seed, 101, v) * len(sizes)) % len(sizes)]
        cams.append(seeded_orbit(D, s, s, seed, view=v, fov_deg=fov_deg))
    return cams


def flythrough(D, w, h, nframes, seed, fov_deg=45.0) -> list:
    """Seeded camera path through the inside of a volume: a slow circle at a seeded height,
    looking ahead and slightly inward."""
    D = np.asarray(D, dtype=np.float64)
    c = D / 2.0
    rad = 0.30 * float(min(D[0], D[1]))
    zc = D[2] * (0.35 + 0.3 * draw01(seed, 102, 0))
    a0 = 2.0 * math.pi * draw01(seed, 102, 1)
    cams = []
    for f in range(nframes):
        a = a0 + 0.02 * f
        eye = np.array([c[0] + rad * math.cos(a), c[1] + rad * math.sin(a), zc])
        ahead = np.array([c[0] + 0.8 * rad * math.cos(a + 0.4), c[1] + 0.8 * rad * math.sin(a + 0.4),
                          zc - 0.05 * D[2]])
        cams.append(look_at(eye, ahead, w, h, fov_deg))
    return cams


# ------------------------------------------------------- transfer functions

def tf_ramp(alpha_start=0.1, alpha_max=0.08, n=256) -> np.ndarray:
    """Piecewise-linear RGBA ramp: alpha 0 below ``alpha_start``, rising linearly to
    ``alpha_max`` at 1.0; colour a warm ramp.  float32 [n][4]."""
    x = np.arange(n, dtype=np.float64) / (n - 1)
    a = np.where(x < alpha_start, 0.0, alpha_max * (x - alpha_start) / (1.0 - alpha_start))
    rgb = np.stack([np.clip(0.2 + 0.8 * x, 0, 1), np.clip(x * x, 0, 1), np.clip(1.0 - x, 0, 1)], axis=1)
    return np.concatenate([rgb, a[:, None]], axis=1).astype(np.float32)


def tf_peaks(seed, npeaks=3, n=256) -> np.ndarray:
    """Seeded opacity peaks: triangular, centre U[0.1,0.9], half-width U[0.02,0.1],
    height U[0.05,0.5]; alpha = max over peaks; colour of the highest-contributing peak."""
    x = np.arange(n, dtype=np.float64) / (n - 1)
    alpha = np.zeros(n)
    rgb = np.zeros((n, 3))
    for p in range(npeaks):
        c = 0.1 + 0.8 * draw01(seed, 103, 8 * p)
        hw = 0.02 + 0.08 * draw01(seed, 103, 8 * p + 1)
        ht = 0.05 + 0.45 * draw01(seed, 103, 8 * p + 2)
        col = np.array([draw01(seed, 103, 8 * p + 3 + i) for i in range(3)])
        a = ht * np.clip(1.0 - np.abs(x - c) / hw, 0.0, None)
        take = a > alpha
        alpha = np.where(take, a, alpha)
        rgb[take] = col
    return np.concatenate([rgb, alpha[:, None]], axis=1).astype(np.float32)


def tf_perturbed(tf, seed, rel_sigma=0.05) -> np.ndarray:
    """Seeded perturbation of a transfer function: Gaussian noise with sigma = rel_sigma * max,
    clamped at 0 (the target of the differentiable workload).  Box-Muller on the counter draws."""
    tf = np.asarray(tf, dtype=np.float64)
    n = tf.size
    u1 = np.array([draw01(seed, 104, 2 * i) for i in range(n)])
    u2 = np.array([draw01(seed, 104, 2 * i + 1) for i in range(n)])
    g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    out = tf + rel_sigma * float(np.max(tf)) * g.reshape(tf.shape)
    return np.clip(out, 0.0, None).astype(np.float32)


def pixel_subset(w, h, n, seed) -> np.ndarray:
    """n distinct seeded pixels of a w x h image as int32 (px, py) pairs, shape [n, 2]."""
    n = min(int(n), w * h)
    keys = np.array([draw01(seed, 105, i) for i in range(w * h)]) if w * h <= 1 << 16 else None
    if keys is not None:
        idx = np.argsort(keys, kind="stable")[:n]
    else:
        rng = np.random.Generator(np.random.PCG64(seed))
        idx = rng.choice(w * h, size=n, replace=False)
    idx = np.sort(idx)
    return np.stack([idx % w, idx // w], axis=1).astype(np.int32)


# --------------------------------------------------- on-demand brick source

class BrickSource(ctypes.Structure):
    """Parameters of a procedural noise + spheres volume served brick by brick (synth.c)."""
    _fields_ = [("D0", ctypes.c_int64 * 3), ("brick", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("out8", ctypes.c_int32), ("nthreads", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("octaves", ctypes.c_int32), ("nspheres", ctypes.c_int32), ("period0", ctypes.c_double),
                ("r_lo", ctypes.c_double), ("r_hi", ctypes.c_double), ("v_lo", ctypes.c_double),
                ("v_hi", ctypes.c_double)]


def brick_source(D0, brick, levels, seed, *, dtype="u8", octaves=5, period0=128.0, nspheres=200,
                 radius=(4.0, 60.0), value=(0.3, 1.0), nthreads=0) -> BrickSource:
    s = BrickSource()
    s.D0[:] = [int(v) for v in D0]
    s.brick, s.levels, s.out8 = int(brick), int(levels), 1 if dtype == "u8" else 0
    s.nthreads = _threads(nthreads)
    s.seed, s.octaves, s.nspheres = int(seed), int(octaves), int(nspheres)
    s.period0, s.r_lo, s.r_hi, s.v_lo, s.v_hi = float(period0), radius[0], radius[1], value[0], value[1]
    return s


def brick_provider_address() -> int:
    """Address of synth_brick_provider(void* user, int n, const int32_t* reqs, void* dst): fills n
    bricks of (B+1)^3 voxels (apron included) for requests [level, bx, by, bz]."""
    lib = _load()
    return ctypes.cast(lib.synth_brick_provider, ctypes.c_void_p).value


def provide_bricks(src: BrickSource, reqs) -> np.ndarray:
    """Host call of the same provider: [n, B+1, B+1, B+1] voxels for requests [n, 4]."""
    lib = _load()
    reqs = np.ascontiguousarray(reqs, dtype=np.int32).reshape(-1, 4)
    B1 = src.brick + 1
    out = np.empty((reqs.shape[0], B1, B1, B1), dtype=np.uint8 if src.out8 else np.uint16)
    lib.synth_brick_provider.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.synth_brick_provider.restype = ctypes.c_int
    if lib.synth_brick_provider(ctypes.byref(src), reqs.shape[0], reqs.ctypes.data, out.ctypes.data) != 0:
        raise RuntimeError("synth_brick_provider failed")
    return out


def noise_spheres_level(D0, level, seed, *, dtype="u8", **kw) -> np.ndarray:
    """A whole level of the procedural volume (for small sizes), shape (Dz, Dy, Dx)."""
    Dl = [int(v) for v in D0]
    for _ in range(level):
        Dl = [(v + 1) // 2 for v in Dl]
    if dtype == "u16":
        return noise_spheres_region(D0, level, Dl, (0, 0, 0), Dl, seed, **kw)
    lib = _load()
    lib.synth_noise_spheres_region8.argtypes = lib.synth_noise_spheres_region.argtypes
    lib.synth_noise_spheres_region8.restype = ctypes.c_int
    nthreads = kw.pop("nthreads", 0)
    octaves, period0 = kw.pop("octaves", 5), kw.pop("period0", 128.0)
    nspheres, radius, value = kw.pop("nspheres", 200), kw.pop("radius", (4.0, 60.0)), kw.pop("value", (0.3, 1.0))
    out = np.empty((Dl[2], Dl[1], Dl[0]), dtype=np.uint8)
    rc = lib.synth_noise_spheres_region8(_dims(D0), level, _dims(Dl), _dims((0, 0, 0)), _dims(Dl), seed, octaves,
                                         period0, nspheres, radius[0], radius[1], value[0], value[1],
                                         out.ctypes.data, _threads(nthreads))
    if rc != 0:
        raise RuntimeError("synth_noise_spheres_region8 failed")
    return out
