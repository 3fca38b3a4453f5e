"""The five seeded workloads (inputs only: volumes, cameras, transfer functions, parameters).

They stand in for the paper's raycasting datasets (Sec. IV-A, Table I: a 4352^3 float32
Mandelbulb and a 1634x12723x9070 uint16 kidney scan, both in 64^3 bricks, not available
here) and its procedural on-demand volume (Sec. V-C).

c1  plain FP32 single view: 128^3 u8 blobs + noise, 32^3 bricks, 2 levels, 256^2
c2  reduced precision: 1024^3 u16 fractal noise + 200 spheres, 64^3 bricks, 5 levels,
    footprint LOD, 1920x1080, stored as u16 and as f16
c3  batched: 64 views of side {256,512,768,1024}, 2048^3 u8 blobs + noise, 32^3 bricks,
    6 levels, footprint LOD
c4  differentiable: 256^3 f32 blobs, 16 views at 512^2, forward + adjoint
c5  out of core: 4096^3 u8 procedural on demand, 64^3 bricks, 7 levels, 16 GiB cache,
    30-frame fly-through at 1920x1080
"""
from __future__ import annotations

import numpy as np

from . import (batched_views, blobs, flythrough, noise_spheres, seeded_orbit, tf_peaks, tf_ramp)


def c1(seed: int = 1) -> dict:
    D = (128, 128, 128)
    return {
        "key": "c1", "D": D, "brick": 32, "levels": 2, "src": "u8", "store": "u8",
        "make": lambda: blobs(D, seed, nblobs=8, sigma=(6.0, 20.0), amp=(60.0, 200.0), noise=16.0),
        "cams": [seeded_orbit(D, 256, 256, seed)],
        "tf": tf_ramp(alpha_start=0.1, alpha_max=0.08),
        "params": {"step": 0.5, "et": 0.99, "lod_mode": 0},
        "name": "plain single view, 128^3 u8 blobs+noise, 32^3 bricks, 2 levels, 256x256",
    }


def c2(seed: int = 2) -> dict:
    D = (1024, 1024, 1024)
    return {
        "key": "c2", "D": D, "brick": 64, "levels": 5, "src": "u16", "store": "u16",
        "make": lambda: noise_spheres(D, seed, octaves=5, period0=128.0, nspheres=200, radius=(4.0, 60.0),
                                      value=(0.3, 1.0)),
        "cams": [seeded_orbit(D, 1920, 1080, seed)],
        "tf": tf_peaks(seed),
        "params": {"step": 0.5, "et": 0.99, "lod_mode": 1, "lod_bias": 0},
        "name": "reduced-precision single view, 1024^3 u16 noise+spheres, 64^3 bricks, 5 levels, 1920x1080",
    }


def c3(seed: int = 3, brick: int = 32) -> dict:
    D = (2048, 2048, 2048)
    return {
        "key": "c3", "D": D, "brick": brick, "levels": 6, "src": "u8", "store": "u8",
        # blobs scaled with the volume (sigma 3%..10% of the edge) so the frame is not empty
        "make": lambda: blobs(D, seed, nblobs=32, sigma=(0.03 * D[0], 0.10 * D[0]), amp=(60.0, 200.0), noise=16.0),
        "cams": batched_views(D, 64, seed),
        "tf": tf_ramp(alpha_start=0.1, alpha_max=0.08),
        "params": {"step": 0.5, "et": 0.99, "lod_mode": 1, "lod_bias": 0},
        "name": "batched 64 views {256..1024}^2, 2048^3 u8 blobs+noise, 32^3 bricks, 6 levels",
    }


def c4(seed: int = 4) -> dict:
    D = (256, 256, 256)
    return {
        "key": "c4", "D": D, "brick": 32, "levels": 1, "src": "f32", "store": "f32",
        "make": lambda: blobs(D, seed, dtype="f32", nblobs=8, sigma=(12.0, 40.0), amp=(0.2, 1.0), noise=0.02, vmax=1.0),
        "cams": [seeded_orbit(D, 512, 512, seed, view=v) for v in range(16)],
        "tf": tf_ramp(alpha_start=0.05, alpha_max=0.1),
        "params": {"step": 0.5, "et": 0.99, "lod_mode": 0},
        "name": "differentiable, 256^3 f32 blobs, 16 views 512x512, forward + adjoint",
    }


def c5(seed: int = 5) -> dict:
    D = (4096, 4096, 4096)
    return {
        "key": "c5", "D": D, "brick": 64, "levels": 7, "src": "u16", "store": "u8",
        "cache_bytes": 16 << 30,
        "cams": flythrough(D, 1920, 1080, 30, seed),
        "tf": tf_peaks(seed),
        "params": {"step": 0.5, "et": 0.99, "lod_mode": 1, "lod_bias": 0},
        "noise": {"octaves": 5, "period0": 512.0, "nspheres": 1000, "radius": (8.0, 120.0), "value": (0.3, 1.0)},
        "name": "out-of-core 4096^3 procedural, 64^3 bricks, 7 levels, 16 GiB cache, 30-frame fly-through",
    }


def c2s(seed: int = 2) -> dict:
    """c2 at 512^3 (same generator scaled by 1/2, same image and TF): the case profiled in detail,
    a few GB on the device at most."""
    D = (512, 512, 512)
    return {
        "key": "c2s", "D": D, "brick": 64, "levels": 4, "src": "u16", "store": "u16",
        "make": lambda: noise_spheres(D, seed, octaves=5, period0=64.0, nspheres=200, radius=(2.0, 30.0),
                                      value=(0.3, 1.0)),
        "cams": [seeded_orbit(D, 1920, 1080, seed)],
        "tf": tf_peaks(seed),
        "params": {"step": 0.5, "et": 0.99, "lod_mode": 1, "lod_bias": 0},
        "name": "reduced-precision single view, 512^3 u16 noise+spheres, 64^3 bricks, 4 levels, 1920x1080",
    }


def c4s(seed: int = 4) -> dict:
    """c4 with 2 of its 16 views (same volume, TF and target): the case the adjoint is profiled in
    detail on, a few GB on the device at most."""
    wl = c4(seed)
    wl.update(key="c4s", cams=wl["cams"][:2],
              name="differentiable, 256^3 f32 blobs, 2 views 512x512, forward + adjoint")
    return wl
