"""Shared test helpers: workload recipes and oracle/GPU comparison rules."""
from __future__ import annotations

import numpy as np

import synth

# max-abs per-channel tolerances (float32 arithmetic path; reduced-precision storage path)
TOL_FP32 = 1e-4
TOL_REDUCED = 2e-3
# early-termination margin within which float32 and float64 may decide differently
AMB = 1e-5


def store_levels(orc, raw0: np.ndarray, src_dtype: str, store_dtype: str, nlevels: int) -> list:
    """The oracle's own view of the stored pyramid: transcode level 0 as the storage
    definition says, then box-filter level by level."""
    if src_dtype == store_dtype:
        l0 = raw0
    elif (src_dtype, store_dtype) == ("u16", "f16"):
        l0 = orc.u16_to_f16(raw0)
    elif (src_dtype, store_dtype) == ("u8", "f32"):
        l0 = orc.u8_to_f32(raw0)
    elif (src_dtype, store_dtype) == ("u16", "f32"):
        l0 = orc.u16_to_f32(raw0)
    else:
        raise ValueError((src_dtype, store_dtype))
    return orc.pyramid(l0, nlevels, store_dtype)


def compare(gpu: np.ndarray, ref: dict, tol: float, idx=None):
    """GPU rgba [n,4] vs oracle result; a pixel passes when it matches the primary result, or
    the alternate one where early termination was within rounding of the threshold.
    Returns (max error over the accepted candidate, pixels that failed, pixels using the alternate)."""
    rp, ra, amb = ref["rgba"], ref["alt_rgba"], ref["amb"]
    if idx is not None:
        rp, ra, amb = rp[idx], ra[idx], amb[idx]
    gpu = gpu.astype(np.float64)
    ep = np.abs(gpu - rp).max(axis=1)
    ea = np.abs(gpu - ra).max(axis=1)
    use_alt = amb & (ep > tol) & (ea <= tol)
    err = np.where(use_alt, ea, ep)
    bad = np.flatnonzero(err > tol)
    return float(err.max(initial=0.0)), bad, use_alt


def compare_projection(gpu: np.ndarray, ref: dict, tol: float):
    """MOP/MIP: alpha within tol of the oracle's; each colour within tol of the range the oracle
    gives over the samples whose opacity ties the maximum within its ambiguity bound.
    Returns (max error, pixels that failed, pixels with a non-degenerate range)."""
    gpu = gpu.astype(np.float64)
    ea = np.abs(gpu[:, 3] - ref["rgba"][:, 3])
    below = np.clip(ref["lo"][:, :3] - gpu[:, :3], 0, None).max(axis=1)
    above = np.clip(gpu[:, :3] - ref["hi"][:, :3], 0, None).max(axis=1)
    err = np.maximum(ea, np.maximum(below, above))
    strict = np.all(ref["lo"] == ref["hi"], axis=1)
    return float(err.max(initial=0.0)), np.flatnonzero(err > tol), int((~strict).sum())


def c1_inputs(seed=1):
    """Plain FP32 single view: 128^3 u8 blobs + noise, 32^3 bricks, 2 levels, 256x256 orbit view,
    45 deg FOV, step 0.5, piecewise-linear ramp TF, early termination at 0.99."""
    D = (128, 128, 128)
    raw = synth.blobs(D, seed, nblobs=8, sigma=(6.0, 20.0), amp=(60.0, 200.0), noise=16.0)
    cam = synth.seeded_orbit(D, 256, 256, seed)
    tf = synth.tf_ramp(alpha_start=0.1, alpha_max=0.08)
    params = {"step": 0.5, "et": 0.99, "bg": (0.0, 0.0, 0.0, 0.0)}
    return D, raw, cam, tf, params
