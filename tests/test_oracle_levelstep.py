"""Pins for the oracle's level-scaled sampling (flag bit 16): a sample on level l stands for 2^l
reference steps -- the next sample is dt * 2^l further, and its opacity is corrected to
1 - (1 - a)^(2^l).

* constant density with every sample forced onto level 2 (steps of 4 dt) gives the same
  transmittance and colour as the level-0 render with steps dt -- (1 - a)^256 by hand over
  128 voxels -- the property the correction exists for;
* the sample positions and levels equal a numpy float32 restatement of the rule;
* brute force: numpy float32 decisions, scipy trilinear on the sample's level, the correction,
  a Python compositing loop, on several storage types.
"""
import numpy as np
import pytest
from scipy import ndimage

import synth

from test_oracle_decisions import axis_camera, _ray_numpy
from test_oracle_values import _random_levels

LEVEL_STEP = 16


def test_constant_medium_transmittance_independent_of_level(orc):
    levels = [np.full((128 >> l,) * 3, 100, np.uint8) for l in range(3)]
    vol = orc.Volume(levels, "u8", 32)
    tf = synth.tf_ramp(alpha_start=0.0, alpha_max=0.05)
    cam = axis_camera((-100.0, 64.0, 64.0), (1, 0, 0))
    bg = (0.1, 0.2, 0.3, 0.5)
    fine = orc.render(vol, cam, tf, {"et": 2.0, "bg": bg})
    coarse = orc.render(vol, cam, tf, {"et": 2.0, "bg": bg, "lod_mode": 1, "lod_bias": 20, "flags": LEVEL_STEP})
    assert fine["n"][0] == 256 and coarse["n"][0] == 64   # 128 voxels in steps of 0.5 and of 2
    a = float(tf[100, 3])
    T = (1 - a) ** 256
    bg64 = np.float64(np.float32(bg))
    want = np.concatenate([tf[100, :3].astype(np.float64) * (1 - T) + T * bg64[:3], [(1 - T) + T * bg64[3]]])
    np.testing.assert_allclose(fine["rgba"][0], want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(coarse["rgba"][0], want, rtol=0, atol=1e-12)
    # without the flag the coarse level keeps steps of dt and the uncorrected opacity
    plain = orc.render(vol, cam, tf, {"et": 2.0, "bg": bg, "lod_mode": 1, "lod_bias": 20})
    np.testing.assert_allclose(plain["rgba"][0], want, rtol=0, atol=1e-12)
    assert plain["n"][0] == 256


def level_step_walk(cam, D, px, py, step, nlevels, bias):
    """numpy float32: (t_k, l_k) of every sample of pixel (px, py)."""
    d, t0, t1 = _ray_numpy(cam, D, px, py)
    scale = (np.float32(2) * np.float32(cam["tan_half_fov"])) / np.float32(cam["h"])
    out, t = [], np.float32(t0)
    if not t0 < t1:
        return out, d
    while t < t1:
        q = np.float32(t * scale)
        lvl = int(np.frexp(np.float64(q))[1]) - 1 + bias if q >= np.float32(2.0 ** -126) else 0
        lvl = min(max(lvl, 0), nlevels - 1)
        out.append((t, lvl))
        t = np.float32(t + np.float32(np.ldexp(np.float32(step), lvl)))
    return out, d


def test_positions_and_levels_match_float32_restatement(orc):
    D = (40, 36, 30)
    shapes = [(30, 36, 40), (15, 18, 20), (8, 9, 10), (4, 5, 5)]
    vol = orc.Volume([np.zeros(s, np.uint8) for s in shapes], "u8", 8)
    cam = dict(synth.seeded_orbit(D, 9, 7, 13, fit=0.7), h=3)
    params = {"lod_mode": 1, "lod_bias": -2, "flags": LEVEL_STEP}
    seen = set()
    for py in range(3):
        for px in range(9):
            recs, n = orc.trace(vol, cam, params, px, py)
            walk, _ = level_step_walk(cam, D, px, py, 0.5, 4, -2)
            assert n == len(walk)
            np.testing.assert_array_equal(recs["t_bits"].view(np.float32), np.array([w[0] for w in walk], np.float32))
            np.testing.assert_array_equal(recs["level"], [w[1] for w in walk])
            seen.update(int(l) for l in recs["level"])
    assert len(seen) >= 2


def brute_force_level_step(levels_f64, D, cam, tf, px, py, step, et, bg, bias):
    walk, d = level_step_walk(cam, D, px, py, step, len(levels_f64), bias)
    o = np.asarray(cam["eye"], np.float32)
    xs = np.arange(256, dtype=np.float64)
    T, C, k = 1.0, np.zeros(3), 0
    for t, lvl in walk:
        k += 1
        p = [np.float32(o[a] + t * d[a]) for a in range(3)]
        arr = levels_f64[lvl]
        ratio = [np.float32(np.float32(arr.shape[2 - a]) / np.float32(D[a])) for a in range(3)]
        coords = np.array([[float(np.float32(p[a] * ratio[a]) - np.float32(0.5))] for a in (2, 1, 0)])
        val = ndimage.map_coordinates(arr, coords, order=1, mode="nearest")[0]
        x = min(max(val, 0.0), 1.0) * 255.0
        rgba = [np.interp(x, xs, tf[:, ch].astype(np.float64)) for ch in range(4)]
        a = 1 - (1 - rgba[3]) ** (2 ** lvl)
        C += T * a * np.array(rgba[:3])
        T *= 1 - a
        if (1 - T) >= et:
            break
    return np.array([*(C + T * np.array(bg[:3])), (1 - T) + T * bg[3]]), k


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_brute_force_small_volume(orc, dtype):
    rng = np.random.default_rng(23)
    D = (12, 10, 9)
    raws, f64 = _random_levels(dtype, [(9, 10, 12), (5, 5, 6), (3, 3, 3)], rng)
    vol = orc.Volume(raws, dtype, 4)
    tf = synth.tf_peaks(6)
    tf[:, 3] = np.clip(tf[:, 3] + 0.05, 0, 1)
    bg = tuple(float(np.float32(b)) for b in (0.2, 0.1, 0.0, 0.3))
    et = float(np.float32(0.99))
    for view in range(3):
        cam = dict(synth.seeded_orbit(D, 11, 9, 21, view=view, fit=0.7), h=1)
        params = {"bg": bg, "et": 0.99, "lod_mode": 1, "lod_bias": -2, "flags": LEVEL_STEP}
        out = orc.render(vol, cam, tf, params)
        for i in range(11):
            want, n = brute_force_level_step(f64, D, cam, tf, i, 0, 0.5, et, bg, -2)
            assert out["n"][i] == n
            np.testing.assert_allclose(out["rgba"][i], want, rtol=0, atol=1e-12)
