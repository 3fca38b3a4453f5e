"""Pins for the oracle's maximum projections (MOP, MIP; Sec. V-A renders the Kidney data with MOP).

* transparent TF / empty volume -> the background, exactly (both modes);
* constant density -> the one-sample composite of tf(c), by hand;
* a linear ramp along the ray with a TF linear in the entry index -> the last sample wins;
  its value, TF colour and composite evaluated in 50-digit mpmath from closed-form positions;
* brute force: scipy.ndimage.map_coordinates (order 1, edge mode) per sample, numpy.interp for
  the TF, numpy argmax / max for the selection, on every dtype with and without LOD;
* the candidate range (lo, hi) with a wide margin spans exactly the outputs of all samples.
"""
import mpmath
import numpy as np
import pytest
from scipy import ndimage

import synth

from test_oracle_decisions import axis_camera, _ray_numpy
from test_oracle_values import _random_levels, ramp_tf


def one_sample(rgba, bg):
    a = rgba[3]
    return np.array([a * rgba[0] + (1 - a) * bg[0], a * rgba[1] + (1 - a) * bg[1],
                     a * rgba[2] + (1 - a) * bg[2], a + (1 - a) * bg[3]])


@pytest.mark.parametrize("mode", ["mop", "mip"])
def test_transparent_is_background(orc, mode):
    bg = (0.25, 0.5, 0.125, 1.0)
    cam = synth.seeded_orbit((16, 16, 16), 9, 7, 5)
    vol = orc.Volume([np.random.default_rng(0).integers(0, 256, (16, 16, 16), dtype=np.uint8)], "u8", 8)
    tf0 = synth.tf_ramp().copy(); tf0[:, 3] = 0
    out = orc.render_max(vol, cam, tf0, {"bg": bg}, mode)
    np.testing.assert_array_equal(out["rgba"], np.tile(np.float64(np.float32(bg)), (63, 1)))
    if mode == "mop":
        # an empty volume under a TF with alpha 0 at value 0 as well
        out2 = orc.render_max(orc.Volume([np.zeros((16, 16, 16), np.uint8)], "u8", 8), cam, synth.tf_ramp(),
                              {"bg": bg}, mode)
        np.testing.assert_array_equal(out2["rgba"], out["rgba"])


@pytest.mark.parametrize("mode", ["mop", "mip"])
def test_constant_density(orc, mode):
    vol = orc.Volume([np.full((64, 64, 64), 100, np.uint8)], "u8", 32)
    tf = synth.tf_ramp(alpha_start=0.0, alpha_max=0.5)
    bg = np.float64(np.float32([0.1, 0.2, 0.3, 0.5]))
    cam = axis_camera((-100.0, 32.0, 32.0), (1, 0, 0))
    out = orc.render_max(vol, cam, tf, {"bg": tuple(bg)}, mode)
    assert out["n"][0] == 128                           # 64 voxels / 0.5, by hand
    want = one_sample(tf[100].astype(np.float64), bg)   # x = 100 exactly: entry 100
    np.testing.assert_allclose(out["rgba"][0], want, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(out["lo"], out["rgba"])
    np.testing.assert_array_equal(out["hi"], out["rgba"])


@pytest.mark.parametrize("mode", ["mop", "mip"])
def test_linear_ramp_last_sample(orc, mode):
    # v(i) = i / 128 along x; ray along +x; alpha_j increases with j, so both modes keep the
    # last sample, at p = 0.5 * 257 -> grid coordinate 128 (clamped), value 1
    v = (np.arange(129, dtype=np.float64) / 128).astype(np.float32)
    vol = orc.Volume([np.broadcast_to(v, (8, 8, 129)).copy()], "f32", 16)
    tf = ramp_tf()
    cam = axis_camera((-50.0, 4.0, 4.0), (1, 0, 0))
    out = orc.render_max(vol, cam, tf, {"et": 0.5}, mode)  # et plays no part here
    assert out["n"][0] == 258
    mpmath.mp.dps = 50
    x = min(max(mpmath.mpf(257) / 2 - mpmath.mpf(1) / 2, 0), 128)
    j = x / 128 * 255
    al = mpmath.mpf(2) ** -10 + j * mpmath.mpf(2) ** -14
    col = [j * mpmath.mpf(2) ** -8, mpmath.mpf(1) / 2, 1 - j * mpmath.mpf(2) ** -8]
    want = [float(al * c) for c in col] + [float(al)]
    np.testing.assert_allclose(out["rgba"][0], want, rtol=0, atol=1e-14)
    # a ray of the same data, reversed: the ramp now decreases along it and the first
    # sample (grid coordinate 128 again) is the one kept
    cam2 = axis_camera((200.0, 4.0, 4.0), (-1, 0, 0))
    out2 = orc.render_max(vol, cam2, tf, {}, mode)
    np.testing.assert_allclose(out2["rgba"][0], want, rtol=0, atol=1e-14)


def brute_force_samples(levels_f64, D, cam, tf, px, py, step, lod=False, bias=0):
    """Every sample's TF coordinate and RGBA: float32 ray (numpy), footprint level from
    numpy.frexp, scipy trilinear with edge clamping on that level's grid, numpy.interp TF."""
    d, t0, t1 = _ray_numpy(cam, D, px, py)
    o = np.asarray(cam["eye"], np.float32)
    xs_tf = np.arange(256, dtype=np.float64)
    scale = (np.float32(2) * np.float32(cam["tan_half_fov"])) / np.float32(cam["h"])
    xs, rgbas = [], []
    if not t0 < t1:
        return np.zeros(0), np.zeros((0, 4))
    k = 0
    while True:
        t = np.float32(t0 + np.float32(k) * np.float32(step))
        if not t < t1:
            break
        p = [np.float32(o[a] + t * d[a]) for a in range(3)]
        lvl = 0
        if lod:
            q = np.float32(t * scale)
            if q >= np.float32(2.0 ** -126):
                lvl = int(np.frexp(np.float64(q))[1]) - 1 + bias
            lvl = min(max(lvl, 0), len(levels_f64) - 1)
        arr = levels_f64[lvl]
        ratio = [np.float32(np.float32(arr.shape[2 - a]) / np.float32(D[a])) for a in range(3)]
        coords = np.array([[float(np.float32(p[a] * ratio[a]) - np.float32(0.5))] for a in (2, 1, 0)])
        val = ndimage.map_coordinates(arr, coords, order=1, mode="nearest")[0]
        x = min(max(val, 0.0), 1.0) * 255.0
        xs.append(x)
        rgbas.append([np.interp(x, xs_tf, tf[:, ch].astype(np.float64)) for ch in range(4)])
        k += 1
    return np.array(xs), np.array(rgbas)


@pytest.mark.parametrize("dtype", ["u8", "u16", "f16", "f32"])
@pytest.mark.parametrize("lod", [False, True])
def test_brute_force_small_volume(orc, dtype, lod):
    rng = np.random.default_rng(17)
    D = (12, 10, 9)
    raws, f64 = _random_levels(dtype, [(9, 10, 12), (5, 5, 6), (3, 3, 3)], rng)
    vol = orc.Volume(raws, dtype, 4)
    # opacity peaks over a ramp, red ramping too: no flat ends, so a clamp error shows
    tf = synth.tf_peaks(5)
    ramp = np.arange(256) / 255.0
    tf[:, 3] = np.clip(tf[:, 3] + 0.2 * ramp, 0, 1)
    tf[:, 0] = ramp
    bg = tuple(float(np.float32(b)) for b in (0.2, 0.1, 0.0, 0.3))
    bg64 = np.array(bg)
    xs_tf = np.arange(256, dtype=np.float64)
    for view in range(3):
        cam = synth.seeded_orbit(D, 11, 9, 23, view=view, fit=0.7)
        if lod:
            cam = dict(cam, h=1)
        params = {"bg": bg, "lod_mode": int(lod), "lod_bias": -2 if lod else 0}
        mop = orc.render_max(vol, cam, tf, params, "mop")
        mip = orc.render_max(vol, cam, tf, params, "mip")
        ties = 0
        for i in range(0, 11 * cam["h"], 3 if lod else 5):
            px, py = i % 11, i // 11
            xs, rgbas = brute_force_samples(f64, D, cam, tf, px, py, 0.5, lod=lod, bias=-2)
            assert mop["n"][i] == len(xs) == mip["n"][i]
            if len(xs) == 0:
                np.testing.assert_array_equal(mop["rgba"][i], bg64)
                np.testing.assert_array_equal(mip["rgba"][i], bg64)
                continue
            # MIP: the TF at the largest coordinate
            want = one_sample(np.array([np.interp(xs.max(), xs_tf, tf[:, ch].astype(np.float64))
                                        for ch in range(4)]), bg64)
            np.testing.assert_allclose(mip["rgba"][i], want, rtol=0, atol=1e-12)
            # MOP: the first sample of largest opacity (numpy.argmax keeps the first)
            want = one_sample(rgbas[np.argmax(rgbas[:, 3])], bg64)
            if np.array_equal(mop["lo"][i], mop["hi"][i]):
                np.testing.assert_allclose(mop["rgba"][i], want, rtol=0, atol=1e-12)
            else:
                ties += 1
                assert np.all(want >= mop["lo"][i] - 1e-12) and np.all(want <= mop["hi"][i] + 1e-12)
                assert mop["rgba"][i][3] == pytest.approx(want[3], abs=1e-5)
        assert ties <= 2


def test_candidate_range_spans_near_maximal_samples(orc):
    rng = np.random.default_rng(5)
    D = (12, 10, 9)
    raws, f64 = _random_levels("u16", [(9, 10, 12)], rng)
    vol = orc.Volume(raws, "u16", 4)
    tf = synth.tf_peaks(5)
    bg = (0.2, 0.1, 0.0, 0.3)
    bg64 = np.float64(np.float32(bg))
    cam = synth.seeded_orbit(D, 11, 9, 23, view=1, fit=0.7)
    margin = 0.05
    out = orc.render_max(vol, cam, tf, {"bg": bg}, "mop", amb=margin)
    wide = 0
    for i in range(0, 99, 4):
        xs, rgbas = brute_force_samples(f64, D, cam, tf, i % 11, i // 11, 0.5)
        if len(xs) == 0:
            continue
        amax = rgbas[:, 3].max()
        cand = np.array([one_sample(r, bg64) for r in rgbas if r[3] >= amax - margin + 1e-9])
        strict = np.array([one_sample(r, bg64) for r in rgbas if r[3] >= amax - margin - 1e-9])
        # the oracle's range lies between the ranges of the candidates just inside and just
        # outside the margin (rounding of the brute force's opacities)
        assert np.all(out["lo"][i] <= cand.min(0) + 1e-12) and np.all(out["hi"][i] >= cand.max(0) - 1e-12)
        assert np.all(out["lo"][i] >= strict.min(0) - 1e-12) and np.all(out["hi"][i] <= strict.max(0) + 1e-12)
        wide += len(cand) > 1
    assert wide > 3


def test_mop_keeps_the_first_of_equal_opacities(orc):
    # every TF entry has alpha 1/2, colour r = j / 256: all samples tie on opacity, so MOP keeps
    # the first one -- on a ray along -x through the ramp, grid coordinate 128, value 1, entry 255
    v = (np.arange(129, dtype=np.float64) / 128).astype(np.float32)
    vol = orc.Volume([np.broadcast_to(v, (8, 8, 129)).copy()], "f32", 16)
    j = np.arange(256, dtype=np.float64)
    tf = np.stack([j / 256, np.full(256, 0.25), np.zeros(256), np.full(256, 0.5)], 1).astype(np.float32)
    cam = axis_camera((200.0, 4.0, 4.0), (-1, 0, 0))
    out = orc.render_max(vol, cam, tf, {}, "mop")
    np.testing.assert_array_equal(out["rgba"][0], [0.5 * 255 / 256, 0.125, 0.0, 0.5])
    # every sample is a candidate: the range runs from entry 0's colour to entry 255's
    np.testing.assert_array_equal(out["lo"][0], [0.0, 0.125, 0.0, 0.5])
    np.testing.assert_array_equal(out["hi"][0], out["rgba"][0])
