"""Pins for the oracle's value layer: compositing, interpolation, transfer function, adjoint.

* empty volume / transparent TF -> the background, exactly;
* constant density -> 1 - (1 - a)^n, n by hand (with and without early termination);
* a linear ramp with a linear TF -> the discrete sum evaluated in 50-digit mpmath from
  closed-form sample values;
* brute force: scipy.ndimage.map_coordinates (order 1, edge mode) for the trilinear step,
  numpy.interp for the TF, a plain Python compositing loop;
* adjoint: central finite differences of the float64 oracle itself, plus the closed-form
  derivative of 1 - (1 - a)^n.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy import ndimage

import synth

from test_oracle_decisions import axis_camera, _ray_numpy


def ramp_tf():
    """TF whose entries are exactly linear in the entry index (all values dyadic):
    alpha_j = 2^-10 + j 2^-14, r_j = j 2^-8, g = 0.5, b = 1 - j 2^-8."""
    j = np.arange(256, dtype=np.float64)
    tf = np.stack([j * 2.0 ** -8, np.full(256, 0.5), 1 - j * 2.0 ** -8, 2.0 ** -10 + j * 2.0 ** -14], 1)
    return tf.astype(np.float32)


def test_empty_volume_is_background(orc):
    vol = orc.Volume([np.zeros((16, 16, 16), np.uint8)], "u8", 8)
    tf = synth.tf_ramp()          # alpha = 0 below 0.1
    bg = (0.25, 0.5, 0.125, 1.0)
    cam = synth.seeded_orbit((16, 16, 16), 9, 7, 5)
    out = orc.render(vol, cam, tf, {"bg": bg})
    np.testing.assert_array_equal(out["rgba"], np.tile(np.float64(np.float32(bg)), (63, 1)))
    # a transparent TF gives the same on any data
    vol2 = orc.Volume([np.random.default_rng(0).integers(0, 256, (16, 16, 16), dtype=np.uint8)], "u8", 8)
    tf0 = tf.copy(); tf0[:, 3] = 0
    out2 = orc.render(vol2, cam, tf0, {"bg": bg})
    np.testing.assert_array_equal(out2["rgba"], out["rgba"])


def constant_case(orc, value, et):
    vol = orc.Volume([np.full((128, 128, 128), value, np.uint8)], "u8", 32)
    tf = synth.tf_ramp(alpha_start=0.0, alpha_max=0.05)
    cam = axis_camera((-100.0, 64.0, 64.0), (1, 0, 0))
    out = orc.render(vol, cam, tf, {"et": et, "bg": (0.1, 0.2, 0.3, 0.5)})
    a = float(tf[value, 3]); rgb = tf[value, :3].astype(np.float64)
    return out, a, rgb


def test_constant_density_closed_form(orc):
    out, a, rgb = constant_case(orc, 100, et=2.0)      # threshold never reached
    n = 256                                               # by hand (see the decision tests)
    assert out["n"][0] == n
    T = (1 - a) ** n
    bg = np.float64(np.float32([0.1, 0.2, 0.3, 0.5]))
    np.testing.assert_allclose(out["rgba"][0, :3], rgb * (1 - T) + T * bg[:3], rtol=0, atol=1e-12)
    assert out["rgba"][0, 3] == pytest.approx((1 - T) + T * bg[3], abs=1e-12)


def test_constant_density_early_termination(orc):
    out, a, rgb = constant_case(orc, 250, et=0.99)
    et = float(np.float32(0.99))
    m = math.ceil(math.log(1 - et) / math.log(1 - a))   # smallest m with 1-(1-a)^m >= et
    assert 1 - (1 - a) ** m >= et > 1 - (1 - a) ** (m - 1)
    assert out["n"][0] == min(256, m)
    T = (1 - a) ** m
    assert out["rgba"][0, 3] == pytest.approx((1 - T) + T * float(np.float32(0.5)), abs=1e-12)


def test_linear_ramp_discrete_sum(orc):
    # f32 volume 129 x 8 x 8 with v(i) = i / 128 along x (exact); ray along +x at the centre
    D = (129, 8, 8)
    v = (np.arange(129, dtype=np.float64) / 128).astype(np.float32)
    vol = orc.Volume([np.broadcast_to(v, (8, 8, 129)).copy()], "f32", 16)
    tf = ramp_tf()
    cam = axis_camera((-50.0, 4.0, 4.0), (1, 0, 0))
    out = orc.render(vol, cam, tf, {"et": 2.0})
    # samples at p = 0.5 k, k = 0..257; grid coordinate x = p - 0.5 clamped to [0, 128]
    mpmath.mp.dps = 50
    T = mpmath.mpf(1); C = [mpmath.mpf(0)] * 3
    n = 258
    for k in range(n):
        x = min(max(mpmath.mpf(k) / 2 - mpmath.mpf(1) / 2, 0), 128)
        val = x / 128                                   # interpolated ramp value
        j = val * 255                                    # TF coordinate; entries are linear in j
        al = mpmath.mpf(2) ** -10 + j * mpmath.mpf(2) ** -14
        col = [j * mpmath.mpf(2) ** -8, mpmath.mpf(1) / 2, 1 - j * mpmath.mpf(2) ** -8]
        for ch in range(3):
            C[ch] += T * al * col[ch]
        T *= (1 - al)
    assert out["n"][0] == n
    np.testing.assert_allclose(out["rgba"][0], [float(C[0]), float(C[1]), float(C[2]), float(1 - T)],
                               rtol=0, atol=1e-12)


def brute_force_pixel(levels_f64, D, cam, tf, px, py, step, et, bg, lod=False, bias=0):
    """Plain restatement: float32 ray (numpy), footprint level from numpy.frexp, scipy trilinear
    with edge clamping on that level's grid, numpy.interp TF, a Python compositing loop."""
    d, t0, t1 = _ray_numpy(cam, D, px, py)
    o = np.asarray(cam["eye"], np.float32)
    if not t0 < t1:
        return np.array(bg, np.float64), 0
    T, C, k = 1.0, np.zeros(3), 0
    xs = np.arange(256, dtype=np.float64)
    scale = (np.float32(2) * np.float32(cam["tan_half_fov"])) / np.float32(cam["h"])
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
        rgba = [np.interp(x, xs, tf[:, ch].astype(np.float64)) for ch in range(4)]
        C += T * rgba[3] * np.array(rgba[:3])
        T *= 1 - rgba[3]
        k += 1
        if (1 - T) >= et:
            break
    return np.array([*(C + T * np.array(bg[:3])), (1 - T) + T * bg[3]]), k


def _random_levels(dtype, shapes, rng):
    raws, f64 = [], []
    for shp in shapes:
        if dtype == "u8":
            r = rng.integers(0, 256, shp, dtype=np.uint8); f = r / 255.0
        elif dtype == "u16":
            r = rng.integers(0, 65536, shp, dtype=np.uint16); f = r / 65535.0
        elif dtype == "f16":
            r = (rng.random(shp) * 1.2 - 0.1).astype(np.float16); f = r.astype(np.float64); r = r.view(np.uint16)
        else:
            r = rng.random(shp, dtype=np.float32) * np.float32(1.2) - np.float32(0.1); f = r.astype(np.float64)
        raws.append(r); f64.append(f)
    return raws, f64


@pytest.mark.parametrize("dtype", ["u8", "u16", "f16", "f32"])
@pytest.mark.parametrize("lod", [False, True])
def test_brute_force_small_volume(orc, dtype, lod):
    rng = np.random.default_rng(11)
    D = (12, 10, 9)
    # independent random levels (the render does not care how levels were made)
    raws, f64 = _random_levels(dtype, [(9, 10, 12), (5, 5, 6), (3, 3, 3)], rng)
    vol = orc.Volume(raws, dtype, 4)
    tf = synth.tf_peaks(4)
    tf[:, 3] = np.clip(tf[:, 3] + 0.05, 0, 1)
    bg = tuple(float(np.float32(b)) for b in (0.2, 0.1, 0.0, 0.3))
    et = float(np.float32(0.99))
    for view in range(3):
        cam = synth.seeded_orbit(D, 11, 9, 21, view=view, fit=0.7)
        if lod:
            # footprint large enough that samples spread over all three levels
            cam = dict(cam, h=1)
        params = {"bg": bg, "et": 0.99, "lod_mode": int(lod), "lod_bias": -2 if lod else 0}
        h = cam["h"]
        npx = 11 * h
        out = orc.render(vol, cam, tf, params)
        for i in range(0, npx, 3 if lod else 7):
            px, py = i % 11, i // 11
            want, n = brute_force_pixel(f64, D, cam, tf, px, py, 0.5, et, bg, lod=lod, bias=-2)
            assert out["n"][i] == n
            np.testing.assert_allclose(out["rgba"][i], want, rtol=0, atol=1e-12)


def test_ambiguity_flags_only_near_threshold(orc):
    vol = orc.Volume([synth.blobs((48, 48, 48), 3, sigma=(4, 10))], "u8", 16)
    tf = synth.tf_ramp(alpha_max=0.3)
    cam = synth.seeded_orbit((48, 48, 48), 64, 64, 3)
    out = orc.render(vol, cam, tf, {"et": 0.99}, amb=1e-3)
    amb = out["amb"]
    assert amb.any()
    # the alternate flips one decision: its sample count differs, unless that decision fell on
    # the ray's last sample (then both results are the same)
    same_n = out["alt_n"] == out["n"]
    np.testing.assert_array_equal(out["alt_rgba"][amb & same_n], out["rgba"][amb & same_n])
    assert np.any(amb & ~same_n)
    np.testing.assert_array_equal(out["alt_rgba"][~amb], out["rgba"][~amb])
    # output alpha is a probability
    assert np.all((out["rgba"][:, 3] >= 0) & (out["rgba"][:, 3] <= 1))


# ------------------------------------------------------------------ adjoint


def test_grad_closed_form_constant(orc):
    # f32 constant volume at TF coordinate x = 100.5 (i = 100, w = 0.5), no termination:
    # I_a = 1 - (1 - a)^n, a = (tf[100].a + tf[101].a)/2; dI_a/dtf[100].a = 0.5 n (1 - a)^(n-1)
    val = np.float32(100.5 / 255.0)
    vol = orc.Volume([np.full((128, 128, 128), val, np.float32)], "f32", 32)
    tf = synth.tf_ramp(alpha_start=0.0, alpha_max=0.02)
    cam = axis_camera((-100.0, 64.0, 64.0), (1, 0, 0))
    dtf, dvox = orc.render_grad(vol, cam, tf, {"et": 2.0}, np.array([[0, 0, 0, 1.0]]))
    x = float(val) * 255.0
    w = x - 100
    a = (1 - w) * float(tf[100, 3]) + w * float(tf[101, 3])
    n = 256
    g = n * (1 - a) ** (n - 1)
    assert dtf[100, 3] == pytest.approx((1 - w) * g, rel=1e-12)
    assert dtf[101, 3] == pytest.approx(w * g, rel=1e-12)
    assert np.all(dtf[:, :3] == 0)
    # dI_a/dv summed over voxels = n (1-a)^(n-1) * 255 * (tf[101].a - tf[100].a)  (weights sum to 1)
    assert dvox.sum() == pytest.approx(g * 255 * (float(tf[101, 3]) - float(tf[100, 3])), rel=1e-9)


def _loss_and_grad(orc, vol, cams, tf, target, params):
    L, dtf, dvox = 0.0, np.zeros((256, 4)), np.zeros(vol.levels[0].shape)
    ns = []
    for cam, tgt in zip(cams, target):
        out = orc.render(vol, cam, tf, params)
        r = out["rgba"] - tgt
        L += 0.5 * float(np.sum(r * r))
        g1, g2 = orc.render_grad(vol, cam, tf, params, r)
        dtf += g1; dvox += g2
        ns.append(out["n"])
    return L, dtf, dvox, np.concatenate(ns)


def _fd_setup(orc, linear_tf):
    D = (20, 18, 16)
    # values stay inside (0, 0.95]: the clamp to [0, 1] before the TF has a kink at 0 and 1
    raw = synth.blobs(D, 5, dtype="f32", nblobs=5, sigma=(3, 6), amp=(0.2, 1.0), noise=0.05, vmax=0.95)
    vol = orc.Volume([raw], "f32", 8)
    if linear_tf:
        j = np.arange(256) / 255.0
        tf = np.stack([0.2 + 0.6 * j, 0.9 - 0.5 * j, 0.3 + 0.2 * j, 0.02 + 0.25 * j], 1).astype(np.float32)
    else:
        tf = synth.tf_peaks(7)
        tf[:, 3] = np.clip(tf[:, 3] + 0.03, 0, 1)
    cams = [synth.seeded_orbit(D, 24, 20, 9, view=v) for v in range(2)]
    params = {"et": 0.99, "bg": (0.1, 0.1, 0.2, 0.0)}
    tgt_tf = synth.tf_perturbed(tf, 13)
    target = [orc.render(vol, c, tgt_tf, params)["rgba"] for c in cams]
    return vol, raw, tf, cams, target, params


def test_grad_tf_matches_central_differences(orc):
    vol, raw, tf, cams, target, params = _fd_setup(orc, linear_tf=False)
    L0, dtf, _, n0 = _loss_and_grad(orc, vol, cams, tf, target, params)
    rng = np.random.default_rng(2)
    used = np.flatnonzero(np.abs(dtf).sum(1) > 0)
    h = 1e-3
    checked = 0
    for _ in range(64):
        j, ch = int(rng.choice(used)), int(rng.integers(0, 4))
        tp, tm = tf.copy(), tf.copy()
        tp[j, ch] += h; tm[j, ch] -= h
        hp, hm = float(tp[j, ch]) - float(tf[j, ch]), float(tf[j, ch]) - float(tm[j, ch])
        Lp, _, _, np_ = _loss_and_grad(orc, vol, cams, tp, target, params)
        Lm, _, _, nm = _loss_and_grad(orc, vol, cams, tm, target, params)
        if not (np.array_equal(np_, n0) and np.array_equal(nm, n0)):
            continue        # an early-termination index moved: the loss has a jump here
        fd = (Lp - Lm) / (hp + hm)
        # L is quadratic in the TF entries for fixed sample indices; central FD of a quadratic
        # in one coordinate is exact up to float64 rounding
        assert fd == pytest.approx(dtf[j, ch], rel=1e-4, abs=1e-9), (j, ch)
        checked += 1
    assert checked >= 48


@pytest.mark.parametrize("linear_tf,h", [(True, 1e-3), (False, 1e-6)])
def test_grad_voxel_matches_central_differences(orc, linear_tf, h):
    vol, raw, tf, cams, target, params = _fd_setup(orc, linear_tf)
    L0, _, dvox, n0 = _loss_and_grad(orc, vol, cams, tf, target, params)
    rng = np.random.default_rng(4)
    cand = np.argwhere(np.abs(dvox) > 1e-3 * np.abs(dvox).max())
    checked = 0
    for _ in range(64):
        z, y, x = cand[int(rng.integers(0, len(cand)))]
        rp, rm = raw.copy(), raw.copy()
        rp[z, y, x] += np.float32(h); rm[z, y, x] -= np.float32(h)
        hp = float(rp[z, y, x]) - float(raw[z, y, x]); hm = float(raw[z, y, x]) - float(rm[z, y, x])
        Lp, _, _, np_ = _loss_and_grad(orc, orc.Volume([rp], "f32", 8), cams, tf, target, params)
        Lm, _, _, nm = _loss_and_grad(orc, orc.Volume([rm], "f32", 8), cams, tf, target, params)
        if not (np.array_equal(np_, n0) and np.array_equal(nm, n0)):
            continue
        fd = (Lp - Lm) / (hp + hm)
        # linear TF: no knots, so the only curvature is smooth (O(h^2)); the non-linear TF uses a
        # step small enough that crossing a knot is rare, and a crossing shows as a large miss
        assert fd == pytest.approx(dvox[z, y, x], rel=1e-4, abs=1e-7 * np.abs(dvox).max()), (z, y, x)
        checked += 1
    assert checked >= 40
