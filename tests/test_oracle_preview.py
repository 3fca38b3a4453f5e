"""Pins for the oracle's progressive preview (Sec. III-H: a coarse image first, refined as bricks
arrive): under a residency map, a sample whose brick is absent on its level is taken on the
finest coarser resident level at the same position, or composites nothing.

* every brick resident -> exactly the full render (DVR and MOP);
* nothing resident -> the background, every sample still passed;
* only the coarsest level resident -> exactly the render whose footprint LOD puts every sample
  on the coarsest level (lod_bias +20), with LOD on or off;
* brute force with a random residency map: numpy float32 decisions for the level and brick
  on every level, scipy trilinear on the level chosen, a Python compositing loop.
"""
import numpy as np
import pytest
from scipy import ndimage

import synth

from test_oracle_decisions import _ray_numpy
from test_oracle_values import _random_levels


def pt_offsets(shapes, B):
    offs, n = [], 0
    for (Dz, Dy, Dx) in shapes:
        offs.append(n)
        n += -(-Dx // B) * -(-Dy // B) * -(-Dz // B)
    return offs, n


def small_case(dtype="u16", seed=3):
    rng = np.random.default_rng(seed)
    D = (24, 20, 18)
    shapes = [(18, 20, 24), (9, 10, 12), (5, 5, 6), (3, 3, 3)]
    raws, f64 = _random_levels(dtype, shapes, rng)
    return D, shapes, raws, f64


def test_all_resident_is_the_full_render(orc):
    D, shapes, raws, _ = small_case()
    vol = orc.Volume(raws, "u16", 4)
    tf = synth.tf_peaks(2)
    tf[:, 3] = np.clip(tf[:, 3] + 0.03, 0, 1)
    cam = dict(synth.seeded_orbit(D, 13, 11, 4, fit=0.8), h=3)
    params = {"lod_mode": 1, "lod_bias": -2, "bg": (0.1, 0.2, 0.3, 0.4)}
    res = np.ones(orc.page_table_size(vol), np.uint8)
    full = orc.render(vol, cam, tf, params)
    prev = orc.render_preview(vol, cam, tf, params, res)
    np.testing.assert_array_equal(prev["rgba"], full["rgba"])
    np.testing.assert_array_equal(prev["n"], full["n"])
    m_full = orc.render_max(vol, cam, tf, params, "mop")
    m_prev = orc.render_max(vol, cam, tf, params, "mop", resident=res)
    np.testing.assert_array_equal(m_prev["rgba"], m_full["rgba"])


def test_nothing_resident_is_background(orc):
    D, shapes, raws, _ = small_case()
    vol = orc.Volume(raws, "u16", 4)
    tf = synth.tf_ramp(alpha_start=0.0, alpha_max=0.5)
    cam = synth.seeded_orbit(D, 13, 11, 4, fit=0.8)
    bg = (0.1, 0.2, 0.3, 0.4)
    res = np.zeros(orc.page_table_size(vol), np.uint8)
    prev = orc.render_preview(vol, cam, tf, {"bg": bg}, res)
    np.testing.assert_array_equal(prev["rgba"], np.tile(np.float64(np.float32(bg)), (13 * 11, 1)))
    # every sample of every ray is passed (none composites, so none terminates the ray)
    full = orc.render(vol, cam, tf, {"bg": bg, "et": 2.0})
    np.testing.assert_array_equal(prev["n"], full["n"])


@pytest.mark.parametrize("lod", [0, 1])
def test_coarsest_only_equals_coarsest_lod(orc, lod):
    D, shapes, raws, _ = small_case("f32", 5)
    vol = orc.Volume(raws, "f32", 4)
    tf = synth.tf_peaks(6)
    tf[:, 3] = np.clip(tf[:, 3] + 0.03, 0, 1)
    cam = synth.seeded_orbit(D, 13, 11, 7, fit=0.8)
    offs, n = pt_offsets(shapes, 4)
    res = np.zeros(n, np.uint8)
    res[offs[-1]:] = 1
    prev = orc.render_preview(vol, cam, tf, {"lod_mode": lod, "lod_bias": 0}, res)
    coarse = orc.render(vol, cam, tf, {"lod_mode": 1, "lod_bias": 20})
    np.testing.assert_array_equal(prev["rgba"], coarse["rgba"])


def brute_force_preview(levels_f64, shapes, B, resident, D, cam, tf, px, py, step, et, bg, bias):
    d, t0, t1 = _ray_numpy(cam, D, px, py)
    o = np.asarray(cam["eye"], np.float32)
    if not t0 < t1:
        return np.array(bg, np.float64)
    offs, _ = pt_offsets(shapes, B)
    xs = np.arange(256, dtype=np.float64)
    scale = (np.float32(2) * np.float32(cam["tan_half_fov"])) / np.float32(cam["h"])
    T, C, k = 1.0, np.zeros(3), 0
    while True:
        t = np.float32(t0 + np.float32(k) * np.float32(step))
        if not t < t1:
            break
        k += 1
        p = [np.float32(o[a] + t * d[a]) for a in range(3)]
        q = np.float32(t * scale)
        want = int(np.frexp(np.float64(q))[1]) - 1 + bias if q >= np.float32(2.0 ** -126) else 0
        want = min(max(want, 0), len(shapes) - 1)
        use = None
        for lvl in range(want, len(shapes)):
            Dl = shapes[lvl][::-1]   # (Dx, Dy, Dz)
            g = []
            for a in range(3):
                x = np.float32(np.float32(p[a] * np.float32(np.float32(Dl[a]) / np.float32(D[a]))) - np.float32(0.5))
                g.append(min(max(int(np.floor(x)), 0), Dl[a] - 1))
            nb = [-(-Dl[a] // B) for a in range(3)]
            bid = g[0] // B + nb[0] * (g[1] // B + nb[1] * (g[2] // B))
            if resident[offs[lvl] + bid]:
                use = lvl
                break
        if use is None:
            continue
        arr = levels_f64[use]
        ratio = [np.float32(np.float32(arr.shape[2 - a]) / np.float32(D[a])) for a in range(3)]
        coords = np.array([[float(np.float32(p[a] * ratio[a]) - np.float32(0.5))] for a in (2, 1, 0)])
        val = ndimage.map_coordinates(arr, coords, order=1, mode="nearest")[0]
        x = min(max(val, 0.0), 1.0) * 255.0
        rgba = [np.interp(x, xs, tf[:, ch].astype(np.float64)) for ch in range(4)]
        C += T * rgba[3] * np.array(rgba[:3])
        T *= 1 - rgba[3]
        if (1 - T) >= et:
            break
    return np.array([*(C + T * np.array(bg[:3])), (1 - T) + T * bg[3]])


@pytest.mark.parametrize("dtype", ["u8", "f16"])
def test_brute_force_random_residency(orc, dtype):
    D, shapes, raws, f64 = small_case(dtype, 9)
    vol = orc.Volume(raws, dtype, 4)
    tf = synth.tf_peaks(8)
    tf[:, 3] = np.clip(tf[:, 3] + 0.05, 0, 1)
    bg = tuple(float(np.float32(b)) for b in (0.2, 0.1, 0.0, 0.3))
    et = float(np.float32(0.99))
    rng = np.random.default_rng(12)
    _, n = pt_offsets(shapes, 4)
    res = (rng.random(n) < 0.5).astype(np.uint8)
    skipped = 0
    for view in range(2):
        cam = dict(synth.seeded_orbit(D, 11, 9, 21, view=view, fit=0.7), h=2)
        params = {"bg": bg, "et": 0.99, "lod_mode": 1, "lod_bias": -3}
        out = orc.render_preview(vol, cam, tf, params, res)
        for i in range(0, 11 * 2):
            want = brute_force_preview(f64, shapes, 4, res, D, cam, tf, i % 11, i // 11, 0.5, et, bg, -3)
            np.testing.assert_allclose(out["rgba"][i], want, rtol=0, atol=1e-12)
        full = orc.render(vol, cam, tf, params)
        skipped += int(np.any(np.abs(full["rgba"] - out["rgba"]) > 1e-9))
    assert skipped > 0   # the residency map does change the image
