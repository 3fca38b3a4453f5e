"""Pins for the oracle's decision layer: ray setup, slab entry/exit, sample count, LOD level,
voxel index, brick id and local position (chunk addressing, Sec. III-A).

Expected values are worked by hand for exactly representable cases, or recomputed with
numpy float32 scalars written independently of oracle.c.
"""
import math

import numpy as np
import pytest

import synth


def axis_camera(eye, fwd, w=1, h=1, tan=0.5):
    """A camera looking along +x/+y/+z with exactly representable vectors."""
    fwd = np.asarray(fwd, np.float32)
    up = np.array([0, 0, 1], np.float32) if abs(fwd[2]) < 0.5 else np.array([0, 1, 0], np.float32)
    right = np.cross(fwd, up).astype(np.float32)
    return {"eye": np.asarray(eye, np.float32), "right": right, "up": up, "fwd": fwd,
            "tan_half_fov": np.float32(tan), "aspect": np.float32(w / h), "w": w, "h": h}


def test_centre_ray_axis_aligned(orc):
    cam = axis_camera((-100.0, 64.0, 64.0), (1, 0, 0))
    r = orc.ray_info(cam, (128, 128, 128), 0, 0)
    np.testing.assert_array_equal(r["d"], np.array([1, 0, 0], np.float32))
    assert r["hit"] and r["t0"] == 100.0 and r["t1"] == 228.0


def test_sample_count_by_hand(orc):
    # t_k = 100 + 0.5 k < 228  <=>  k < 256: 256 samples on the way through 128 voxels
    cam = axis_camera((-100.0, 64.0, 64.0), (1, 0, 0))
    vol = orc.Volume([np.zeros((128, 128, 128), np.uint8)], "u8", 32)
    recs, n = orc.trace(vol, cam, {"step": 0.5}, 0, 0)
    assert n == 256
    assert recs["k"][-1] == 255
    t = recs["t_bits"].view(np.float32)
    np.testing.assert_array_equal(t, 100.0 + 0.5 * np.arange(256, dtype=np.float32))


def test_eye_inside_starts_at_zero(orc):
    cam = axis_camera((10.0, 5.0, 5.0), (0, 0, 1))
    r = orc.ray_info(cam, (20, 20, 20), 0, 0)
    assert r["hit"] and r["t0"] == 0.0 and r["t1"] == 15.0


def test_miss_cases(orc):
    # parallel to the x slab and outside it: no hit
    cam = axis_camera((-5.0, 30.0, 5.0), (0, 1, 0))
    assert not orc.ray_info(cam, (20, 20, 20), 0, 0)["hit"]
    # pointing away from the box
    cam = axis_camera((-5.0, 5.0, 5.0), (-1, 0, 0))
    assert not orc.ray_info(cam, (20, 20, 20), 0, 0)["hit"]
    # grazing the far face exactly: o_x = D is outside ([0, D) is half-open)
    cam = axis_camera((20.0, 5.0, -3.0), (0, 0, 1))
    assert not orc.ray_info(cam, (20, 20, 20), 0, 0)["hit"]


def _ray_numpy(cam, D, px, py):
    """Independent float32 restatement of the pixel -> ray rule (numpy scalars are binary32)."""
    f = np.float32
    u = ((f(px) + f(0.5)) / f(cam["w"])) * f(2) - f(1)
    v = f(1) - ((f(py) + f(0.5)) / f(cam["h"])) * f(2)
    cx = u * (f(cam["tan_half_fov"]) * f(cam["aspect"]))
    cy = v * f(cam["tan_half_fov"])
    d = [(f(cam["fwd"][a]) + cx * f(cam["right"][a])) + cy * f(cam["up"][a]) for a in range(3)]
    inv = f(1) / np.sqrt(f((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]))
    d = [x * inv for x in d]
    o = [f(cam["eye"][a]) for a in range(3)]
    t0, t1 = f(0), f(np.inf)
    for a in range(3):
        if d[a] == 0:
            continue
        ta = (f(0) - o[a]) / d[a]
        tb = (f(D[a]) - o[a]) / d[a]
        t0 = max(t0, min(ta, tb))
        t1 = min(t1, max(ta, tb))
    return np.array(d, np.float32), t0, t1


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rays_match_float32_restatement_and_fp64(orc, seed):
    D = (128, 96, 80)
    cam = synth.seeded_orbit(D, 37, 29, seed)
    for px, py in [(0, 0), (36, 28), (18, 14), (5, 20), (30, 3)]:
        r = orc.ray_info(cam, D, px, py)
        d, t0, t1 = _ray_numpy(cam, D, px, py)
        np.testing.assert_array_equal(r["d"], d)
        assert r["t0"] == t0 and r["t1"] == t1
        # within float32 rounding of the exact float64 direction, unit length
        u = (2 * (px + 0.5) / cam["w"] - 1) * float(cam["tan_half_fov"]) * float(cam["aspect"])
        v = (1 - 2 * (py + 0.5) / cam["h"]) * float(cam["tan_half_fov"])
        d64 = (np.float64(cam["fwd"]) + u * np.float64(cam["right"]) + v * np.float64(cam["up"]))
        d64 /= np.linalg.norm(d64)
        assert np.max(np.abs(r["d"] - d64)) < 1e-6


def test_lod_level_by_hand(orc):
    # tan = 0.5, h = 256: footprint scale (2 * 0.5) / 256 = 2^-8, so q = t / 256 exactly
    cam = axis_camera((0, 0, 0), (1, 0, 0), w=256, h=256, tan=0.5)
    L = 5
    cases = [(0.0, 0), (100.0, 0), (255.99, 0), (256.0, 0), (511.99, 0), (512.0, 1), (1023.0, 1),
             (1024.0, 2), (4096.0, 4), (1e9, 4)]
    for t, want in cases:
        assert orc.lod_level(cam, t, 0, L) == want, t
    assert orc.lod_level(cam, 512.0, 0, L, mode=0) == 0
    assert orc.lod_level(cam, 512.0, 1, L) == 2
    assert orc.lod_level(cam, 512.0, -1, L) == 0
    assert orc.lod_level(cam, 256.0, 1, L) == 1
    assert orc.lod_level(cam, 128.0, 1, L) == 0


def test_resolve_by_hand(orc):
    # ray along +x at y = 37.3, z = 2.75 through a 100 x 50 x 20 volume, bricks of 16
    D = (100, 50, 20)
    cam = axis_camera((-10.0, 37.3, 2.75), (1, 0, 0))
    vol = orc.Volume([np.zeros((20, 50, 100), np.uint8)], "u8", 16)
    recs, n = orc.trace(vol, cam, {"step": 0.5}, 0, 0)
    assert n == 200
    y = np.float32(37.3) - np.float32(0.5)            # 36.8 -> voxel 36, brick 2, local 4
    assert int(np.floor(y)) == 36
    nbx, nby = 7, 4                                    # ceil(100/16), ceil(50/16)
    for rec in recs:
        p = np.float32(-10.0) + np.float32(10.0 + 0.5 * rec["k"])   # exact
        i = int(np.floor(p - np.float32(0.5)))
        ix = min(max(i, 0), 99)
        assert tuple(rec["i0"]) == (ix, 36, 2)
        assert tuple(rec["local"]) == (ix % 16, 4, 2)
        assert rec["brick_id"] == ix // 16 + nbx * (2 + nby * 0)
        assert rec["level"] == 0


def test_resolve_coarse_level(orc):
    # level 1 of a 100^3 volume has 50 voxels per axis; ratio 0.5 exactly
    D = (100, 100, 100)
    cam = axis_camera((-10.0, 61.0, 17.0), (1, 0, 0), w=1, h=1, tan=0.5)
    lv = [np.zeros((100, 100, 100), np.uint8), np.zeros((50, 50, 50), np.uint8)]
    vol = orc.Volume(lv, "u8", 8)
    # lod_scale = 1/1 = 1 so q = t: every sample with t >= 2 is on level 1
    recs, n = orc.trace(vol, cam, {"step": 0.5, "lod_mode": 1}, 0, 0)
    assert n == 200
    for rec in recs:
        t = 10.0 + 0.5 * rec["k"]
        assert rec["level"] == (1 if t >= 2.0 else 0)
        p = -10.0 + t
        x1 = int(np.floor(np.float32(p) * np.float32(0.5) - np.float32(0.5)))
        assert rec["i0"][0] == min(max(x1, 0), 49)
        assert rec["i0"][1] == 30 and rec["i0"][2] == 8   # 61*0.5-0.5 = 30.0, 17*0.5-0.5 = 8.0
        assert rec["brick_id"] == rec["i0"][0] // 8 + 7 * (3 + 7 * 1)


def test_virtual_volume_traces_like_a_dense_one(orc):
    """The decision layer reads level dims only: a dims-only volume traces exactly like a dense
    one, so traces of volumes too large to hold are pinned by the same rules."""
    D = (40, 36, 30)
    shapes = [(30, 36, 40), (15, 18, 20), (8, 9, 10)]
    dense = orc.Volume([np.zeros(s, np.uint8) for s in shapes], "u8", 8)
    virt = orc.VirtualVolume(D, 3, "u8", 8)
    cam = dict(synth.seeded_orbit(D, 9, 7, 13, fit=0.7), h=3)
    for params in ({"lod_mode": 1, "lod_bias": -1}, {"lod_mode": 0}):
        for px, py in ((0, 0), (4, 1), (8, 2)):
            a, na = orc.trace(dense, cam, params, px, py)
            b, nb = orc.trace(virt, cam, params, px, py)
            assert na == nb
            np.testing.assert_array_equal(a, b)
    # and at coordinates no dense array could hold: a 2^20-voxel cube, level-0 brick ids past 2^32
    big = orc.VirtualVolume((1 << 20,) * 3, 7, "u8", 64)
    cam = synth.look_at((524288.0, 524300.0, 524310.0), (600000.0, 700000.0, 520000.0), 8, 6, fov_deg=50.0)
    recs, n = orc.trace(big, cam, {"lod_mode": 1, "lod_bias": 0}, 3, 2, max_samples=4000)
    assert n > 4000 and recs["brick_id"].max() > 2 ** 32
