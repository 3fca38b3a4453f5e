"""GPU parity of level-scaled sampling (VOL_RENDER_LEVEL_STEP: samples dt * 2^l apart on level l,
opacity corrected to 1 - (1 - a)^(2^l)) against the FP64 oracle.

Bit-exact: sample depths, levels, voxel and brick indices (trace records), renders after miss
passes vs fully resident.  Tolerance: 1e-4 max-abs per channel (2e-3 on reduced-precision
storage); early-termination ties as in the other parity tests."""
import numpy as np
import pytest
import torch

import synth
from _helpers import AMB, TOL_FP32, TOL_REDUCED, c1_inputs, compare, store_levels

pytestmark = pytest.mark.gpu

LEVEL_STEP = 16
PREVIEW = 8


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    assert torch.cuda.is_available()
    return volume


def gpu_volume(P, raw0, dtype, brick, levels):
    Dz, Dy, Dx = raw0.shape
    vol = P.Volume((Dx, Dy, Dz), dtype, brick, levels)
    vol.upload_level(0, raw0, dtype)
    if levels > 1:
        vol.build_lod(0)
    return vol


def tf_dev(tf):
    return torch.from_numpy(np.ascontiguousarray(tf, dtype=np.float32)).cuda()


@pytest.mark.parametrize("lod", [0, 1])
def test_trace_bit_exact(P, orc, lod):
    D, raw, cam, tf, params = c1_inputs(seed=2)
    cam = dict(cam, h=16, w=16, aspect=np.float32(1.0))
    params = dict(params, lod_mode=lod, lod_bias=-2 if lod else 0, flags=LEVEL_STEP)   # levels 1 and 2
    vol = gpu_volume(P, raw, "u8", 32, 3)
    pix = synth.pixel_subset(16, 16, 120, 7)
    recs, counts = vol.trace(cam, params, pix, 800)
    ovol = orc.Volume(store_levels(orc, raw, "u8", "u8", 3), "u8", 32)
    levels = set()
    for i, (px, py) in enumerate(pix):
        want, n = orc.trace(ovol, cam, params, int(px), int(py), 800)
        assert counts[i] == n
        got = recs[i, :min(n, 800)]
        for f in ("k", "t_bits", "level", "i0", "local", "brick_id"):
            np.testing.assert_array_equal(got[f], want[f], err_msg=f"pixel {(px, py)} field {f}")
        levels.update(int(l) for l in got["level"])
    if lod:
        assert len(levels) >= 2


@pytest.mark.parametrize("lod", [0, 1])
def test_c1_frame_vs_oracle(P, orc, lod):
    D, raw, cam, tf, params = c1_inputs()
    # a small footprint scale so that the footprint LOD spans levels 0..2 over the frame
    cam = dict(cam, h=64, w=64)
    params = dict(params, lod_mode=lod, lod_bias=-1 if lod else 0, flags=LEVEL_STEP)
    vol = gpu_volume(P, raw, "u8", 32, 3)
    out, ns = vol.render(cam, tf_dev(tf), params, nsamples=True)
    gpu = out.cpu().numpy()
    ovol = orc.Volume(store_levels(orc, raw, "u8", "u8", 3), "u8", 32)
    ref = orc.render(ovol, cam, tf, params, amb=AMB)
    err, bad, alt = compare(gpu, ref, TOL_FP32)
    assert len(bad) == 0, (err, len(bad))
    n = ns.cpu().numpy()
    assert np.all((n == ref["n"]) | (alt & (n == ref["alt_n"])))
    if lod:
        plain = vol.render(cam, tf_dev(tf), dict(params, flags=0), nsamples=True)[1].cpu().numpy()
        assert n.sum() < plain.sum()   # coarse levels take longer steps


@pytest.mark.parametrize("store", ["u16", "f16"])
def test_reduced_precision_lod(P, orc, store):
    D = (160, 144, 128)
    raw16 = synth.noise_spheres(D, 7, octaves=5, period0=64.0, nspheres=30, radius=(4.0, 30.0), value=(0.3, 1.0))
    levels = store_levels(orc, raw16, "u16", store, 4)
    vol = P.Volume(D, store, 32, 4)
    vol.upload_level(0, levels[0], store)
    vol.build_lod(0)
    tf = synth.tf_peaks(7)
    cam = synth.seeded_orbit(D, 96, 72, 7, view=2)
    params = {"lod_mode": 1, "lod_bias": 0, "flags": LEVEL_STEP}
    gpu = vol.render(cam, tf_dev(tf), params).cpu().numpy()
    ref = orc.render(orc.Volume(levels, store, 32), cam, tf, params, amb=AMB)
    err, bad, _ = compare(gpu, ref, TOL_REDUCED)
    assert len(bad) == 0, (err, len(bad))


def test_miss_path_and_preview(P, orc):
    """Bricks loaded on request (rays suspended with their sample depth) give the resident
    image bit for bit; a preview under level-scaled sampling matches the oracle's."""
    D, raw, cam, tf, params = c1_inputs(seed=5)
    params = dict(params, lod_mode=1, lod_bias=0, flags=LEVEL_STEP)
    B = 16
    levels = store_levels(orc, raw, "u8", "u8", 3)
    full = gpu_volume(P, raw, "u8", B, 3)
    want = full.render(cam, tf_dev(tf), params).cpu().numpy()

    def brick(level, b):
        arr = levels[level]
        Dz, Dy, Dx = arr.shape
        zi = np.minimum(b[2] * B + np.arange(B + 1), Dz - 1)
        yi = np.minimum(b[1] * B + np.arange(B + 1), Dy - 1)
        xi = np.minimum(b[0] * B + np.arange(B + 1), Dx - 1)
        return arr[np.ix_(zi, yi, xi)]

    slot = P.plan(D, "u8", B, 3).slot_bytes
    vol = P.Volume(D, "u8", B, 3, cache_bytes=300 * slot)
    vol.set_provider(brick, "u8")
    got = vol.render(cam, tf_dev(tf), dict(params, max_passes=400)).cpu().numpy()
    assert vol.stats()["passes"] > 1
    np.testing.assert_array_equal(got, want)

    # preview: only the two coarser levels resident
    pv = P.Volume(D, "u8", B, 3)
    ovol = orc.Volume(levels, "u8", B)
    res = np.zeros(orc.page_table_size(ovol), np.uint8)
    off = 0
    for l, arr in enumerate(levels):
        Dz, Dy, Dx = arr.shape
        nb = [-(-Dx // B), -(-Dy // B), -(-Dz // B)]
        if l > 0:
            for bz in range(nb[2]):
                for by in range(nb[1]):
                    for bx in range(nb[0]):
                        pv.upload_brick(l, (bx, by, bz), brick(l, (bx, by, bz)), "u8")
                        res[off + bx + nb[0] * (by + nb[1] * bz)] = 1
        off += nb[0] * nb[1] * nb[2]
    pparams = dict(params, flags=LEVEL_STEP | PREVIEW)
    gpu = pv.render(cam, tf_dev(tf), pparams).cpu().numpy()
    assert pv.stats()["preview_samples"] > 0
    ref = orc.render_preview(ovol, cam, tf, pparams, res, amb=AMB)
    err, bad, _ = compare(gpu, ref, TOL_FP32)
    assert len(bad) == 0, (err, len(bad))


def test_rejected_combinations(P):
    D, raw, cam, tf, params = c1_inputs()
    vol = gpu_volume(P, raw, "u8", 32, 2)
    with pytest.raises(RuntimeError):
        vol.render(cam, tf_dev(tf), dict(params, flags=LEVEL_STEP), grad=True)
    with pytest.raises(RuntimeError):
        vol.render(cam, tf_dev(tf), dict(params, flags=LEVEL_STEP, composite="mop"))
