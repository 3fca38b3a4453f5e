"""GPU parity of the maximum projections (MOP, the compositing of the paper's Kidney renderings,
Sec. V-A; and MIP) through the C ABI against the FP64 oracle on the same seeded inputs.

Tolerance: max-abs per channel 1e-4 (float32 arithmetic), 2e-3 on reduced-precision storage.  MOP
keeps the first sample of largest opacity, a decision that float32 and float64 opacities can take
differently when two samples lie within rounding of each other: there the output alpha must still
match and each colour channel lie within the range of the near-maximal samples' outputs, which
the oracle reports (lo, hi).  Bit-exact: empty-space skipping, batching, the miss path."""
import numpy as np
import pytest
import torch

import synth
from _helpers import TOL_FP32, TOL_REDUCED, c1_inputs, store_levels
from _helpers import compare_projection as check

pytestmark = pytest.mark.gpu

SKIP = 2  # VOL_RENDER_SKIP_EMPTY
AMB_MOP = 1e-5


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    assert torch.cuda.is_available()
    return volume


def gpu_volume(P, raw0, dtype, brick, levels, cache_bytes=0, layout="quad"):
    Dz, Dy, Dx = raw0.shape
    vol = P.Volume((Dx, Dy, Dz), dtype, brick, levels, cache_bytes, layout=layout)
    vol.upload_level(0, raw0, dtype)
    if levels > 1:
        vol.build_lod(0)
    return vol


def tf_dev(tf):
    return torch.from_numpy(np.ascontiguousarray(tf, dtype=np.float32)).cuda()


def tf_for(kind, seed):
    if kind == "ramp":
        return synth.tf_ramp(alpha_start=0.1, alpha_max=0.08)
    tf = synth.tf_peaks(seed)
    tf[:, 3] = np.clip(tf[:, 3] + 0.01, 0, 1)
    return tf


@pytest.mark.parametrize("mode", ["mop", "mip"])
@pytest.mark.parametrize("lod", [0, 1])
@pytest.mark.parametrize("tfk", ["ramp", "peaks"])
def test_c1_projection_vs_oracle(P, orc, mode, lod, tfk):
    D, raw, cam, _, params = c1_inputs()
    tf = tf_for(tfk, 3)
    params = dict(params, lod_mode=lod, composite=mode, bg=(0.1, 0.2, 0.0, 0.25))
    vol = gpu_volume(P, raw, "u8", 32, 2)
    out, ns = vol.render(cam, tf_dev(tf), params, nsamples=True)
    torch.cuda.synchronize()
    gpu = out.cpu().numpy()
    ovol = orc.Volume(store_levels(orc, raw, "u8", "u8", 2), "u8", 32)
    ref = orc.render_max(ovol, cam, tf, params, mode, amb=AMB_MOP)
    err, bad, near = check(gpu, ref, TOL_FP32)
    assert len(bad) == 0, f"{len(bad)} pixels above {TOL_FP32}, max err {err}"
    # a ray stops early only where nothing later can be kept; never past its last sample
    n_gpu = ns.cpu().numpy()
    assert np.all(n_gpu <= ref["n"])
    assert vol.stats()["device_error"] == 0
    print(f"{mode} lod={lod} tf={tfk}: max err {err:.3g}, near-tied pixels {near}, "
          f"samples {int(n_gpu.sum())} of {int(ref['n'].sum())}")


@pytest.mark.parametrize("mode", ["mop", "mip"])
@pytest.mark.parametrize("store", ["u16", "f16"])
def test_reduced_precision_lod(P, orc, mode, store):
    """Noise + spheres in u16, stored as u16 or binary16, 4 levels, footprint LOD."""
    D = (160, 144, 128)
    raw16 = synth.noise_spheres(D, 7, octaves=5, period0=64.0, nspheres=30, radius=(4.0, 30.0),
                                value=(0.3, 1.0))
    levels = store_levels(orc, raw16, "u16", store, 4)
    vol = P.Volume(D, store, 32, 4)
    vol.upload_level(0, levels[0], store)
    vol.build_lod(0)
    tf = synth.tf_peaks(7)
    cam = synth.seeded_orbit(D, 160, 120, 7, view=2)
    params = {"lod_mode": 1, "lod_bias": 0, "composite": mode}
    gpu = vol.render(cam, tf_dev(tf), params).cpu().numpy()
    ref = orc.render_max(orc.Volume(levels, store, 32), cam, tf, params, mode, amb=AMB_MOP)
    err, bad, near = check(gpu, ref, TOL_REDUCED)
    assert len(bad) == 0, (err, len(bad))
    print(f"{mode} {store}: max err {err:.3g}, near-tied pixels {near}")


@pytest.mark.parametrize("dtype", ["u8", "u16", "f16", "f32"])
def test_ragged_volume_all_types(P, orc, dtype):
    """Odd dims, bricks of 8, values outside [0, 1] for the float types (the TF clamp), a camera
    inside the volume and one outside, both modes."""
    D = (37, 29, 23)
    rng = np.random.default_rng(21)
    if dtype == "u8":
        raw = rng.integers(0, 256, (23, 29, 37), dtype=np.uint8)
    elif dtype == "u16":
        raw = rng.integers(0, 65536, (23, 29, 37), dtype=np.uint16)
    elif dtype == "f16":
        raw = (rng.random((23, 29, 37)) * 1.4 - 0.2).astype(np.float16).view(np.uint16)
    else:
        raw = (rng.random((23, 29, 37), dtype=np.float32) * np.float32(1.4) - np.float32(0.2))
    vol = gpu_volume(P, raw, dtype, 8, 3)
    ovol = orc.Volume(store_levels(orc, raw, dtype, dtype, 3), dtype, 8)
    tf = synth.tf_peaks(4)
    ramp = np.arange(256, dtype=np.float32) / 255
    tf[:, 3] = np.clip(tf[:, 3] + 0.1 * ramp, 0, 1)
    tf[:, 0] = ramp
    cams = [synth.look_at((18.0, 14.0, 11.0), (30.0, 20.0, 15.0), 45, 33, fov_deg=70.0),
            synth.seeded_orbit(D, 41, 31, 8)]
    for mode in ("mop", "mip"):
        for cam in cams:
            for lod in (0, 1):
                params = {"lod_mode": lod, "lod_bias": 2 if lod else 0, "bg": (0.1, 0.0, 0.2, 0.5),
                          "composite": mode}
                gpu = vol.render(cam, tf_dev(tf), params).cpu().numpy()
                ref = orc.render_max(ovol, cam, tf, params, mode, amb=AMB_MOP)
                err, bad, _ = check(gpu, ref, TOL_FP32)
                assert len(bad) == 0, (mode, lod, err)


@pytest.mark.parametrize("mode", ["mop", "mip"])
@pytest.mark.parametrize("dtype,layout,lod", [("u8", "quad", 0), ("u16", "compact", 1), ("f16", "quad", 1),
                                              ("f32", "quad", 0)])
def test_skip_is_exact(P, orc, mode, dtype, layout, lod):
    D = (130, 97, 111)
    base = synth.blobs(D, 31, dtype="f32", nblobs=9, sigma=(5, 14), amp=(0.3, 1.0), noise=0.02, vmax=1.0)
    raw = {"u8": (base * 255).astype(np.uint8), "u16": (base * 65535).astype(np.uint16),
           "f16": base.astype(np.float16).view(np.uint16), "f32": base}[dtype]
    vol = P.Volume(D, dtype, 16, 3, layout=layout)
    vol.upload_level(0, raw, dtype)
    vol.build_lod(0)
    tf = synth.tf_peaks(31)
    tfd = tf_dev(tf)
    cams = [synth.seeded_orbit(D, 96, 80, 31, view=v) for v in range(3)] + \
           [synth.look_at((60.0, 40.0, 50.0), (100.0, 80.0, 70.0), 64, 48, fov_deg=70.0)]
    params = {"lod_mode": lod, "lod_bias": 1 if lod else 0, "composite": mode}
    a, na = vol.render(cams, tfd, params, nsamples=True)
    a, na = a.clone(), na.clone()
    b, nb = vol.render(cams, tfd, dict(params, flags=SKIP), nsamples=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(b.cpu().numpy(), a.cpu().numpy())
    np.testing.assert_array_equal(nb.cpu().numpy(), na.cpu().numpy())
    ovol = orc.Volume(store_levels(orc, raw, dtype, dtype, 3), dtype, 16)
    cam = cams[0]
    ref = orc.render_max(ovol, cam, tf, params, mode, amb=AMB_MOP)
    err, bad, _ = check(b.cpu().numpy()[:cam["w"] * cam["h"]], ref, TOL_FP32)
    assert len(bad) == 0, err


@pytest.mark.parametrize("mode", ["mop", "mip"])
def test_batched_and_miss_path_equal_resident(P, orc, mode):
    """Several views in one launch equal single-view renders; a cache holding half of the
    bricks, filled on request through the provider, gives the resident image bit for bit."""
    D, raw, _, tf, params = c1_inputs(seed=5)
    tf = tf_for("peaks", 5)
    params = dict(params, lod_mode=1, composite=mode)
    levels = store_levels(orc, raw, "u8", "u8", 2)
    B = 16
    full = gpu_volume(P, raw, "u8", B, 2)
    cams = [synth.seeded_orbit(D, s, s, 5, view=i) for i, s in enumerate([96, 17, 64, 40])]
    want = full.render(cams, tf_dev(tf), params).cpu().numpy()
    off = 0
    for cam in cams:
        n = cam["w"] * cam["h"]
        np.testing.assert_array_equal(full.render(cam, tf_dev(tf), params).cpu().numpy(), want[off:off + n])
        off += n

    def provider(level, b):
        arr = levels[level]
        Dz, Dy, Dx = arr.shape
        zi = np.minimum(b[2] * B + np.arange(B + 1), Dz - 1)
        yi = np.minimum(b[1] * B + np.arange(B + 1), Dy - 1)
        xi = np.minimum(b[0] * B + np.arange(B + 1), Dx - 1)
        return arr[np.ix_(zi, yi, xi)]

    slot = P.plan(D, "u8", B, 2).slot_bytes
    vol = P.Volume(D, "u8", B, 2, cache_bytes=300 * slot)   # 300 of 584 bricks
    vol.set_provider(provider, "u8")
    for flags in (0, SKIP):
        got = vol.render(cams, tf_dev(tf), dict(params, max_passes=400, flags=flags)).cpu().numpy()
        st = vol.stats()
        assert st["device_error"] == 0
        if flags == 0:   # the first frame starts from an empty cache; the second may find it warm
            assert st["passes"] > 1 and st["bricks_loaded"] > 0
        np.testing.assert_array_equal(got, want)


def test_projection_arguments(P):
    D, raw, cam, tf, params = c1_inputs()
    vol = gpu_volume(P, raw, "u8", 32, 1)
    with pytest.raises(RuntimeError):
        vol.render(cam, tf_dev(tf), dict(params, composite="mop"), grad=True)
    with pytest.raises(RuntimeError):
        vol.render(cam, tf_dev(tf), dict(params, composite=3))
    # transparent TF: the background in both modes, exactly
    tf0 = tf.copy(); tf0[:, 3] = 0
    bg = (0.25, 0.5, 0.125, 1.0)
    for mode in ("mop", "mip"):
        out = vol.render(cam, tf_dev(tf0), dict(params, composite=mode, bg=bg)).cpu().numpy()
        np.testing.assert_array_equal(out, np.tile(np.float32(bg), (cam["w"] * cam["h"], 1)))
