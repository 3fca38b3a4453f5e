"""Empty-space skipping (the paper's empty-brick skipping): bricks whose value range the
transfer function maps to zero opacity are jumped over.  Those samples composite nothing, so
the image and the per-pixel sample counts must be bit-identical with and without it, for every
storage type, layout, LOD mode, gradient mode and the out-of-core path."""
import numpy as np
import pytest
import torch

import synth
from _helpers import AMB, TOL_FP32, c1_inputs, compare, store_levels

pytestmark = pytest.mark.gpu

SKIP = 2  # VOL_RENDER_SKIP_EMPTY


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    return volume


def both(vol, cams, tf, params, grad=False):
    a, na = vol.render(cams, tf, dict(params), nsamples=True, grad=grad)
    a, na = a.clone(), na.clone()
    b, nb = vol.render(cams, tf, dict(params, flags=SKIP), nsamples=True, grad=grad)
    torch.cuda.synchronize()
    return a.cpu().numpy(), na.cpu().numpy(), b.cpu().numpy(), nb.cpu().numpy()


@pytest.mark.parametrize("dtype,layout,lod", [("u8", "quad", 0), ("u8", "compact", 1), ("u16", "quad", 1),
                                              ("f16", "compact", 0), ("f32", "quad", 0)])
def test_skip_is_exact(P, orc, dtype, layout, lod):
    D = (130, 97, 111)
    base = synth.blobs(D, 31, dtype="f32", nblobs=9, sigma=(5, 14), amp=(0.3, 1.0), noise=0.02, vmax=1.0)
    raw = {"u8": (base * 255).astype(np.uint8), "u16": (base * 65535).astype(np.uint16),
           "f16": base.astype(np.float16).view(np.uint16), "f32": base}[dtype]
    vol = P.Volume(D, dtype, 16, 3, layout=layout)
    vol.upload_level(0, raw, dtype)
    vol.build_lod(0)
    tf = synth.tf_ramp(alpha_start=0.15, alpha_max=0.2)
    tfd = torch.from_numpy(tf).cuda()
    cams = [synth.seeded_orbit(D, 96, 80, 31, view=v) for v in range(3)] + \
           [synth.look_at((60.0, 40.0, 50.0), (100.0, 80.0, 70.0), 64, 48, fov_deg=70.0)]
    params = {"lod_mode": lod, "lod_bias": 1 if lod else 0}
    a, na, b, nb = both(vol, cams, tfd, params)
    np.testing.assert_array_equal(b, a)
    np.testing.assert_array_equal(nb, na)
    # and it is still the oracle's image
    ovol = orc.Volume(store_levels(orc, raw, dtype, dtype, 3), dtype, 16)
    off = 0
    for cam in cams[:2]:
        n = cam["w"] * cam["h"]
        ref = orc.render(ovol, cam, tf, params, amb=AMB)
        err, bad, _ = compare(b[off:off + n], ref, TOL_FP32)
        assert len(bad) == 0, err
        off += n


def test_skip_keeps_gradient_checkpoints(P):
    D = (96, 96, 96)
    raw = synth.blobs(D, 32, dtype="f32", nblobs=5, sigma=(6, 12), amp=(0.3, 1.0), noise=0.0, vmax=1.0)
    vol = P.Volume(D, "f32", 32, 1)
    vol.upload_level(0, raw, "f32")
    tf = synth.tf_ramp(alpha_start=0.2, alpha_max=0.1)
    tfd = torch.from_numpy(tf).cuda()
    cams = [synth.seeded_orbit(D, 64, 64, 32, view=v) for v in range(2)]
    grads = []
    for flags in (0, SKIP):
        img = vol.render(cams, tfd, {"flags": flags}, grad=True)
        dI = torch.from_numpy(np.random.default_rng(1).standard_normal((img.shape[0], 4)).astype(np.float32)).cuda()
        dtf = torch.zeros((256, 4), device="cuda")
        dvox = torch.zeros(raw.shape, device="cuda")
        vol.render_backward(dI, dtf, dvox)
        torch.cuda.synchronize()
        grads.append((img.cpu().numpy(), dtf.cpu().numpy(), dvox.cpu().numpy()))
    np.testing.assert_array_equal(grads[0][0], grads[1][0])
    for g0, g1 in zip(grads[0][1:], grads[1][1:]):
        assert np.abs(g0 - g1).max() <= 1e-5 * np.abs(g0).max() + 1e-9


def test_skip_with_bricks_on_demand(P):
    D, B, L, seed = (256, 256, 256), 32, 4, 9
    gen = dict(octaves=5, period0=64.0, nspheres=40, radius=(4.0, 30.0), value=(0.3, 1.0))
    tf = synth.tf_peaks(seed)
    tfd = torch.from_numpy(tf).cuda()
    cams = synth.flythrough(D, 160, 90, 3, seed)
    imgs = []
    for flags in (0, SKIP):
        slot = P.plan(D, "u8", B, L, layout="compact").slot_bytes
        vol = P.Volume(D, "u8", B, L, cache_bytes=150 * slot, layout="compact")
        src = synth.brick_source(D, B, L, seed, dtype="u8", **gen)
        vol.set_provider_batch(synth.brick_provider_address(), src, "u8")
        imgs.append([vol.render(c, tfd, {"lod_mode": 1, "max_passes": 2000, "flags": flags}).cpu().numpy()
                     for c in cams])
        vol.close()
    for a, b in zip(*imgs):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("store,brick,layout", [("u16", 64, "quad"), ("f16", 32, "compact"), ("u8", 32, "quad"),
                                               ("f32", 64, "compact"), ("u8", 8, "compact"), ("u16", 16, "compact")])
def test_macro_cell_skip_is_exact(P, orc, store, brick, layout):
    """Noise + spheres under a TF of narrow opacity peaks: no large brick is empty, but many
    8^3-voxel cells are (8, 4 or 2 per brick axis; an 8^3 brick is one cell).  Images and sample
    counts are bit-identical with the skipping, which jumps over a measured share of the samples;
    MOP and MIP likewise; and the image is the oracle's."""
    D = (200, 176, 160)
    raw16 = synth.noise_spheres(D, 21, octaves=5, period0=48.0, nspheres=30, radius=(4.0, 30.0), value=(0.3, 1.0))
    src = "u16" if store in ("u16", "f16", "f32") else "u8"
    raw = raw16 if src == "u16" else (raw16 >> 8).astype(np.uint8)
    vol = P.Volume(D, store, brick, 3, layout=layout)
    vol.upload_level(0, raw, src)
    vol.build_lod(0)
    tf = synth.tf_peaks(21)
    tfd = torch.from_numpy(tf).cuda()
    cams = [synth.seeded_orbit(D, 120, 90, 21, view=v) for v in range(2)] + \
           [synth.look_at((90.0, 70.0, 60.0), (150.0, 120.0, 110.0), 80, 60, fov_deg=70.0)]
    params = {"lod_mode": 1}
    a, na, b, nb = both(vol, cams, tfd, params)
    skipped = vol.stats()["skipped_samples"]
    np.testing.assert_array_equal(b, a)
    np.testing.assert_array_equal(nb, na)
    assert skipped > 0.05 * na.sum(), (skipped, na.sum())
    for mode in ("mop", "mip"):
        pm = dict(params, composite=mode)
        a2, na2, b2, nb2 = both(vol, cams, tfd, pm)
        np.testing.assert_array_equal(b2, a2)
        np.testing.assert_array_equal(nb2, na2)
    ovol = orc.Volume(store_levels(orc, raw, src, store, 3), store, brick)
    ref = orc.render(ovol, cams[0], tf, params, amb=AMB)
    n0 = cams[0]["w"] * cams[0]["h"]
    err, bad, _ = compare(b[:n0], ref, 2e-3 if store in ("u16", "f16") else TOL_FP32)
    assert len(bad) == 0, err
    assert np.all((nb[:n0] == ref["n"]) | (ref["amb"] & (nb[:n0] == ref["alt_n"])))


def test_skip_counts_add_up(P):
    """Composited plus jumped-over samples: every sample a ray passes, with and without skipping."""
    D = (128, 128, 128)
    raw = synth.noise_spheres(D, 5, octaves=4, period0=32.0, nspheres=10, radius=(4.0, 20.0), value=(0.3, 1.0))
    vol = P.Volume(D, "u16", 32, 1)
    vol.upload_level(0, raw, "u16")
    tf = synth.tf_peaks(5)
    tfd = torch.from_numpy(tf).cuda()
    cam = synth.seeded_orbit(D, 128, 128, 5)
    # MIP visits samples to the exit (or to the largest coordinate): many fall in cells below
    # the kept coordinate
    _, n_all = vol.render(cam, tfd, {"composite": "mip"}, nsamples=True)
    _, n_skip = vol.render(cam, tfd, {"composite": "mip", "flags": SKIP}, nsamples=True)
    torch.cuda.synchronize()
    st = vol.stats()
    np.testing.assert_array_equal(n_all.cpu().numpy(), n_skip.cpu().numpy())
    assert 0 < st["skipped_samples"] < int(n_all.sum().item())
