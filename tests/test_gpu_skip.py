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
