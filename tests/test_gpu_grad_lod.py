"""GPU adjoint with footprint LOD: samples on coarser levels send their voxel gradient down the
pyramid through the box filter's adjoint.  Compared with the FP64 oracle's gradient (same
tolerance as the level-0 adjoint: max |g_gpu - g_oracle| <= 1e-4 max |g_oracle| + 1e-7, cosine
>= 1 - 1e-6), and through the autograd function, whose density gradient must match."""
import numpy as np
import pytest
import torch

import synth
from _helpers import AMB, TOL_FP32, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    return volume


def grad_close(g, ref, what):
    scale = float(np.abs(ref).max())
    err = float(np.abs(g - ref).max())
    assert err <= 1e-4 * scale + 1e-7, f"{what}: max err {err:.3g} vs scale {scale:.3g}"
    cos = float(np.sum(g * ref) / (np.linalg.norm(g) * np.linalg.norm(ref) + 1e-300))
    assert cos >= 1 - 1e-6, f"{what}: cosine {cos}"
    return err / max(scale, 1e-300)


def case():
    D = (64, 56, 48)
    raw = synth.blobs(D, 9, dtype="f32", nblobs=7, sigma=(4, 10), amp=(0.2, 1.0), noise=0.03, vmax=0.9)
    # eyes just outside the box and a coarse image: the footprint spans levels 0..2 along a ray
    cams = [synth.look_at((-3.0, 28.0, 24.0), (70.0, 29.0, 25.0), 48, 12, fov_deg=60.0),
            synth.look_at((32.0, -3.0, 20.0), (31.0, 60.0, 26.0), 40, 10, fov_deg=60.0)]
    tf = synth.tf_peaks(12)
    tf[:, 3] = np.clip(tf[:, 3] + 0.03, 0, 1)
    params = {"step": 0.5, "et": 0.99, "bg": (0.1, 0.2, 0.3, 0.4), "lod_mode": 1, "lod_bias": 0}
    return D, raw, cams, tf, params


@pytest.mark.parametrize("skip", [0, 2])
def test_lod_gradients_match_oracle(P, orc, skip):
    D, raw, cams, tf, params = case()
    params = dict(params, flags=skip)
    L = 3
    vol = P.Volume(D, "f32", 16, L)
    vol.upload_level(0, raw, "f32")
    vol.build_lod(0)
    tfd = torch.from_numpy(tf).cuda()
    img = vol.render(cams, tfd, params, grad=True).cpu().numpy()
    rng = np.random.default_rng(4)
    dI = (rng.standard_normal((img.shape[0], 4)) * 0.1).astype(np.float32)
    dtf = torch.zeros((256, 4), device="cuda")
    dvox = torch.zeros(raw.shape, device="cuda")
    vol.render_backward(torch.from_numpy(dI).cuda(), dtf, dvox)
    torch.cuda.synchronize()
    assert vol.stats()["device_error"] == 0
    ovol = orc.Volume(orc.pyramid(raw, L, "f32"), "f32", 16)
    odtf, odvox = np.zeros((256, 4)), np.zeros(raw.shape)
    off, levels = 0, set()
    for cam in cams:
        n = cam["w"] * cam["h"]
        ref = orc.render(ovol, cam, tf, params, amb=AMB)
        err, bad, use_alt = compare(img[off:off + n], ref, TOL_FP32)
        assert len(bad) == 0, err
        g1, g2 = orc.render_grad(ovol, cam, tf, params, dI[off:off + n].astype(np.float64),
                                 alt_select=use_alt.astype(np.int32), amb=AMB)
        odtf += g1
        odvox += g2
        for px in range(0, cam["w"], 4):
            recs, _ = orc.trace(ovol, cam, params, px, cam["h"] // 2)
            levels.update(int(l) for l in recs["level"])
        off += n
    assert levels >= {0, 1, 2}
    r1 = grad_close(dtf.cpu().numpy(), odtf, "dtf")
    r2 = grad_close(dvox.cpu().numpy(), odvox, "dvoxel")
    print(f"LOD grad: rel err dtf {r1:.2e} dvoxel {r2:.2e}")


def test_autograd_through_lod(P, orc):
    D, raw, cams, tf, params = case()
    vol = P.Volume(D, "f32", 16, 3)
    density = torch.from_numpy(raw).cuda().requires_grad_(True)
    tfd = torch.from_numpy(tf).cuda().requires_grad_(True)
    img = P.RaycastFn.apply(density, tfd, vol, cams, params)
    w = torch.from_numpy(np.random.default_rng(6).standard_normal(tuple(img.shape)).astype(np.float32)).cuda()
    (img * w).sum().backward()
    ovol = orc.Volume(orc.pyramid(raw, 3, "f32"), "f32", 16)
    odvox = np.zeros(raw.shape)
    off = 0
    wn = w.cpu().numpy().astype(np.float64)
    gimg = img.detach().cpu().numpy()
    for cam in cams:
        n = cam["w"] * cam["h"]
        ref = orc.render(ovol, cam, tf, params, amb=AMB)
        _, bad, use_alt = compare(gimg[off:off + n], ref, TOL_FP32)
        assert len(bad) == 0
        odvox += orc.render_grad(ovol, cam, tf, params, wn[off:off + n], alt_select=use_alt.astype(np.int32),
                                 amb=AMB)[1]
        off += n
    grad_close(density.grad.cpu().numpy(), odvox, "autograd dvoxel")
