"""GPU adjoint parity: dL/dtf and dL/dvoxel from the CUDA adjoint (checkpointed transmittance
recompute) against the FP64 oracle's exact gradient, and against central finite differences of
the FP64 oracle (h = 1e-3) on 64 seeded coordinates.

The upstream gradient dL/dI is a seeded synthetic array: the adjoint is linear in it, so any
fixed dL/dI tests the whole vector-Jacobian product, and nothing the oracle receives comes from
the GPU path.  Where float32 and float64 take a different early-termination decision (within
rounding of the threshold) the oracle's alternate result is selected for that pixel.

Gradient tolerance (derived from float32 accumulation over <= 1000 samples per ray and
order-free atomics): max |g_gpu - g_oracle| <= 1e-4 * max |g_oracle| + 1e-7 per tensor, and
cosine similarity >= 1 - 1e-6.
"""
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


def run_case(P, orc, raw, cams, tf, params, dI_seed, pixel_mask=None):
    D = raw.shape[::-1]
    vol = P.Volume(D, "f32", 16 if max(D) < 128 else 32, 1)
    vol.upload_level(0, raw, "f32")
    tfd = torch.from_numpy(tf).cuda()
    img = vol.render(cams, tfd, params, grad=True)
    npx = img.shape[0]
    rng = np.random.default_rng(dI_seed)
    dI = rng.standard_normal((npx, 4)).astype(np.float32) * np.float32(0.1)
    if pixel_mask is not None:
        dI[~pixel_mask] = 0
    dtf = torch.zeros((256, 4), dtype=torch.float32, device="cuda")
    dvox = torch.zeros(raw.shape, dtype=torch.float32, device="cuda")
    vol.render_backward(torch.from_numpy(dI).cuda(), dtf, dvox)
    torch.cuda.synchronize()
    assert vol.stats()["device_error"] == 0
    gimg = img.cpu().numpy()
    ovol = orc.Volume([raw], "f32", 16)
    odtf, odvox = np.zeros((256, 4)), np.zeros(raw.shape)
    off = 0
    for cam in cams:
        n = cam["w"] * cam["h"]
        sel = np.arange(n) if pixel_mask is None else np.flatnonzero(pixel_mask[off:off + n])
        pix = np.stack([sel % cam["w"], sel // cam["w"]], 1).astype(np.int32)
        if len(pix):
            ref = orc.render(ovol, cam, tf, params, pixels=pix, amb=AMB)
            err, bad, use_alt = compare(gimg[off + sel], ref, TOL_FP32)
            assert len(bad) == 0, err
            g1, g2 = orc.render_grad(ovol, cam, tf, params, dI[off + sel].astype(np.float64), pixels=pix,
                                     alt_select=use_alt.astype(np.int32), amb=AMB)
            odtf += g1
            odvox += g2
        off += n
    return vol, dtf.cpu().numpy(), dvox.cpu().numpy(), odtf, odvox, dI


def small_case():
    D = (40, 36, 32)
    raw = synth.blobs(D, 5, dtype="f32", nblobs=6, sigma=(4, 9), amp=(0.2, 1.0), noise=0.03, vmax=0.95)
    cams = [synth.seeded_orbit(D, 48, 40, 5, view=v) for v in range(2)]
    tf = synth.tf_peaks(8)
    tf[:, 3] = np.clip(tf[:, 3] + 0.03, 0, 1)
    return D, raw, cams, tf, {"step": 0.5, "et": 0.99, "bg": (0.1, 0.2, 0.3, 0.4)}


def test_small_gradients_match_oracle(P, orc):
    D, raw, cams, tf, params = small_case()
    _, dtf, dvox, odtf, odvox, _ = run_case(P, orc, raw, cams, tf, params, 1)
    r1 = grad_close(dtf, odtf, "dtf")
    r2 = grad_close(dvox, odvox, "dvoxel")
    print(f"small grad: rel err dtf {r1:.2e} dvoxel {r2:.2e}")


def test_small_gradients_match_central_differences(P, orc):
    """FD of the FP64 oracle's L = sum(dI * I) at 32 TF and 32 voxel coordinates (h = 1e-3)."""
    D, raw, cams, tf, params = small_case()
    j = np.arange(256) / 255.0
    tf = np.stack([0.2 + 0.6 * j, 0.9 - 0.5 * j, 0.3 + 0.2 * j, 0.02 + 0.25 * j], 1).astype(np.float32)
    _, dtf, dvox, _, _, dI = run_case(P, orc, raw, cams, tf, params, 2)
    ovol = orc.Volume([raw], "f32", 16)

    def L(vol_, tf_):
        tot, ns = 0.0, []
        off = 0
        for cam in cams:
            n = cam["w"] * cam["h"]
            out = orc.render(vol_, cam, tf_, params)
            tot += float(np.sum(dI[off:off + n].astype(np.float64) * out["rgba"]))
            ns.append(out["n"])
            off += n
        return tot, np.concatenate(ns)

    _, n0 = L(ovol, tf)
    rng = np.random.default_rng(3)
    h = 1e-3
    checked = 0
    used = np.flatnonzero(np.abs(dtf).sum(1) > 1e-3 * np.abs(dtf).max())
    for _ in range(32):
        jj, ch = int(rng.choice(used)), int(rng.integers(0, 4))
        tp, tm = tf.copy(), tf.copy()
        tp[jj, ch] += h; tm[jj, ch] -= h
        (Lp, np_), (Lm, nm) = L(ovol, tp), L(ovol, tm)
        if not (np.array_equal(np_, n0) and np.array_equal(nm, n0)):
            continue
        fd = (Lp - Lm) / (float(tp[jj, ch]) - float(tm[jj, ch]))
        assert abs(dtf[jj, ch] - fd) <= 1e-3 * abs(fd) + 1e-5 * np.abs(dtf).max(), (jj, ch, dtf[jj, ch], fd)
        checked += 1
    cand = np.argwhere(np.abs(dvox) > 1e-2 * np.abs(dvox).max())
    for _ in range(32):
        z, y, x = cand[int(rng.integers(0, len(cand)))]
        rp, rm = raw.copy(), raw.copy()
        rp[z, y, x] += np.float32(h); rm[z, y, x] -= np.float32(h)
        (Lp, np_), (Lm, nm) = L(orc.Volume([rp], "f32", 16), tf), L(orc.Volume([rm], "f32", 16), tf)
        if not (np.array_equal(np_, n0) and np.array_equal(nm, n0)):
            continue
        fd = (Lp - Lm) / (float(rp[z, y, x]) - float(rm[z, y, x]))
        assert abs(dvox[z, y, x] - fd) <= 1e-3 * abs(fd) + 1e-5 * np.abs(dvox).max(), ((z, y, x), dvox[z, y, x], fd)
        checked += 1
    assert checked >= 48


def test_full_size_differentiable_workload_sampled(P, orc):
    """256^3 f32 blobs, 16 views at 512x512, checkpoints every 32 samples: the forward and adjoint
    run at full size in the benchmark's launch configuration; dL/dI is non-zero on 4096 seeded
    pixels, so the exact gradient is the oracle's sum over just those rays."""
    D = (256, 256, 256)
    raw = synth.blobs(D, 4, dtype="f32", nblobs=8, sigma=(12.0, 40.0), amp=(0.2, 1.0), noise=0.02, vmax=1.0)
    cams = [synth.seeded_orbit(D, 512, 512, 4, view=v) for v in range(16)]
    tf = synth.tf_ramp(alpha_start=0.05, alpha_max=0.1)
    params = {"step": 0.5, "et": 0.99}
    npx = 16 * 512 * 512
    mask = np.zeros(npx, bool)
    mask[np.random.default_rng(9).choice(npx, 4096, replace=False)] = True
    _, dtf, dvox, odtf, odvox, _ = run_case(P, orc, raw, cams, tf, params, 3, pixel_mask=mask)
    grad_close(dtf, odtf, "dtf")
    grad_close(dvox, odvox, "dvoxel")


def test_autograd_function_matches_direct_calls(P):
    D, raw, cams, tf, params = small_case()
    vol = P.Volume(D, "f32", 16, 1)
    dens = torch.from_numpy(raw).cuda().requires_grad_(True)
    tfd = torch.from_numpy(tf).cuda().requires_grad_(True)
    img = P.RaycastFn.apply(dens, tfd, vol, cams, params)
    target = torch.zeros_like(img)
    loss = 0.5 * ((img - target) ** 2).sum()
    loss.backward()
    vol2 = P.Volume(D, "f32", 16, 1)
    vol2.upload_level(0, raw, "f32")
    img2 = vol2.render(cams, tfd.detach(), params, grad=True)
    assert torch.equal(img.detach(), img2)
    dtf = torch.zeros_like(tfd)
    dvox = torch.zeros_like(dens)
    vol2.render_backward(img2 - target, dtf, dvox)
    torch.cuda.synchronize()
    grad_close(tfd.grad.cpu().numpy(), dtf.cpu().numpy(), "dtf")
    grad_close(dens.grad.cpu().numpy(), dvox.cpu().numpy(), "dvoxel")


def test_checkpoint_recompute_equals_store_all(P, orc):
    """Transmittance recomputed forward from checkpoints every 32 samples against the store-all
    debug mode (T kept before every sample and read back): the same images bit for bit, and the
    same gradients up to the order of the atomic additions; both against the FP64 oracle."""
    D, raw, cams, tf, params = small_case()
    vol = P.Volume(D, "f32", 16, 1)
    vol.upload_level(0, raw, "f32")
    tfd = torch.from_numpy(tf).cuda()
    rng = np.random.default_rng(11)
    npx = sum(c["w"] * c["h"] for c in cams)
    dI = torch.from_numpy(rng.standard_normal((npx, 4)).astype(np.float32) * np.float32(0.1)).cuda()
    res = {}
    for name, flags in (("ckpt32", 0), ("all", P.C.VOL_RENDER_CKPT_ALL)):
        img, ns = vol.render(cams, tfd, dict(params, flags=flags), grad=True, nsamples=True)
        dtf = torch.zeros((256, 4), dtype=torch.float32, device="cuda")
        dvox = torch.zeros(raw.shape, dtype=torch.float32, device="cuda")
        vol.render_backward(dI, dtf, dvox)
        torch.cuda.synchronize()
        assert vol.stats()["device_error"] == 0
        res[name] = (img.cpu().numpy(), ns.cpu().numpy(), dtf.cpu().numpy(), dvox.cpu().numpy())
    a, b = res["ckpt32"], res["all"]
    assert int(a[1].max()) > 64  # rays span several checkpoint segments
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    for i, what in ((2, "dtf"), (3, "dvoxel")):
        scale = float(np.abs(b[i]).max())
        err = float(np.abs(a[i] - b[i]).max())
        assert err <= 1e-6 * scale, f"{what}: checkpointed vs store-all max err {err:.3g} (scale {scale:.3g})"
    ovol = orc.Volume([raw], "f32", 16)
    odtf, odvox = np.zeros((256, 4)), np.zeros(raw.shape)
    off = 0
    dIh = dI.cpu().numpy().astype(np.float64)
    for cam in cams:
        n = cam["w"] * cam["h"]
        pix = np.stack([np.arange(n) % cam["w"], np.arange(n) // cam["w"]], 1).astype(np.int32)
        ref = orc.render(ovol, cam, tf, params, pixels=pix, amb=AMB)
        _, bad, use_alt = compare(b[0][off:off + n], ref, TOL_FP32)
        assert len(bad) == 0
        g1, g2 = orc.render_grad(ovol, cam, tf, params, dIh[off:off + n], pixels=pix,
                                 alt_select=use_alt.astype(np.int32), amb=AMB)
        odtf += g1
        odvox += g2
        off += n
    grad_close(b[2], odtf, "dtf (store-all)")
    grad_close(b[3], odvox, "dvoxel (store-all)")


def test_value_tape_equals_recompute(P):
    """The adjoint reading the forward's value tape against the adjoint interpolating every value
    again from the bricks: the same images bit for bit, the same gradients up to the order of the
    atomic additions, with and without footprint LOD."""
    D, raw, cams, tf, params = small_case()
    for lod in (0, 1):
        vol = P.Volume(D, "f32", 16, 3 if lod else 1)
        vol.upload_level(0, raw, "f32")
        if lod:
            vol.build_lod(0)
        tfd = torch.from_numpy(tf).cuda()
        npx = sum(c["w"] * c["h"] for c in cams)
        dI = torch.from_numpy(np.random.default_rng(12).standard_normal((npx, 4)).astype(np.float32) * np.float32(0.1)).cuda()
        res = []
        for flags in (0, P.C.VOL_RENDER_GRAD_RECOMPUTE):
            pr = dict(params, flags=flags, lod_mode=lod, lod_bias=1 if lod else 0)
            img = vol.render(cams, tfd, pr, grad=True)
            dtf = torch.zeros((256, 4), dtype=torch.float32, device="cuda")
            dvox = torch.zeros(raw.shape, dtype=torch.float32, device="cuda")
            vol.render_backward(dI, dtf, dvox)
            torch.cuda.synchronize()
            assert vol.stats()["device_error"] == 0
            res.append((img.cpu().numpy(), dtf.cpu().numpy(), dvox.cpu().numpy()))
        np.testing.assert_array_equal(res[0][0], res[1][0])
        # (float32 sums of many atomic additions in another order: a few ulps of the largest entry)
        for i in (1, 2):
            scale = float(np.abs(res[1][i]).max())
            assert scale > 0 and float(np.abs(res[0][i] - res[1][i]).max()) <= 1e-5 * scale


def test_value_tape_across_suspended_rays(P):
    """Bricks arriving during a gradient render (rays suspend at missing bricks and resume): the
    value tape holds every sample's value across the resumption, so the gradients equal those of
    a volume that was resident from the start."""
    D, raw, cams, tf, params = small_case()
    B = 16
    tfd = torch.from_numpy(tf).cuda()
    npx = sum(c["w"] * c["h"] for c in cams)
    dI = torch.from_numpy(np.random.default_rng(13).standard_normal((npx, 4)).astype(np.float32) * np.float32(0.1)).cuda()

    def brick(level, b):
        idx = [np.minimum(np.arange(b[a] * B, b[a] * B + B + 1), D[a] - 1) for a in range(3)]
        return np.ascontiguousarray(raw[idx[2]][:, idx[1]][:, :, idx[0]])

    res = []
    for lazy in (False, True):
        vol = P.Volume(D, "f32", B, 1)
        if lazy:
            vol.set_provider(brick, "f32")
        else:
            vol.upload_level(0, raw, "f32")
        img = vol.render(cams, tfd, dict(params, max_passes=1000), grad=True)
        if lazy:
            assert vol.stats()["passes"] > 1  # rays waited for bricks
        dtf = torch.zeros((256, 4), dtype=torch.float32, device="cuda")
        dvox = torch.zeros(raw.shape, dtype=torch.float32, device="cuda")
        vol.render_backward(dI, dtf, dvox)
        torch.cuda.synchronize()
        assert vol.stats()["device_error"] == 0
        res.append((img.cpu().numpy(), dtf.cpu().numpy(), dvox.cpu().numpy()))
        vol.close()
    np.testing.assert_array_equal(res[0][0], res[1][0])
    for i in (1, 2):
        scale = float(np.abs(res[0][i]).max())
        assert float(np.abs(res[0][i] - res[1][i]).max()) <= 1e-5 * scale
