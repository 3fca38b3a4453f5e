"""The differentiable workload at its full configuration: 256^3 float32 blobs, 16 views at 512x512,
checkpoints every 32 samples, loss L = 1/2 sum (I - I*)^2 against target images rendered with the
seeded perturbed transfer function (sigma 0.05 max, clamped at 0).

The GPU adjoint's gradient is checked against central finite differences (h = 1e-3) of the FP64
oracle's loss on 64 seeded coordinates:
  * 32 voxels (of 64 seeded candidates), on the full 16 x 512^2 image set.  A voxel's value reaches only the samples inside
    the 2x2x2-voxel cube around it, so only the pixels whose rays can cross that cube (the cube's
    projection into each view, widened by 2 pixels) change: the loss difference is exact when only
    those pixels are rendered again, and the GPU gradient at the voxel is exact with dL/dI kept on
    them alone.
  * 32 transfer-function coordinates (in a seeded order of the entries in use), on a reduced image (2 views at 128x128) of the same volume, for
    the cost of re-rendering every pixel twice per coordinate.
The targets I* are the oracle's.  Coordinates where the loss has a kink within +-h are skipped: a
ray's sample count changes (an early-termination decision), or -- for voxels -- a sample's
transfer-function coordinate crosses an entry where the piecewise-linear function bends, which
shows as the central differences at h and h/4 disagreeing (a smooth loss gives both within O(h^2))."""
import numpy as np
import pytest
import torch

import synth
from _helpers import AMB, TOL_FP32, compare
from synth import workloads

pytestmark = pytest.mark.gpu
H = 1e-3


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    return volume


def support_pixels(cam, vox):
    """Pixels (px, py) of view `cam` whose rays can cross the cube of side 2 around voxel vox = (x,
    y, z) (level-0 grid: its value enters samples at grid positions within one voxel of it)."""
    eye = np.asarray(cam["eye"], np.float64)
    r, u, f = (np.asarray(cam[k], np.float64) for k in ("right", "up", "fwd"))
    tan, asp, w, h = float(cam["tan_half_fov"]), float(cam["aspect"]), cam["w"], cam["h"]
    c = np.asarray(vox, np.float64) + 0.5
    pts = np.array([[c[0] + dx, c[1] + dy, c[2] + dz] for dx in (-1, 1) for dy in (-1, 1) for dz in (-1, 1)])
    d = pts - eye
    z = d @ f
    assert np.all(z > 0)
    px = ((d @ r) / (z * tan * asp) + 1.0) * 0.5 * w - 0.5
    py = (1.0 - (d @ u) / (z * tan)) * 0.5 * h - 0.5
    x0, x1 = max(0, int(np.floor(px.min())) - 2), min(w - 1, int(np.ceil(px.max())) + 2)
    y0, y1 = max(0, int(np.floor(py.min())) - 2), min(h - 1, int(np.ceil(py.max())) + 2)
    if x0 > x1 or y0 > y1:
        return np.zeros((0, 2), np.int32)
    xs, ys = np.meshgrid(np.arange(x0, x1 + 1), np.arange(y0, y1 + 1))
    return np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)


def loss_on(orc, ovol, cams, tf, params, pix_by_view, targets):
    tot, ns = 0.0, []
    for v, pix in pix_by_view:
        out = orc.render(ovol, cams[v], tf, params, pixels=pix)
        tot += 0.5 * float(np.sum((out["rgba"] - targets[v]) ** 2))
        ns.append(out["n"])
    return tot, (np.concatenate(ns) if ns else np.zeros(0, np.int32))


def gpu_grad(P, vol, cams, tfd, params, dI):
    vol.render(cams, tfd, params, grad=True)
    dtf = torch.zeros((256, 4), dtype=torch.float32, device="cuda")
    dvox = torch.zeros(tuple(vol.dims[::-1]), dtype=torch.float32, device="cuda")
    vol.render_backward(torch.from_numpy(dI).cuda(), dtf, dvox)
    torch.cuda.synchronize()
    assert vol.stats()["device_error"] == 0
    return dtf.cpu().numpy(), dvox.cpu().numpy()


def test_c4_voxel_gradients_match_central_differences(P, orc):
    wl = workloads.c4()
    raw = wl["make"]()
    D, cams, params = wl["D"], wl["cams"], dict(wl["params"])
    tf = wl["tf"]
    tgt_tf = synth.tf_perturbed(tf, 13)
    vol = P.Volume(D, "f32", wl["brick"], 1)
    vol.upload_level(0, raw, "f32")
    tfd = torch.from_numpy(tf).cuda()
    # choose voxels with a sizeable gradient (selection only: the loss for it uses GPU targets)
    img = vol.render(cams, tfd, params).cpu().numpy()
    tgt_gpu = vol.render(cams, torch.from_numpy(tgt_tf).cuda(), params).cpu().numpy()
    _, dsel = gpu_grad(P, vol, cams, tfd, params, (img - tgt_gpu).astype(np.float32))
    cand = np.argwhere(np.abs(dsel) > 0.05 * np.abs(dsel).max())
    rng = np.random.default_rng(41)
    voxels = [tuple(int(c) for c in cand[i][::-1]) for i in rng.choice(len(cand), 64, replace=False)]
    # the pixels each voxel can affect, their union, and the oracle's targets there
    offs = np.cumsum([0] + [c["w"] * c["h"] for c in cams])
    boxes = [[(v, support_pixels(cams[v], vox)) for v in range(len(cams))] for vox in voxels]
    union = []
    for v in range(len(cams)):
        allp = np.concatenate([b[v][1] for b in boxes])
        union.append((v, np.unique(allp, axis=0) if len(allp) else allp))
    ovol = orc.Volume([raw], "f32", wl["brick"])
    targets_u, dI = {}, np.zeros((offs[-1], 4), np.float32)
    for v, pix in union:
        if not len(pix):
            continue
        tgt = orc.render(ovol, cams[v], tgt_tf, params, pixels=pix)["rgba"]
        ref = orc.render(ovol, cams[v], tf, params, pixels=pix, amb=AMB)
        idx = offs[v] + pix[:, 1].astype(np.int64) * cams[v]["w"] + pix[:, 0]
        err, bad, _ = compare(img[idx], ref, TOL_FP32)
        assert len(bad) == 0, err
        targets_u[v] = {tuple(p): t for p, t in zip(pix.tolist(), tgt)}
        dI[idx] = (img[idx] - tgt).astype(np.float32)
    # the GPU gradient of the loss over the union (exact at the chosen voxels)
    _, dvox = gpu_grad(P, vol, cams, tfd, params, dI)
    scale = np.abs(dvox).max()
    checked = 0
    for vox, box in zip(voxels, boxes):  # seeded order, until 32 voxels are checked
        if checked == 32:
            break
        x, y, z = vox
        tg = {v: np.array([targets_u[v][tuple(p)] for p in pix.tolist()]) for v, pix in box if len(pix)}
        pv = [(v, pix) for v, pix in box if len(pix)]
        _, n0 = loss_on(orc, ovol, cams, tf, params, pv, tg)
        fds, kink = [], False
        for h in (H, H / 4):
            rp, rm = raw.copy(), raw.copy()
            rp[z, y, x] += np.float32(h)
            rm[z, y, x] -= np.float32(h)
            Lp, np_ = loss_on(orc, orc.Volume([rp], "f32", wl["brick"]), cams, tf, params, pv, tg)
            Lm, nm = loss_on(orc, orc.Volume([rm], "f32", wl["brick"]), cams, tf, params, pv, tg)
            kink |= not (np.array_equal(np_, n0) and np.array_equal(nm, n0))
            fds.append((Lp - Lm) / (float(rp[z, y, x]) - float(rm[z, y, x])))
        fd = fds[0]
        if kink or abs(fds[0] - fds[1]) > 2e-4 * abs(fd) + 1e-6 * scale:
            continue  # the loss bends within +-h here
        g = float(dvox[z, y, x])
        assert abs(g - fd) <= 1e-3 * abs(fd) + 1e-5 * scale, (vox, g, fd)
        checked += 1
    assert checked == 32, checked


def test_c4_tf_gradients_match_central_differences(P, orc):
    """TF entries reach every pixel, so a +-h change of one flips some ray's early-termination
    decision almost always: each coordinate's loss is taken over the pixels whose sample counts
    stay put under +-h (and whose decision is not within rounding of the threshold), and the GPU
    gradient with dL/dI kept on those same pixels.  An entry that many samples share (the
    near-empty values) makes the loss strongly curved in it, so the differences at h and h/4 are
    combined by Richardson's extrapolation."""
    wl = workloads.c4()
    raw = wl["make"]()
    D, params = wl["D"], dict(wl["params"])
    cams = [synth.seeded_orbit(D, 128, 128, 4, view=v) for v in range(2)]  # reduced image
    tf = wl["tf"]
    tgt_tf = synth.tf_perturbed(tf, 13)
    vol = P.Volume(D, "f32", wl["brick"], 1)
    vol.upload_level(0, raw, "f32")
    tfd = torch.from_numpy(tf).cuda()
    img = vol.render(cams, tfd, params).cpu().numpy()
    ovol = orc.Volume([raw], "f32", wl["brick"])
    full = [(v, np.stack(np.meshgrid(np.arange(c["w"]), np.arange(c["h"])), -1).reshape(-1, 2).astype(np.int32))
            for v, c in enumerate(cams)]
    tgt = np.concatenate([orc.render(ovol, cams[v], tgt_tf, params, pixels=pix)["rgba"] for v, pix in full])
    base = [orc.render(ovol, cams[v], tf, params, pixels=pix, amb=AMB) for v, pix in full]
    err, bad, _ = compare(img, {k: np.concatenate([b[k] for b in base]) for k in ("rgba", "alt_rgba", "amb")}, TOL_FP32)
    assert len(bad) == 0, err
    n0 = np.concatenate([b["n"] for b in base])
    amb = np.concatenate([b["amb"] for b in base])
    dI_all = (img - tgt).astype(np.float32)

    def render_all(t):
        outs = [orc.render(ovol, cams[v], t, params, pixels=pix) for v, pix in full]
        return np.concatenate([o["rgba"] for o in outs]), np.concatenate([o["n"] for o in outs])

    dtf0, _ = gpu_grad(P, vol, cams, tfd, params, dI_all)
    scale = np.abs(dtf0).max()
    rng = np.random.default_rng(42)
    used = np.argwhere(np.abs(dtf0) > 1e-3 * scale)
    assert len(used) >= 32, len(used)
    checked = 0
    for k in rng.permutation(len(used))[:128]:  # seeded order, until 32 coordinates are checked
        if checked == 32:
            break
        j, ch = (int(c) for c in used[k])
        runs = []
        for h in (H, H / 4):
            tp, tm = tf.copy(), tf.copy()
            tp[j, ch] += h
            tm[j, ch] -= h
            runs.append((render_all(tp), render_all(tm), float(tp[j, ch]) - float(tm[j, ch])))
        keep = ~amb
        for (_, np_), (_, nm), _ in runs:
            keep &= (np_ == n0) & (nm == n0)
        if keep.mean() < 0.9:
            continue
        fds = [(0.5 * np.sum((Ip[keep] - tgt[keep]) ** 2) - 0.5 * np.sum((Im[keep] - tgt[keep]) ** 2)) / dh
               for (Ip, _), (Im, _), dh in runs]
        # the loss is smooth in a TF entry (it moves no sample across an entry) but can be strongly
        # curved where many samples share the entry: Richardson's extrapolation of the central
        # differences at h and h/4 removes their h^2 error term
        fd = (16.0 * fds[1] - fds[0]) / 15.0
        dI = dI_all.copy()
        dI[~keep] = 0
        dtf, _ = gpu_grad(P, vol, cams, tfd, params, dI)
        assert abs(dtf[j, ch] - fd) <= 1e-3 * abs(fd) + 1e-5 * scale, ((j, ch), dtf[j, ch], fd)
        checked += 1
    assert checked == 32, checked
