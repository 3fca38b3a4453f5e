"""Pins for the oracle's gradient through the LOD pyramid (footprint LOD; each coarser level is the
box filter of the one below, so a level-0 voxel reaches the image through every level).

* the box filter's adjoint (orc_downsample_transpose) satisfies <D x, y> = <x, D^T y> against an
  independent numpy float64 restatement of the filter (edge replication), on odd sizes;
* the level-0 gradient of a render whose samples span three levels equals central differences
  of the oracle's own loss, with the pyramid rebuilt from the perturbed level 0.
"""
import numpy as np
import pytest

import synth


def box_filter_np(x):
    """numpy float64 2x2x2 mean, a child index past the edge replaced by the last voxel."""
    Dz, Dy, Dx = x.shape
    p = np.pad(x, ((0, Dz % 2), (0, Dy % 2), (0, Dx % 2)), mode="edge")
    return p.reshape(p.shape[0] // 2, 2, p.shape[1] // 2, 2, p.shape[2] // 2, 2).mean(axis=(1, 3, 5))


@pytest.mark.parametrize("shape", [(7, 6, 5), (9, 1, 4), (2, 3, 3), (1, 1, 1)])
def test_box_filter_adjoint_identity(orc, shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape)
    cshape = tuple((s + 1) // 2 for s in shape)
    y = rng.standard_normal(cshape)
    lhs = float(np.sum(box_filter_np(x) * y))
    rhs = float(np.sum(x * orc.downsample_transpose(y, shape)))
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)
    # every coarse voxel hands out exactly its value: the shares sum to the coarse total
    assert float(orc.downsample_transpose(y, shape).sum()) == pytest.approx(float(y.sum()), rel=1e-12, abs=1e-12)


def _setup(orc):
    D = (24, 20, 18)
    raw = synth.blobs(D, 3, dtype="f32", nblobs=5, sigma=(3, 6), amp=(0.2, 1.0), noise=0.05, vmax=0.9)
    j = np.arange(256) / 255.0
    tf = np.stack([0.2 + 0.6 * j, 0.9 - 0.5 * j, 0.3 + 0.2 * j, 0.02 + 0.2 * j], 1).astype(np.float32)
    # eyes just outside the box, few image rows: along each ray the footprint grows by more than
    # a factor 4, so the samples of a ray spread over levels 0..2
    cams = [synth.look_at((-2.0, 10.0, 9.0), (30.0, 10.5, 9.5), 20, 4, fov_deg=60.0),
            synth.look_at((12.0, -2.0, 8.0), (11.0, 30.0, 9.0), 20, 4, fov_deg=60.0)]
    params = {"et": 2.0, "bg": (0.1, 0.1, 0.2, 0.0), "lod_mode": 1, "lod_bias": 0}
    target = [np.random.default_rng(v).random((c["w"] * c["h"], 4)) * 0.5 for v, c in enumerate(cams)]
    return D, raw, tf, cams, params, target


def _loss_and_grad(orc, raw, tf, cams, params, target):
    vol = orc.Volume(orc.pyramid(raw, 3, "f32"), "f32", 8)
    L, dvox, levels = 0.0, np.zeros(raw.shape), set()
    for cam, tgt in zip(cams, target):
        out = orc.render(vol, cam, tf, params)
        r = out["rgba"] - tgt
        L += 0.5 * float(np.sum(r * r))
        dvox += orc.render_grad(vol, cam, tf, params, r)[1]
        for px in range(0, cam["w"], 3):
            recs, _ = orc.trace(vol, cam, params, px, cam["h"] // 2)
            levels.update(int(l) for l in recs["level"])
    return L, dvox, levels


def test_level0_gradient_through_pyramid_matches_central_differences(orc):
    D, raw, tf, cams, params, target = _setup(orc)
    L0, dvox, levels = _loss_and_grad(orc, raw, tf, cams, params, target)
    assert levels >= {0, 1, 2}
    rng = np.random.default_rng(8)
    cand = np.argwhere(np.abs(dvox) > 1e-3 * np.abs(dvox).max())
    h = 1e-2
    for _ in range(24):
        z, y, x = cand[int(rng.integers(0, len(cand)))]
        rp, rm = raw.copy(), raw.copy()
        rp[z, y, x] += np.float32(h)
        rm[z, y, x] -= np.float32(h)
        hp = float(rp[z, y, x]) - float(raw[z, y, x])
        hm = float(raw[z, y, x]) - float(rm[z, y, x])
        Lp = _loss_and_grad(orc, rp, tf, cams, params, target)[0]
        Lm = _loss_and_grad(orc, rm, tf, cams, params, target)[0]
        fd = (Lp - Lm) / (hp + hm)
        assert fd == pytest.approx(dvox[z, y, x], rel=2e-4, abs=1e-6 * np.abs(dvox).max()), (z, y, x)
