"""Full-size parity in the benchmark's launch configuration, checked on sampled outputs the
oracle computes one by one: every pixel is rendered on the GPU, the oracle renders a seeded
subset; page-table resolve and LOD selection are compared record by record on a seeded subset
of pixels of one view of each image size (C2: 4096 pixels, and 256 more with a LOD bias of +2 so
that the coarser levels of its pyramid (2 and 3) are traced and rendered at full size too; C3: 32 pixels in each of
the 4 sizes)."""
import numpy as np
import pytest
import torch

import synth
from synth import workloads
from _helpers import AMB, TOL_FP32, TOL_REDUCED, compare, compare_projection

pytestmark = pytest.mark.gpu

SKIP = 2         # VOL_RENDER_SKIP_EMPTY
LEVEL_STEP = 16  # VOL_RENDER_LEVEL_STEP


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    return volume


@pytest.fixture(scope="module")
def c2_data(orc):
    wl = workloads.c2()
    raw = wl["make"]()
    lev_u16 = orc.pyramid(raw, wl["levels"], "u16")
    lev_f16 = orc.pyramid(orc.u16_to_f16(raw), wl["levels"], "f16")
    return wl, raw, lev_u16, lev_f16


def check_sampled(P, orc, wl, raw, store, levels, npix, tol, ntrace=24, maxs=4096, params=None):
    params = dict(wl["params"] if params is None else params)
    vol = P.Volume(wl["D"], store, wl["brick"], wl["levels"])
    vol.upload_level(0, raw, wl["src"])
    vol.build_lod(0)
    tf = torch.from_numpy(wl["tf"]).cuda()
    out, ns = vol.render(wl["cams"], tf, params, nsamples=True)
    torch.cuda.synchronize()
    gpu, ngpu = out.cpu().numpy(), ns.cpu().numpy()
    assert vol.stats()["device_error"] == 0
    ovol = orc.Volume(levels, store, wl["brick"])
    worst, off = 0.0, 0
    for v, cam in enumerate(wl["cams"]):
        n = cam["w"] * cam["h"]
        k = max(1, npix // len(wl["cams"]))
        pix = synth.pixel_subset(cam["w"], cam["h"], k, 100 + v)
        idx = off + pix[:, 1].astype(np.int64) * cam["w"] + pix[:, 0]
        ref = orc.render(ovol, cam, wl["tf"], params, pixels=pix, amb=AMB)
        err, bad, alt = compare(gpu[idx], ref, tol)
        assert len(bad) == 0, f"view {v}: {len(bad)} pixels above {tol}, max {err}"
        agree = (ngpu[idx] == ref["n"]) | (alt & (ngpu[idx] == ref["alt_n"]))
        assert agree.all()
        worst = max(worst, err)
        off += n
    # decisions, record by record, on one view of each image size
    levels_seen = set()
    sizes = {}
    for v, cam in enumerate(wl["cams"]):
        sizes.setdefault((cam["w"], cam["h"]), v)
    for v in sorted(sizes.values()):
        cam = wl["cams"][v]
        pix = synth.pixel_subset(cam["w"], cam["h"], ntrace, 999 + v)
        recs, counts = vol.trace(cam, params, pix, maxs)
        for i, (px, py) in enumerate(pix):
            want, n = orc.trace(ovol, cam, params, int(px), int(py), maxs)
            assert counts[i] == n
            got = recs[i, :min(n, maxs)]
            for f in ("k", "t_bits", "level", "i0", "local", "brick_id"):
                np.testing.assert_array_equal(got[f], want[f], err_msg=f"view {v} pixel {(px, py)} field {f}")
            levels_seen |= set(np.unique(got["level"]).tolist())
    vol.close()
    return worst, levels_seen


@pytest.mark.parametrize("store", ["u16", "f16"])
def test_c2_reduced_precision_sampled(P, orc, c2_data, store):
    wl, raw, lev_u16, lev_f16 = c2_data
    # (each trace is compared over its first 2048 samples: the frame's longest rays have about 1,700)
    worst, seen = check_sampled(P, orc, wl, raw, store, lev_u16 if store == "u16" else lev_f16, 4096, TOL_REDUCED,
                                ntrace=4096 if store == "u16" else 256, maxs=2048)
    print(f"C2 {store}: max abs err {worst:.3g} on 4096 sampled pixels; levels traced {sorted(seen)}")
    assert worst <= TOL_FP32  # decoded alike on both sides: only float32 arithmetic differs
    assert len(seen) >= 2


def test_c2_coarse_levels_sampled(P, orc, c2_data):
    """The same frame with a LOD bias of +2: its samples fall on levels 2 and 3 of the 1024^3
    pyramid, which the benchmark's view does not reach."""
    wl, raw, lev_u16, _ = c2_data
    params = dict(wl["params"], lod_bias=2)
    worst, seen = check_sampled(P, orc, wl, raw, "u16", lev_u16, 2048, TOL_REDUCED, ntrace=256, maxs=2048,
                                params=params)
    print(f"C2 lod_bias +2: max abs err {worst:.3g} on 2048 sampled pixels; levels traced {sorted(seen)}")
    assert worst <= TOL_FP32
    assert max(seen) >= 3 and len(seen) >= 2


def test_c2_bench_variants_sampled(P, orc, c2_data):
    """The variant lines bench.py times on the full C2 frame (u16 store): maximum-opacity and
    maximum-intensity projection, level-scaled sampling and empty-space skipping, each on 1024
    seeded pixels against the oracle (skipping must also give the default image bit for bit)."""
    wl, raw, lev_u16, _ = c2_data
    vol = P.Volume(wl["D"], "u16", wl["brick"], wl["levels"])
    vol.upload_level(0, raw, wl["src"])
    vol.build_lod(0)
    tf = torch.from_numpy(wl["tf"]).cuda()
    ovol = orc.Volume(lev_u16, "u16", wl["brick"])
    cam = wl["cams"][0]
    pix = synth.pixel_subset(cam["w"], cam["h"], 1024, 7)
    idx = pix[:, 1].astype(np.int64) * cam["w"] + pix[:, 0]
    base = dict(wl["params"])
    default = vol.render(cam, tf, base).cpu().numpy()
    np.testing.assert_array_equal(vol.render(cam, tf, dict(base, flags=SKIP)).cpu().numpy(), default)
    for mode in ("mop", "mip"):
        prm = dict(base, composite=mode)
        gpu = vol.render(cam, tf, prm).cpu().numpy()[idx]
        ref = orc.render_max(ovol, cam, wl["tf"], prm, mode, pixels=pix, amb=AMB)
        err, bad, near = compare_projection(gpu, ref, TOL_REDUCED)
        assert len(bad) == 0, f"{mode}: {len(bad)} pixels above {TOL_REDUCED}, max {err}"
        assert err <= TOL_FP32
        np.testing.assert_array_equal(vol.render(cam, tf, dict(prm, flags=SKIP)).cpu().numpy()[idx], gpu)
    prm = dict(base, flags=LEVEL_STEP)
    out, ns = vol.render(cam, tf, prm, nsamples=True)
    gpu, n = out.cpu().numpy()[idx], ns.cpu().numpy()[idx]
    ref = orc.render(ovol, cam, wl["tf"], prm, pixels=pix, amb=AMB)
    err, bad, alt = compare(gpu, ref, TOL_REDUCED)
    assert len(bad) == 0 and err <= TOL_FP32, (err, len(bad))
    assert np.all((n == ref["n"]) | (alt & (n == ref["alt_n"])))
    assert vol.stats()["device_error"] == 0
    vol.close()


def test_c3_batched_sampled(P, orc):
    wl = workloads.c3()
    raw = wl["make"]()
    levels = orc.pyramid(raw, wl["levels"], "u8")
    worst, seen = check_sampled(P, orc, wl, raw, "u8", levels, 64 * 48, TOL_FP32, ntrace=32, maxs=8192)
    print(f"C3: max abs err {worst:.3g} over 64 views; levels traced {sorted(seen)}")
