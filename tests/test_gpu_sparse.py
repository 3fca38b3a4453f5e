"""The three-level sparse page table (Sec. III-E; the virtual zettabyte volume of Sec. V-C).

* On a volume the flat table can also hold, the sparse one gives the same images bit for bit:
  a fly-through through a cache that must evict, and repeated previews converging to the
  full render.
* On a virtual volume of 2^20 voxels per axis (level-0 brick ids past 2^32), the decision records
  (depth, level, voxel, brick id) of GPU traces equal the oracle's, and a frame renders with
  bricks generated on demand."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

GEN = dict(octaves=5, period0=64.0, nspheres=60, radius=(4.0, 30.0), value=(0.3, 1.0))
PREVIEW = 8


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    assert torch.cuda.is_available()
    return volume


def procedural(P, D, B, L, seed, cache_bytes, sparse, gen=GEN):
    vol = P.Volume(D, "u8", B, L, cache_bytes=cache_bytes, layout="compact", sparse_pt=sparse)
    src = synth.brick_source(D, B, L, seed, dtype="u8", **gen)
    vol.set_provider_batch(synth.brick_provider_address(), src, "u8")
    return vol


def test_sparse_equals_flat_flythrough(P):
    D, B, L, seed = (384, 320, 256), 32, 5, 13
    # nearly transparent: the rays cross the volume (about 220 bricks a frame)
    tfd = torch.from_numpy(synth.tf_ramp(alpha_start=0.3, alpha_max=0.02)).cuda()
    cams = synth.flythrough(D, 256, 144, 4, seed)
    slot = P.plan(D, "u8", B, L, layout="compact").slot_bytes
    params = {"lod_mode": 1, "lod_bias": 0, "max_passes": 5000}
    flat = procedural(P, D, B, L, seed, 120 * slot, False)
    sparse = procedural(P, D, B, L, seed, 120 * slot, True)
    evicted = 0
    for cam in cams:
        want = flat.render(cam, tfd, params).cpu().numpy()
        got = sparse.render(cam, tfd, params).cpu().numpy()
        st = sparse.stats()
        assert st["device_error"] == 0 and st["resident"] <= 120
        evicted += st["evicted"]
        np.testing.assert_array_equal(got, want)
    assert evicted > 0, (evicted, st)


def test_sparse_previews_converge(P):
    D, B, L, seed = (256, 224, 192), 32, 4, 7
    tfd = torch.from_numpy(synth.tf_peaks(seed)).cuda()
    cam = synth.seeded_orbit(D, 160, 120, seed)
    slot = P.plan(D, "u8", B, L, layout="compact").slot_bytes
    params = {"lod_mode": 1, "lod_bias": 0, "max_passes": 5000}
    want = procedural(P, D, B, L, seed, 4000 * slot, False).render(cam, tfd, params).cpu().numpy()
    sparse = procedural(P, D, B, L, seed, 4000 * slot, True)
    counts = []
    for _ in range(30):
        got = sparse.render(cam, tfd, dict(params, flags=PREVIEW)).cpu().numpy()
        counts.append(sparse.stats()["preview_samples"])
        if counts[-1] == 0:
            break
    assert counts[0] > 0 and counts[-1] == 0, counts
    np.testing.assert_array_equal(got, want)


def test_virtual_volume_traces_match_oracle(P, orc):
    D, B, L = (1 << 20,) * 3, 64, 7
    vol = P.Volume(D, "u8", B, L, cache_bytes=256 * P.plan((256,) * 3, "u8", B, 1, layout="compact").slot_bytes,
                   layout="compact", sparse_pt=True)
    virt = orc.VirtualVolume(D, L, "u8", B)
    cam = synth.look_at((524288.0, 524300.0, 524310.0), (600000.0, 700000.0, 520000.0), 16, 12, fov_deg=50.0)
    params = {"lod_mode": 1, "lod_bias": 0}
    pix = synth.pixel_subset(16, 12, 40, 3)
    recs, counts = vol.trace(cam, params, pix, 3000)
    ids = []
    for i, (px, py) in enumerate(pix):
        want, n = orc.trace(virt, cam, params, int(px), int(py), 3000)
        assert counts[i] == n
        got = recs[i, :min(n, 3000)]
        for f in ("k", "t_bits", "level", "i0", "local", "brick_id"):
            np.testing.assert_array_equal(got[f], want[f], err_msg=f"pixel {(px, py)} field {f}")
        assert np.all(got["slot"] == 0xFFFFFFFF)   # nothing resident yet
        ids.append(got["brick_id"].max())
    assert max(ids) > 2 ** 32


def test_render_virtual_volume_on_demand(P):
    """1 EB of u8 voxels served by the procedural source: one frame with footprint LOD."""
    D, B, L = (1 << 20,) * 3, 64, 8
    slot = P.plan((512,) * 3, "u8", B, 1, layout="compact").slot_bytes
    gen = dict(octaves=4, period0=2048.0, nspheres=4000, radius=(200.0, 4000.0), value=(0.3, 1.0))
    vol = procedural(P, D, B, L, 3, 6000 * slot, True, gen)
    # opaque from value 0.1 on: the rays end within a few bricks of the eye
    tfd = torch.from_numpy(synth.tf_ramp(alpha_start=0.1, alpha_max=0.3)).cuda()
    cam = synth.look_at((524288.0, 524288.0, 524288.0), (560000.0, 540000.0, 530000.0), 96, 64, fov_deg=60.0)
    params = {"lod_mode": 1, "lod_bias": 1, "max_passes": 2000}
    img = vol.render(cam, tfd, params).cpu().numpy()
    st = vol.stats()
    assert st["device_error"] == 0 and st["bricks_loaded"] > 0 and st["resident"] <= 6000
    assert np.isfinite(img).all() and img[:, 3].max() > 0.1
    # a second render of the same view finds every brick resident: one pass, same image
    img2 = vol.render(cam, tfd, params).cpu().numpy()
    assert vol.stats()["passes"] == 1
    np.testing.assert_array_equal(img2, img)
