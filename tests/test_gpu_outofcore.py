"""Out-of-core rendering with bricks generated on demand (the procedural source of the
zettabyte demonstration, Sec. V-C; request queue Sec. III-H; LRU eviction Sec. III-C/E).

* Every level is produced directly by the procedural source (not box-downsampled).  A small
  case is checked against the FP64 oracle, which gets the same levels as dense arrays.
* The image does not depend on the cache size: a fly-through rendered through a cache far
  smaller than the frame's working set (evictions, many request passes) equals, bit for bit,
  the one rendered with room for every brick."""
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


GEN = dict(octaves=5, period0=64.0, nspheres=60, radius=(4.0, 30.0), value=(0.3, 1.0))


def procedural_volume(P, D, brick, levels, seed, cache_bytes, layout="compact"):
    vol = P.Volume(D, "u8", brick, levels, cache_bytes=cache_bytes, layout=layout)
    src = synth.brick_source(D, brick, levels, seed, dtype="u8", **GEN)
    vol.set_provider_batch(synth.brick_provider_address(), src, "u8")
    return vol


def test_procedural_lod_matches_oracle(P, orc):
    D, B, L, seed = (160, 128, 96), 16, 4, 21
    levels = [synth.noise_spheres_level(D, l, seed, dtype="u8", **GEN) for l in range(L)]
    ovol = orc.Volume(levels, "u8", B)
    slot = P.plan(D, "u8", B, L, layout="compact").slot_bytes
    vol = procedural_volume(P, D, B, L, seed, cache_bytes=120 * slot)
    tf = synth.tf_peaks(seed)
    tf[:, 3] = np.clip(tf[:, 3] + 0.02, 0, 1)
    tfd = torch.from_numpy(tf).cuda()
    cams = synth.flythrough(D, 72, 48, 3, seed)
    params = {"lod_mode": 1, "lod_bias": 2, "max_passes": 500}
    for i, cam in enumerate(cams):
        gpu = vol.render(cam, tfd, params).cpu().numpy()
        st = vol.stats()
        assert st["device_error"] == 0
        if i == 0:
            assert st["passes"] > 1 and st["bricks_loaded"] > 0   # later frames may find every brick cached
        ref = orc.render(ovol, cam, tf, params, amb=AMB)
        err, bad, _ = compare(gpu, ref, TOL_FP32)
        assert len(bad) == 0, err


@pytest.mark.parametrize("layout", ["compact", "quad"])
def test_flythrough_independent_of_cache_size(P, layout):
    D, B, L, seed = (512, 512, 512), 32, 5, 5
    tf = synth.tf_peaks(seed)
    tfd = torch.from_numpy(tf).cuda()
    cams = synth.flythrough(D, 320, 180, 8, seed)
    params = {"lod_mode": 1, "lod_bias": 0, "max_passes": 2000}
    big = procedural_volume(P, D, B, L, seed, cache_bytes=0, layout=layout)
    slot = P.plan(D, "u8", B, L, layout=layout).slot_bytes
    small = procedural_volume(P, D, B, L, seed, cache_bytes=400 * slot, layout=layout)
    evicted = loaded = 0
    for cam in cams:
        want = big.render(cam, tfd, params).cpu().numpy()
        got = small.render(cam, tfd, params).cpu().numpy()
        st = small.stats()
        evicted += st["evicted"]
        loaded += st["bricks_loaded"]
        assert st["device_error"] == 0
        np.testing.assert_array_equal(got, want)
    assert evicted > 0 and loaded > 400


@pytest.mark.parametrize("cache_slots", [0, 300])
def test_overlapped_loading_equals_serial(P, cache_slots):
    """Bricks generated on a library thread while the GPU resumes rays (the default with a batch
    provider) give the image of loading everything between passes (VOL_RENDER_SERIAL_LOADS),
    with room for every brick and with a cache that must evict during the frame."""
    D, B, L, seed = (384, 320, 256), 32, 5, 13
    tf = synth.tf_peaks(seed)
    tfd = torch.from_numpy(tf).cuda()
    cams = synth.flythrough(D, 256, 144, 4, seed)
    slot = P.plan(D, "u8", B, L, layout="compact").slot_bytes
    cache = cache_slots * slot
    params = {"lod_mode": 1, "lod_bias": 0, "max_passes": 5000}
    over = procedural_volume(P, D, B, L, seed, cache_bytes=cache)
    serial = procedural_volume(P, D, B, L, seed, cache_bytes=cache)
    loads = 0
    for i, cam in enumerate(cams):
        want = serial.render(cam, tfd, dict(params, flags=4)).cpu().numpy()
        got, ns = over.render(cam, tfd, params, nsamples=True)
        st = over.stats()
        assert st["device_error"] == 0
        loads += st["bricks_loaded"]
        np.testing.assert_array_equal(got.cpu().numpy(), want)
        if i == 0:
            assert st["passes"] > 1 and st["bricks_loaded"] > 0
    assert loads > 0
    if cache_slots:
        assert over.stats()["resident"] <= cache_slots


def test_look_ahead_changes_loads_not_images(P):
    """Rays that wait request the next bricks along them too (default) or not (flag 32): the
    images are the same; the look-ahead takes fewer passes."""
    D, B, L, seed = (384, 320, 256), 32, 5, 17
    tfd = torch.from_numpy(synth.tf_peaks(seed)).cuda()
    cams = synth.flythrough(D, 192, 108, 3, seed)
    params = {"lod_mode": 1, "lod_bias": 0, "max_passes": 5000}
    a = procedural_volume(P, D, B, L, seed, cache_bytes=0)
    b = procedural_volume(P, D, B, L, seed, cache_bytes=0)
    passes = [0, 0]
    for cam in cams:
        ia = a.render(cam, tfd, params).cpu().numpy()
        passes[0] += a.stats()["passes"]
        ib = b.render(cam, tfd, dict(params, flags=32)).cpu().numpy()
        passes[1] += b.stats()["passes"]
        np.testing.assert_array_equal(ia, ib)
    assert passes[0] <= passes[1]
