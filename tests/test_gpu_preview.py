"""Progressive preview (Sec. III-H: a low-resolution image from coarser levels first, refined as
bricks arrive) on the GPU, against the FP64 oracle under the same residency map.

* explicit residency (bricks uploaded one by one): the preview equals the oracle's preview,
  for emission/absorption and for maximum-opacity projection;
* only the coarsest level resident: the preview equals, bit for bit, the render whose footprint
  LOD puts every sample on the coarsest level;
* repeated preview renders with a provider converge to the full render, bit for bit, with
  the count of samples off their own level falling to zero."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from _helpers import AMB, TOL_FP32, compare, store_levels

pytestmark = pytest.mark.gpu

PREVIEW = 8  # VOL_RENDER_PREVIEW


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    assert torch.cuda.is_available()
    return volume


def brick_of(arr, b, B):
    Dz, Dy, Dx = arr.shape
    zi = np.minimum(b[2] * B + np.arange(B + 1), Dz - 1)
    yi = np.minimum(b[1] * B + np.arange(B + 1), Dy - 1)
    xi = np.minimum(b[0] * B + np.arange(B + 1), Dx - 1)
    return arr[np.ix_(zi, yi, xi)]


def bricks_of_level(arr, B):
    Dz, Dy, Dx = arr.shape
    return [(bx, by, bz) for bz in range(-(-Dz // B)) for by in range(-(-Dy // B)) for bx in range(-(-Dx // B))]


BATCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                            ctypes.c_void_p)


def batch_provider(levels, B):
    """A batch provider over given u8 levels, called by the library's loader thread."""
    nvox = (B + 1) ** 3

    def fn(user, n, reqs, dst):
        try:
            out = np.ctypeslib.as_array((ctypes.c_uint8 * (n * nvox)).from_address(dst))
            for j in range(n):
                l, bx, by, bz = (int(reqs[4 * j + q]) for q in range(4))
                out[j * nvox:(j + 1) * nvox] = brick_of(levels[l], (bx, by, bz), B).ravel()
            return 0
        except Exception:
            return 1

    return BATCH_FN(fn)


def case():
    D = (96, 80, 72)
    raw = synth.blobs(D, 17, nblobs=7, sigma=(5.0, 14.0), amp=(60.0, 200.0), noise=12.0)
    return D, raw


@pytest.mark.parametrize("mode", ["dvr", "mop"])
def test_preview_matches_oracle_under_residency(P, orc, mode):
    D, raw = case()
    B, L = 16, 3
    levels = store_levels(orc, raw, "u8", "u8", L)
    vol = P.Volume(D, "u8", B, L)
    ovol = orc.Volume(levels, "u8", B)
    res = np.zeros(orc.page_table_size(ovol), np.uint8)
    rng = np.random.default_rng(4)
    off = 0
    for l, arr in enumerate(levels):
        bl = bricks_of_level(arr, B)
        keep = rng.random(len(bl)) < (0.35 if l == 0 else (0.7 if l == 1 else 1.0))
        for i, (b, k) in enumerate(zip(bl, keep)):
            if k:
                vol.upload_brick(l, b, brick_of(arr, b, B), "u8")
                res[off + i] = 1
        off += len(bl)
    tf = synth.tf_peaks(17)
    tf[:, 3] = np.clip(tf[:, 3] + 0.02, 0, 1)
    tfd = torch.from_numpy(tf).cuda()
    cam = synth.seeded_orbit(D, 120, 100, 17)
    params = {"lod_mode": 1, "lod_bias": -1, "flags": PREVIEW, "bg": (0.1, 0.2, 0.3, 0.4)}
    if mode == "mop":
        params["composite"] = "mop"
    gpu = vol.render(cam, tfd, params).cpu().numpy()
    st = vol.stats()
    assert st["preview_samples"] > 0 and st["passes"] == 1 and st["device_error"] == 0
    assert len(vol.poll_requests()) > 0          # the absent bricks it wanted
    if mode == "dvr":
        ref = orc.render_preview(ovol, cam, tf, params, res, amb=AMB)
        err, bad, _ = compare(gpu, ref, TOL_FP32)
    else:
        ref = orc.render_max(ovol, cam, tf, params, "mop", amb=1e-5, resident=res)
        g = gpu.astype(np.float64)
        e = np.maximum(np.abs(g[:, 3] - ref["rgba"][:, 3]),
                       np.maximum(np.clip(ref["lo"][:, :3] - g[:, :3], 0, None),
                                  np.clip(g[:, :3] - ref["hi"][:, :3], 0, None)).max(axis=1))
        err, bad = float(e.max()), np.flatnonzero(e > TOL_FP32)
    assert len(bad) == 0, (err, len(bad))
    full = orc.render(ovol, cam, tf, {k: v for k, v in params.items() if k != "flags"}) if mode == "dvr" else None
    if full is not None:
        assert np.abs(full["rgba"] - ref["rgba"]).max() > 1e-3   # the residency changes the image


def test_coarsest_only_equals_coarsest_lod(P, orc):
    D, raw = case()
    B, L = 16, 3
    levels = store_levels(orc, raw, "u8", "u8", L)
    part = P.Volume(D, "u8", B, L)
    for b in bricks_of_level(levels[-1], B):
        part.upload_brick(L - 1, b, brick_of(levels[-1], b, B), "u8")
    full = P.Volume(D, "u8", B, L)
    full.upload_level(0, raw, "u8")
    full.build_lod(0)
    tfd = torch.from_numpy(synth.tf_peaks(5)).cuda()
    cams = [synth.seeded_orbit(D, 64, 48, 5, view=v) for v in range(3)]
    for lod in (0, 1):
        got = part.render(cams, tfd, {"lod_mode": lod, "flags": PREVIEW}).cpu().numpy()
        want = full.render(cams, tfd, {"lod_mode": 1, "lod_bias": 20}).cpu().numpy()
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("batch", [True, False])
def test_repeated_previews_converge_to_full_render(P, orc, batch):
    D, raw = case()
    B, L = 16, 3
    levels = store_levels(orc, raw, "u8", "u8", L)
    full = P.Volume(D, "u8", B, L)
    full.upload_level(0, raw, "u8")
    full.build_lod(0)
    tfd = torch.from_numpy(synth.tf_peaks(9)).cuda()
    cam = synth.seeded_orbit(D, 128, 96, 9)
    params = {"lod_mode": 1, "lod_bias": -1}
    want = full.render(cam, tfd, params).cpu().numpy()
    vol = P.Volume(D, "u8", B, L)
    if batch:
        cb = batch_provider(levels, B)
        vol.set_provider_batch(ctypes.cast(cb, ctypes.c_void_p).value, ctypes.c_int(0), "u8")
    else:
        vol.set_provider(lambda level, b: brick_of(levels[level], b, B), "u8")
    counts = []
    for _ in range(40):
        got = vol.render(cam, tfd, dict(params, flags=PREVIEW)).cpu().numpy()
        counts.append(vol.stats()["preview_samples"])
        if counts[-1] == 0:
            break
    assert counts[0] > 0 and counts[-1] == 0, counts
    np.testing.assert_array_equal(got, want)
    # and a regular render now agrees as well
    np.testing.assert_array_equal(vol.render(cam, tfd, params).cpu().numpy(), want)
