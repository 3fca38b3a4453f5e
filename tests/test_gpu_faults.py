"""Failures made on the host, and the request set (the brick-request hash of Sec. III-H).

* A provider that fails (per-brick Python provider, or a batch provider on the loader thread)
  gives VOL_ERR_PROVIDER; with a working provider the same volume then renders the resident
  image bit for bit.
* A cache of 2 bricks and a pass budget of 3: VOL_ERR_INCOMPLETE, no hang, the passes counted.
* Without a provider, the requests of one pass are, as a set, exactly the first non-resident
  brick of every ray (rays that never terminate early), derived from the oracle's decision trace.
No GPU fault is involved: every failure comes from the host."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from _helpers import c1_inputs, store_levels

pytestmark = pytest.mark.gpu

BATCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                            ctypes.c_void_p)


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


def resident_image(P, raw, cam, tf, params, B, L):
    D = raw.shape[::-1]
    full = P.Volume(D, "u8", B, L)
    full.upload_level(0, raw, "u8")
    full.build_lod(0)
    return full.render(cam, tf, params).cpu().numpy()


def test_per_brick_provider_failure(P, orc):
    D, raw, cam, tf, params = c1_inputs(seed=8)
    B, L = 16, 2
    levels = store_levels(orc, raw, "u8", "u8", L)
    tfd = torch.from_numpy(tf).cuda()
    params = dict(params, lod_mode=1, max_passes=500)
    want = resident_image(P, raw, cam, tfd, params, B, L)
    vol = P.Volume(D, "u8", B, L)
    calls = {"n": 0}

    def flaky(level, b):
        calls["n"] += 1
        if calls["n"] == 5:
            raise IOError("simulated read failure")
        return brick_of(levels[level], b, B)

    vol.set_provider(flaky, "u8")
    with pytest.raises(RuntimeError) as e:
        vol.render(cam, tfd, params)
    assert e.value.code == P.C.VOL_ERR_PROVIDER
    vol.set_provider(lambda level, b: brick_of(levels[level], b, B), "u8")
    np.testing.assert_array_equal(vol.render(cam, tfd, params).cpu().numpy(), want)
    assert vol.stats()["device_error"] == 0


def test_batch_provider_failure_on_loader_thread(P, orc):
    D, raw, cam, tf, params = c1_inputs(seed=9)
    B, L = 16, 2
    levels = store_levels(orc, raw, "u8", "u8", L)
    tfd = torch.from_numpy(tf).cuda()
    params = dict(params, lod_mode=1, max_passes=500)
    want = resident_image(P, raw, cam, tfd, params, B, L)
    nvox = (B + 1) ** 3
    state = {"calls": 0, "fail_at": 2}

    def fn(user, n, reqs, dst):
        state["calls"] += 1
        if state["calls"] == state["fail_at"]:
            return 7
        out = np.ctypeslib.as_array((ctypes.c_uint8 * (n * nvox)).from_address(dst))
        for j in range(n):
            l, bx, by, bz = (int(reqs[4 * j + q]) for q in range(4))
            out[j * nvox:(j + 1) * nvox] = brick_of(levels[l], (bx, by, bz), B).ravel()
        return 0

    cb = BATCH_FN(fn)
    vol = P.Volume(D, "u8", B, L, cache_bytes=200 * P.plan(D, "u8", B, L).slot_bytes)
    vol.set_provider_batch(ctypes.cast(cb, ctypes.c_void_p).value, ctypes.c_int(0), "u8")
    with pytest.raises(RuntimeError) as e:
        vol.render(cam, tfd, params)
    assert e.value.code == P.C.VOL_ERR_PROVIDER
    state["fail_at"] = -1
    np.testing.assert_array_equal(vol.render(cam, tfd, params).cpu().numpy(), want)
    assert vol.stats()["device_error"] == 0 and state["calls"] > 2


def test_tiny_cache_runs_out_of_passes(P, orc):
    D, raw, cam, tf, params = c1_inputs(seed=10)
    B, L = 16, 2
    levels = store_levels(orc, raw, "u8", "u8", L)
    vol = P.Volume(D, "u8", B, L, cache_bytes=2 * P.plan(D, "u8", B, L).slot_bytes)
    vol.set_provider(lambda level, b: brick_of(levels[level], b, B), "u8")
    vol.render(cam, torch.from_numpy(tf).cuda(), dict(params, lod_mode=1, max_passes=3), check_incomplete=False)
    st = vol.stats()
    assert vol.last_rc == P.C.VOL_ERR_INCOMPLETE
    assert st["passes"] == 3 and st["resident"] <= 2 and st["device_error"] == 0


def test_requests_are_the_first_missing_brick_of_each_ray(P, orc):
    D, raw, cam, tf, params = c1_inputs(seed=11)
    cam = dict(cam, w=96, h=96)
    B, L = 16, 2
    levels = store_levels(orc, raw, "u8", "u8", L)
    params = dict(params, lod_mode=1, lod_bias=-1, et=2.0)   # no early termination
    vol = P.Volume(D, "u8", B, L)
    ovol = orc.Volume(levels, "u8", B)
    rng = np.random.default_rng(3)
    resident = set()
    for l, arr in enumerate(levels):
        Dz, Dy, Dx = arr.shape
        for bz in range(-(-Dz // B)):
            for by in range(-(-Dy // B)):
                for bx in range(-(-Dx // B)):
                    if rng.random() < 0.6:
                        vol.upload_brick(l, (bx, by, bz), brick_of(arr, (bx, by, bz), B), "u8")
                        resident.add((l, bx, by, bz))
    vol.render(cam, torch.from_numpy(tf).cuda(), params, check_incomplete=False)
    assert vol.last_rc == P.C.VOL_ERR_INCOMPLETE
    got = {tuple(int(x) for x in r) for r in vol.poll_requests()}
    want = set()
    for py in range(cam["h"]):
        for px in range(cam["w"]):
            recs, _ = orc.trace(ovol, cam, params, px, py, 4000)
            for rec in recs:
                l = int(rec["level"])
                nbx, nby = [-(-levels[l].shape[2 - a] // B) for a in range(2)]
                bid = int(rec["brick_id"])
                key = (l, bid % nbx, (bid // nbx) % nby, bid // (nbx * nby))
                if key not in resident:
                    want.add(key)
                    break
    assert len(want) > 10
    assert got == want
    assert vol.stats()["request_overflow"] == 0
