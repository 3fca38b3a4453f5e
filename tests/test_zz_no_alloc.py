"""vol_render_noalloc: the render entry point for callers that may not allocate device memory
after set-up (a host that hands out a fixed device-memory budget once, a render loop that must
never wait in the allocator).  Its scratch lives in a fixed 8 KiB array inside the library.

The test calls it through the C ABI twice in a row on a volume that has never rendered (so no
render scratch of the volume exists) -- with different view sets, so stale scratch from the
first call would show in the second -- checks through the volume's allocation count that the
calls allocated nothing, and compares each image with the one the regular entry point
vol_render() gives for the same inputs on a second volume built from the same data, within the
tests' float32 tolerance.  It is collected last so that a failure here stops a -x run only
after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from _helpers import TOL_FP32, c1_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    return volume


def noalloc(P, vol, cams, tf, params, out):
    from paper_2509_26213_gb300 import _capi as C
    arr = (C.vol_camera * len(cams))(*[P.camera_struct(c) for c in cams])
    p = P.params_struct(**params)
    return C.load().vol_render_noalloc(vol.h, arr, len(cams), ctypes.c_void_p(tf.data_ptr()), ctypes.byref(p),
                                       ctypes.c_void_p(out.data_ptr()), None)


def test_noalloc_matches_regular_render_twice(P):
    D, raw, cam, tf_np, params = c1_inputs(seed=7)
    params = dict(params, lod_mode=1)

    def make():
        v = P.Volume(D, "u8", 32, 2)
        v.upload_level(0, raw, "u8")
        v.build_lod(0)
        return v

    vol, ref = make(), make()
    tf = torch.from_numpy(tf_np).cuda()
    first = [synth.seeded_orbit(D, 96, 80, 7, view=0), synth.seeded_orbit(D, 64, 64, 7, view=1)]
    second = [synth.seeded_orbit(D, 200, 120, 7, view=2)]
    allocs = vol.stats()["allocations"]
    for cams in (first, second):
        npx = sum(c["w"] * c["h"] for c in cams)
        got = torch.full((npx, 4), float("nan"), dtype=torch.float32, device="cuda")
        assert noalloc(P, vol, cams, tf, params, got) == 0
        torch.cuda.synchronize()
        st = vol.stats()
        assert st["allocations"] == allocs, "vol_render_noalloc allocated"
        assert st["device_error"] == 0 and st["launches"] == 1
        want = ref.render(cams, tf, params)
        torch.cuda.synchronize()
        err = float((got - want).abs().max().item())
        assert err <= TOL_FP32, err
    # the regular entry point allocated its render scratch on first use: the count sees it
    assert ref.stats()["allocations"] > allocs


def test_noalloc_rejects_what_it_cannot_do(P):
    from paper_2509_26213_gb300 import _capi as C
    D, raw, cam, tf_np, params = c1_inputs(seed=7)
    tf = torch.from_numpy(tf_np).cuda()
    out = torch.empty((256 * 256 * 65, 4), dtype=torch.float32, device="cuda")
    vol = P.Volume(D, "u8", 32, 1)
    # nothing resident yet: refused before any device work
    assert noalloc(P, vol, [cam], tf, params, out) == C.VOL_ERR_UNSUPPORTED
    vol.upload_level(0, raw, "u8")
    assert noalloc(P, vol, [cam] * (C.VOL_NOALLOC_MAX_VIEWS + 1), tf, params, out) == C.VOL_ERR_INVALID_ARG
    assert noalloc(P, vol, [cam], tf, dict(params, grad=True), out) == C.VOL_ERR_UNSUPPORTED
    assert noalloc(P, vol, [cam], tf, params, out) == 0
    torch.cuda.synchronize()
    # a sparse page table renders emission/absorption only: a projection is refused, not launched
    sp = P.Volume(D, "u8", 32, 1, cache_bytes=64 << 20, sparse_pt=True)
    B1 = 33
    for bz in range(4):
        for by in range(4):
            for bx in range(4):
                blk = np.ascontiguousarray(raw[np.minimum(np.arange(bz * 32, bz * 32 + B1), 127)][
                    :, np.minimum(np.arange(by * 32, by * 32 + B1), 127)][
                    :, :, np.minimum(np.arange(bx * 32, bx * 32 + B1), 127)])
                sp.upload_brick(0, (bx, by, bz), blk, "u8")
    assert noalloc(P, sp, [cam], tf, dict(params, composite="mop"), out) == C.VOL_ERR_UNSUPPORTED
    assert noalloc(P, sp, [cam], tf, params, out) == 0
    torch.cuda.synchronize()
