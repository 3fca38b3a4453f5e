"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Bit-exact: page-table resolve and LOD selection (trace records), LOD downsample and storage
transcode (atlas bytes), batched vs single-view renders, renders after miss passes vs fully
resident.  Tolerance: max-abs per channel 1e-4 (float32 arithmetic; storage decoded alike on
both sides)."""
import numpy as np
import pytest
import torch

import synth
from _helpers import AMB, TOL_FP32, TOL_REDUCED, c1_inputs, compare, store_levels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2509_26213_gb300 as pkg
    pkg.build()
    from paper_2509_26213_gb300 import volume
    assert torch.cuda.is_available()
    return volume


def gpu_volume(P, raw0, src_dtype, store_dtype, brick, levels, cache_bytes=0, layout="quad"):
    Dz, Dy, Dx = raw0.shape
    vol = P.Volume((Dx, Dy, Dz), store_dtype, brick, levels, cache_bytes, layout=layout)
    vol.upload_level(0, raw0, src_dtype)
    if levels > 1:
        vol.build_lod(0)
    return vol


def tf_dev(tf):
    return torch.from_numpy(np.ascontiguousarray(tf, dtype=np.float32)).cuda()


@pytest.mark.parametrize("lod", [0, 1])
def test_c1_full_frame(P, orc, lod):
    D, raw, cam, tf, params = c1_inputs()
    params = dict(params, lod_mode=lod)
    vol = gpu_volume(P, raw, "u8", "u8", 32, 2)
    out, ns = vol.render(cam, tf_dev(tf), params, nsamples=True)
    torch.cuda.synchronize()
    gpu = out.cpu().numpy()
    ovol = orc.Volume(store_levels(orc, raw, "u8", "u8", 2), "u8", 32)
    ref = orc.render(ovol, cam, tf, params, amb=AMB)
    err, bad, alt = compare(gpu, ref, TOL_FP32)
    assert len(bad) == 0, f"{len(bad)} pixels above {TOL_FP32}, max err {err}"
    n_gpu = ns.cpu().numpy()
    agree = (n_gpu == ref["n"]) | (alt & (n_gpu == ref["alt_n"]))
    assert agree.all()
    assert vol.stats()["device_error"] == 0
    print(f"C1 lod={lod}: max abs err {err:.3g}, alternate ET pixels {int(alt.sum())}, samples {int(n_gpu.sum())}")


@pytest.mark.parametrize("lod", [0, 1])
def test_trace_bit_exact(P, orc, lod):
    D, raw, cam, tf, params = c1_inputs(seed=2)
    cam = dict(cam, h=64, w=64, aspect=np.float32(1.0))
    params = dict(params, lod_mode=lod, lod_bias=-1 if lod else 0)   # q spans 2.6..5.6: levels 0 and 1
    vol = gpu_volume(P, raw, "u8", "u8", 32, 2)
    pix = synth.pixel_subset(64, 64, 300, 7)
    recs, counts = vol.trace(cam, params, pix, 600)
    ovol = orc.Volume(store_levels(orc, raw, "u8", "u8", 2), "u8", 32)
    nrec = 0
    for i, (px, py) in enumerate(pix):
        want, n = orc.trace(ovol, cam, params, int(px), int(py), 600)
        assert counts[i] == n
        got = recs[i, :min(n, 600)]
        for f in ("k", "t_bits", "level", "i0", "local", "brick_id"):
            np.testing.assert_array_equal(got[f], want[f], err_msg=f"pixel {(px, py)} field {f}")
        assert np.all(got["slot"] != 0xFFFFFFFF)
        nrec += len(got)
    assert nrec > 10000
    if lod:
        lv = np.concatenate([recs[i, :min(counts[i], 600)]["level"] for i in range(len(pix))])
        assert (lv == 0).any() and (lv == 1).any()


@pytest.mark.parametrize("layout", ["quad", "compact"])
@pytest.mark.parametrize("store,src", [("u8", "u8"), ("u16", "u16"), ("f16", "u16"), ("f32", "f32"),
                                       ("f32", "u8"), ("f16", "f16")])
def test_upload_and_downsample_bit_exact(P, orc, store, src, layout):
    rng = np.random.default_rng(5)
    shape = (33, 45, 70)  # ragged against 16^3 bricks on every axis
    if src == "u8":
        raw = rng.integers(0, 256, shape, dtype=np.uint8)
    elif src == "u16":
        raw = rng.integers(0, 65536, shape, dtype=np.uint16)
    elif src == "f16":
        raw = rng.random(shape).astype(np.float16).view(np.uint16)
    else:
        raw = rng.random(shape, dtype=np.float32)
    L = 4
    vol = gpu_volume(P, raw, src, store, 16, L, layout=layout)
    levels = store_levels(orc, raw, src, store, L)
    npdt = {"u8": np.uint8, "u16": np.uint16, "f16": np.uint16, "f32": np.float32}[store]
    for l, arr in enumerate(levels):
        Dz, Dy, Dx = arr.shape
        nb = vol.level_bricks[l]
        for bz in range(nb[2]):
            for by in range(nb[1]):
                for bx in range(nb[0]):
                    got = vol.download_brick(l, (bx, by, bz)).view(npdt)
                    zi = np.minimum(bz * 16 + np.arange(17), Dz - 1)
                    yi = np.minimum(by * 16 + np.arange(17), Dy - 1)
                    xi = np.minimum(bx * 16 + np.arange(17), Dx - 1)
                    want = arr[np.ix_(zi, yi, xi)]
                    np.testing.assert_array_equal(got, want, err_msg=f"level {l} brick {(bx, by, bz)}")


def test_empty_volume_and_edge_images(P, orc):
    D = (40, 24, 33)
    raw = np.zeros((33, 24, 40), np.uint8)
    vol = gpu_volume(P, raw, "u8", "u8", 16, 3)
    tf = synth.tf_ramp()
    bg = (0.25, 0.5, 0.125, 1.0)
    for (w, h) in [(1, 1), (37, 29), (64, 3), (3, 70)]:
        cam = synth.seeded_orbit(D, w, h, 3)
        for tile in [(8, 8), (16, 16), (32, 4), (32, 1)]:
            out = vol.render(cam, tf_dev(tf), {"bg": bg, "tile_w": tile[0], "tile_h": tile[1]}).cpu().numpy()
            np.testing.assert_array_equal(out, np.tile(np.float32(bg), (w * h, 1)))
    # a camera looking away from the box: every ray misses
    cam = synth.look_at((-50.0, 12.0, 16.0), (-100.0, 12.0, 16.0), 9, 9)
    out = vol.render(cam, tf_dev(tf), {"bg": bg}).cpu().numpy()
    np.testing.assert_array_equal(out, np.tile(np.float32(bg), (81, 1)))


def test_camera_without_field_of_view_is_refused(P):
    """A field of view of zero, negative or not finite gives no footprint (Sec. V-C) and no image:
    VOL_ERR_INVALID_ARG from render and trace, before any device work."""
    D = (40, 24, 33)
    vol = gpu_volume(P, np.zeros((33, 24, 40), np.uint8), "u8", "u8", 16, 2)
    good = synth.seeded_orbit(D, 8, 8, 3)
    for bad in (0.0, -0.5, float("inf"), float("nan")):
        cam = dict(good, tan_half_fov=bad)
        with pytest.raises(RuntimeError) as e:
            vol.render([good, cam], tf_dev(synth.tf_ramp()), {"lod_mode": 1})
        assert e.value.code == P.C.VOL_ERR_INVALID_ARG
        with pytest.raises(RuntimeError) as e:
            vol.trace(cam, {"lod_mode": 1}, np.array([[0, 0]]), 8)
        assert e.value.code == P.C.VOL_ERR_INVALID_ARG
    vol.render(good, tf_dev(synth.tf_ramp()), {"lod_mode": 1})


def test_step_beyond_binary32_sample_indices_is_refused(P):
    """Sample indices stay below 2^24 (past it neighbouring indices give the same depth in
    binary32): a step that puts more samples than that on the volume diagonal (57.1 voxels here)
    is VOL_ERR_INVALID_ARG; one just inside renders."""
    D = (40, 24, 33)
    vol = gpu_volume(P, np.zeros((33, 24, 40), np.uint8), "u8", "u8", 16, 1)
    cam = synth.seeded_orbit(D, 2, 2, 3)
    diag = float(np.sqrt(sum(d * d for d in D)))
    with pytest.raises(RuntimeError) as e:
        vol.render(cam, tf_dev(synth.tf_ramp()), {"step": diag / (2 ** 24 - 32)})
    assert e.value.code == P.C.VOL_ERR_INVALID_ARG
    out = vol.render(cam, tf_dev(synth.tf_ramp(alpha_max=0.0)), {"step": diag / (2 ** 24 - 128), "bg": (0, 0, 0, 1)})
    np.testing.assert_array_equal(out.cpu().numpy(), np.tile(np.float32([0, 0, 0, 1]), (4, 1)))


@pytest.mark.parametrize("dtype", ["u8", "u16", "f16", "f32"])
def test_ragged_volume_inside_camera(P, orc, dtype):
    """Odd dims, bricks of 8, a camera inside the volume, all storage types, LOD on."""
    D = (37, 29, 23)
    rng = np.random.default_rng(9)
    raw = synth.blobs(D, 4, dtype="u8" if dtype == "u8" else "f32", nblobs=6, sigma=(3, 8),
                      amp=(80, 220) if dtype == "u8" else (0.3, 0.9), noise=8 if dtype == "u8" else 0.05)
    if dtype == "u16":
        raw = (raw.astype(np.float64) * 65535).astype(np.uint16)
    if dtype == "f16":
        raw = raw.astype(np.float16).view(np.uint16)
    vol = gpu_volume(P, raw, dtype, dtype, 8, 3)
    ovol = orc.Volume(store_levels(orc, raw, dtype, dtype, 3), dtype, 8)
    tf = synth.tf_peaks(3)
    tf[:, 3] = np.clip(tf[:, 3] + 0.02, 0, 1)
    cams = [synth.look_at((18.0, 14.0, 11.0), (30.0, 20.0, 15.0), 45, 33, fov_deg=70.0),
            synth.seeded_orbit(D, 41, 31, 8)]
    for cam in cams:
        for lod in (0, 1):
            params = {"lod_mode": lod, "lod_bias": 2 if lod else 0, "bg": (0.1, 0.0, 0.2, 0.5)}
            gpu = vol.render(cam, tf_dev(tf), params).cpu().numpy()
            ref = orc.render(ovol, cam, tf, params, amb=AMB)
            err, bad, _ = compare(gpu, ref, TOL_FP32)
            assert len(bad) == 0, (dtype, lod, err)


def test_batched_views_equal_single_and_oracle(P, orc):
    D, raw, _, tf, params = c1_inputs(seed=3)
    vol = gpu_volume(P, raw, "u8", "u8", 32, 2)
    cams = [synth.seeded_orbit(D, s, s, 3, view=i) for i, s in enumerate([17, 64, 40, 96, 33])]
    params = dict(params, lod_mode=1)
    batched = vol.render(cams, tf_dev(tf), params).cpu().numpy()
    ovol = orc.Volume(store_levels(orc, raw, "u8", "u8", 2), "u8", 32)
    off = 0
    for cam in cams:
        n = cam["w"] * cam["h"]
        single = vol.render(cam, tf_dev(tf), params).cpu().numpy()
        np.testing.assert_array_equal(batched[off:off + n], single)
        ref = orc.render(ovol, cam, tf, params, amb=AMB)
        err, bad, _ = compare(batched[off:off + n], ref, TOL_FP32)
        assert len(bad) == 0, err
        off += n


@pytest.mark.parametrize("tile,refill", [((8, 8), 24), ((16, 16), 32), ((32, 4), 1), ((4, 8), 16)])
def test_tile_shape_and_refill_do_not_change_image(P, tile, refill):
    D, raw, cam, tf, params = c1_inputs(seed=4)
    vol = gpu_volume(P, raw, "u8", "u8", 32, 2)
    base = vol.render(cam, tf_dev(tf), params).cpu().numpy()
    out = vol.render(cam, tf_dev(tf), dict(params, tile_w=tile[0], tile_h=tile[1], refill=refill,
                                         ctas_per_sm=1)).cpu().numpy()
    np.testing.assert_array_equal(out, base)


def test_miss_path_with_provider_equals_resident(P, orc):
    """A cache that holds a fraction of the bricks, bricks loaded on request through the
    provider: the final image equals the fully resident render bit for bit."""
    D, raw, cam, tf, params = c1_inputs(seed=5)
    params = dict(params, lod_mode=1, lod_bias=0)
    levels = store_levels(orc, raw, "u8", "u8", 2)
    full = gpu_volume(P, raw, "u8", "u8", 16, 2)
    want = full.render(cam, tf_dev(tf), params).cpu().numpy()
    B = 16

    def provider(level, b):
        arr = levels[level]
        Dz, Dy, Dx = arr.shape
        zi = np.minimum(b[2] * B + np.arange(B + 1), Dz - 1)
        yi = np.minimum(b[1] * B + np.arange(B + 1), Dy - 1)
        xi = np.minimum(b[0] * B + np.arange(B + 1), Dx - 1)
        return arr[np.ix_(zi, yi, xi)]

    slot = P.plan(D, "u8", B, 2).slot_bytes
    vol = P.Volume(D, "u8", B, 2, cache_bytes=300 * slot)   # 300 of 584 bricks
    vol.set_provider(provider, "u8")
    got = vol.render(cam, tf_dev(tf), dict(params, max_passes=200)).cpu().numpy()
    st = vol.stats()
    assert st["passes"] > 1 and st["bricks_loaded"] > 0 and st["device_error"] == 0
    np.testing.assert_array_equal(got, want)
    # a second frame from another angle reuses and evicts
    cam2 = synth.seeded_orbit(D, 256, 256, 5, view=1)
    want2 = full.render(cam2, tf_dev(tf), params).cpu().numpy()
    got2 = vol.render(cam2, tf_dev(tf), dict(params, max_passes=200)).cpu().numpy()
    np.testing.assert_array_equal(got2, want2)
    assert vol.stats()["evicted"] > 0


def test_render_into_page_locked_host_memory(P, orc):
    """An image written straight into page-locked host memory (the kernel writes through the
    host link) equals the image rendered into device memory, bit for bit: several views in one
    launch, and a render whose rays wait for bricks over several passes."""
    D, raw, _, tf, params = c1_inputs(seed=6)
    params = dict(params, lod_mode=1)
    cams = [synth.seeded_orbit(D, s, s, 6, view=i) for i, s in enumerate([64, 37, 96])]
    npx = sum(c["w"] * c["h"] for c in cams)
    full = gpu_volume(P, raw, "u8", "u8", 16, 2)
    want = full.render(cams, tf_dev(tf), params).cpu().numpy()
    host = torch.full((npx, 4), float("nan"), dtype=torch.float32).pin_memory()
    got = full.render(cams, tf_dev(tf), params, out=host)
    torch.cuda.synchronize()
    assert got.data_ptr() == host.data_ptr()
    np.testing.assert_array_equal(host.numpy(), want)
    # the same through the miss path (a cache of half the bricks, bricks from a provider)
    levels = store_levels(orc, raw, "u8", "u8", 2)
    B = 16

    def provider(level, b):
        arr = levels[level]
        Dz, Dy, Dx = arr.shape
        zi = np.minimum(b[2] * B + np.arange(B + 1), Dz - 1)
        yi = np.minimum(b[1] * B + np.arange(B + 1), Dy - 1)
        xi = np.minimum(b[0] * B + np.arange(B + 1), Dx - 1)
        return arr[np.ix_(zi, yi, xi)]

    vol = P.Volume(D, "u8", B, 2, cache_bytes=300 * P.plan(D, "u8", B, 2).slot_bytes)
    vol.set_provider(provider, "u8")
    host.fill_(float("nan"))
    vol.render(cams, tf_dev(tf), dict(params, max_passes=200), out=host)
    torch.cuda.synchronize()
    assert vol.stats()["passes"] > 1
    np.testing.assert_array_equal(host.numpy(), want)


def test_output_the_gpu_cannot_address_is_refused(P):
    """Pageable host memory is neither the GPU's nor mapped for it: the binding refuses it, and
    so does the library itself (checked before any launch) when called through the C ABI."""
    import ctypes
    from paper_2509_26213_gb300 import _capi as C
    D, raw, cam, tf, params = c1_inputs(seed=6)
    vol = gpu_volume(P, raw, "u8", "u8", 32, 1)
    pageable = torch.empty((cam["w"] * cam["h"], 4), dtype=torch.float32)
    with pytest.raises(ValueError):
        vol.render(cam, tf_dev(tf), params, out=pageable)
    buf = np.empty((cam["w"] * cam["h"], 4), np.float32)
    tfd = tf_dev(tf)
    c = (C.vol_camera * 1)(P.camera_struct(cam))
    prm = P.params_struct(**params)
    rc = vol.lib.vol_render(vol.h, c, 1, ctypes.c_void_p(tfd.data_ptr()), ctypes.byref(prm),
                            ctypes.c_void_p(buf.ctypes.data), None)
    assert rc == C.VOL_ERR_INVALID_ARG
    out = torch.empty((cam["w"] * cam["h"], 4), dtype=torch.float32, device="cuda")
    rc = vol.lib.vol_render(vol.h, c, 1, ctypes.c_void_p(tfd.data_ptr()), ctypes.byref(prm),
                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(buf.ctypes.data))
    assert rc == C.VOL_ERR_INVALID_ARG
    assert vol.render(cam, tfd, params, out=out).data_ptr() == out.data_ptr()


def test_requests_without_provider_then_resume(P, orc):
    D, raw, cam, tf, params = c1_inputs(seed=6)
    levels = store_levels(orc, raw, "u8", "u8", 1)
    full = gpu_volume(P, raw, "u8", "u8", 32, 1)
    want = full.render(cam, tf_dev(tf), params).cpu().numpy()
    vol = P.Volume(D, "u8", 32, 1)
    out = vol.render(cam, tf_dev(tf), params, check_incomplete=False)
    assert vol.last_rc == -3  # VOL_ERR_INCOMPLETE
    for _ in range(100):
        req = vol.poll_requests()
        assert len(req) > 0 and len(np.unique(req, axis=0)) == len(req)  # deduplicated
        for l, bx, by, bz in req:
            arr = levels[l]
            zi = np.minimum(bz * 32 + np.arange(33), 127)
            yi = np.minimum(by * 32 + np.arange(33), 127)
            xi = np.minimum(bx * 32 + np.arange(33), 127)
            vol.upload_brick(l, (bx, by, bz), arr[np.ix_(zi, yi, xi)], "u8")
        if vol.resume() == 0:
            break
    np.testing.assert_array_equal(out.cpu().numpy(), want)


@pytest.mark.parametrize("dtype,brick", [("u8", 32), ("u16", 64), ("f16", 16), ("f32", 32)])
def test_quad_and_compact_layouts_give_identical_images(P, orc, dtype, brick):
    """The two atlas layouts gather the same eight corners and interpolate in the same order."""
    D = (70, 45, 66)
    base = synth.blobs(D, 12, dtype="f32", nblobs=7, sigma=(4, 12), amp=(0.2, 0.9), noise=0.05, vmax=1.0)
    raw = {"u8": (base * 255).astype(np.uint8), "u16": (base * 65535).astype(np.uint16),
           "f16": base.astype(np.float16).view(np.uint16), "f32": base}[dtype]
    tf = synth.tf_peaks(12)
    tf[:, 3] = np.clip(tf[:, 3] + 0.02, 0, 1)
    cams = [synth.seeded_orbit(D, 61, 47, 12, view=v) for v in range(3)]
    imgs = []
    for layout in ("quad", "compact"):
        vol = gpu_volume(P, raw, dtype, dtype, brick, 3, layout=layout)
        imgs.append(vol.render(cams, tf_dev(tf), {"lod_mode": 1, "lod_bias": 1}).cpu().numpy())
        vol.close()
    np.testing.assert_array_equal(imgs[0], imgs[1])
    ovol = orc.Volume(store_levels(orc, raw, dtype, dtype, 3), dtype, brick)
    off = 0
    for cam in cams:
        n = cam["w"] * cam["h"]
        ref = orc.render(ovol, cam, tf, {"lod_mode": 1, "lod_bias": 1}, amb=AMB)
        err, bad, _ = compare(imgs[0][off:off + n], ref, TOL_FP32)
        assert len(bad) == 0, err
        off += n


def test_compact_layout_miss_path(P, orc):
    """Out-of-core use with the compact layout (more bricks per cache byte): still the resident image."""
    D, raw, cam, tf, params = c1_inputs(seed=8)
    levels = store_levels(orc, raw, "u8", "u8", 1)
    want = gpu_volume(P, raw, "u8", "u8", 16, 1).render(cam, tf_dev(tf), params).cpu().numpy()
    slot = P.plan(D, "u8", 16, 1, layout="compact").slot_bytes
    vol = P.Volume(D, "u8", 16, 1, cache_bytes=200 * slot, layout="compact")

    def provider(level, b):
        arr = levels[level]
        Dz, Dy, Dx = arr.shape
        idx = [np.minimum(b[a] * 16 + np.arange(17), d - 1) for a, d in ((2, Dz), (1, Dy), (0, Dx))]
        return arr[np.ix_(*idx)]

    vol.set_provider(provider, "u8")
    got = vol.render(cam, tf_dev(tf), dict(params, max_passes=300)).cpu().numpy()
    np.testing.assert_array_equal(got, want)


def test_tile_culling_is_conservative(P, orc):
    """Ray tiles outside a view's bound of the volume's projection are written as misses without
    their rays being set up.  Against the oracle on every pixel, the hit/miss pattern, the sample
    counts and the image are the same, for a volume seen small in a corner of the image, a camera
    whose basis is neither orthogonal nor unit-length, a volume partly behind the eye and one
    that projects outside the image."""
    D = (48, 40, 36)
    raw = np.full(D[::-1], 140, dtype=np.uint8)
    vol = gpu_volume(P, raw, "u8", "u8", 16, 1)
    ovol = orc.Volume(store_levels(orc, raw, "u8", "u8", 1), "u8", 16)
    tf = synth.tf_ramp(alpha_start=0.0, alpha_max=0.05)
    corner = synth.look_at((150.0, 130.0, 110.0), (30.0, 10.0, 5.0), 96, 72, fov_deg=40.0)
    skew = dict(synth.look_at((-60.0, 20.0, 18.0), (24.0, 20.0, 18.0), 80, 64, fov_deg=50.0))
    skew["right"] = np.float32(skew["right"] * 1.3 + 0.2 * skew["up"])
    skew["up"] = np.float32(skew["up"] * 0.8 - 0.1 * skew["fwd"])
    behind = synth.look_at((24.0, 20.0, 40.0), (24.0, 60.0, 40.0), 64, 48, fov_deg=90.0)
    away = synth.look_at((-100.0, -80.0, 18.0), (200.0, -80.0, 18.0), 64, 48, fov_deg=30.0)
    for cam in (corner, skew, behind, away):
        out, ns = vol.render(cam, tf_dev(tf), {}, nsamples=True)
        torch.cuda.synchronize()
        ref = orc.render(ovol, cam, tf, {}, amb=AMB)
        n = ns.cpu().numpy()
        assert np.array_equal(n > 0, ref["n"] > 0)
        assert np.all((n == ref["n"]) | (ref["amb"] & (n == ref["alt_n"])))
        err, bad, _ = compare(out.cpu().numpy(), ref, TOL_FP32)
        assert len(bad) == 0, err
