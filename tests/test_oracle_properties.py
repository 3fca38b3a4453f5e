"""Properties of the oracle's renders that hold for any input, on seeded random small volumes,
cameras and transfer functions (Sec. IV-A front-to-back emission/absorption; Sec. V-C LOD).

* The background enters linearly: out = C + T bg per channel, with T = 1 - (alpha - bg_a T)
  read back from the alpha channel, for two backgrounds and the same samples.
* Raising every TF opacity never lowers the output alpha (more absorption, never less); without
  early termination it also never shortens a ray.
* With one level, footprint LOD selects level 0 everywhere: the image equals lod_mode 0, and any
  bias gives the same.
* A render of a subset of pixels equals the same pixels of the full render.
* Exchanging the TF's colour channels permutes the output's colour channels.
* With TF opacity increasing in the coordinate, MOP and MIP give the same image (Sec. V-A).
* Level-scaled sampling with every sample on level 0 is the plain render.
* The adjoint is linear in dL/dI; dL/dtf is zero on TF entries no lookup reads.
A mistake in the compositing order, a sign, a transposed channel or a level choice breaks one of
them.  (hypothesis is not installed on every machine: the tests are skipped there.)"""
import numpy as np
import pytest

import synth

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

SETTINGS = dict(max_examples=12, deadline=None, derandomize=True)


def case(seed, dtype="u8"):
    rng = np.random.default_rng(seed)
    D = tuple(int(x) for x in rng.integers(9, 24, 3))
    raw = synth.blobs(D, seed, dtype=dtype, nblobs=3, sigma=(2, 6), amp=(0.3, 1.0), noise=0.05, vmax=0.95) \
        if dtype == "f32" else rng.integers(0, 256, D[::-1], dtype=np.uint8)
    tf = rng.random((256, 4)).astype(np.float32)
    tf[:, 3] *= np.float32(rng.uniform(0.02, 0.3))
    cam = synth.seeded_orbit(D, int(rng.integers(3, 9)), int(rng.integers(3, 9)), seed)
    return D, raw, tf, cam


def volume(orc, raw, dtype, levels=1, brick=8):
    lv = orc.pyramid(raw, levels, dtype) if levels > 1 else [raw]
    return orc.Volume(lv, dtype, brick)


@settings(**SETTINGS)
@given(st.integers(0, 10 ** 6))
def test_background_enters_linearly(orc, seed):
    D, raw, tf, cam = case(seed)
    vol = volume(orc, raw, "u8")
    bg1, bg2 = (0.0, 0.0, 0.0, 0.0), (0.5, 0.25, 1.0, 0.75)
    o1 = orc.render(vol, cam, tf, {"bg": bg1, "et": 2.0})
    o2 = orc.render(vol, cam, tf, {"bg": bg2, "et": 2.0})
    np.testing.assert_array_equal(o1["n"], o2["n"])
    T = 1.0 - o1["rgba"][:, 3]                      # bg alpha 0: alpha = 1 - T
    b = np.float64(np.float32(bg2))
    np.testing.assert_allclose(o2["rgba"][:, :3], o1["rgba"][:, :3] + T[:, None] * b[:3], rtol=0, atol=1e-12)
    np.testing.assert_allclose(o2["rgba"][:, 3], (1.0 - T) + T * b[3], rtol=0, atol=1e-12)
    assert np.all((T >= 0) & (T <= 1))


@settings(**SETTINGS)
@given(st.integers(0, 10 ** 6), st.floats(1.0, 3.0))
def test_more_opacity_never_less_alpha(orc, seed, gain):
    D, raw, tf, cam = case(seed)
    vol = volume(orc, raw, "u8")
    hi = tf.copy()
    hi[:, 3] = np.minimum(tf[:, 3] * np.float32(gain), 1).astype(np.float32)
    a = orc.render(vol, cam, tf, {"et": 2.0})
    b = orc.render(vol, cam, hi, {"et": 2.0})
    assert np.all(b["rgba"][:, 3] >= a["rgba"][:, 3] - 1e-12)
    np.testing.assert_array_equal(a["n"], b["n"])   # no early termination: every ray to its exit


@settings(**SETTINGS)
@given(st.integers(0, 10 ** 6), st.integers(-3, 3))
def test_single_level_lod_is_level_zero(orc, seed, bias):
    D, raw, tf, cam = case(seed, "f32")
    vol = volume(orc, raw, "f32")
    plain = orc.render(vol, cam, tf, {"lod_mode": 0})
    lod = orc.render(vol, cam, tf, {"lod_mode": 1, "lod_bias": bias})
    np.testing.assert_array_equal(lod["rgba"], plain["rgba"])
    np.testing.assert_array_equal(lod["n"], plain["n"])


@settings(**SETTINGS)
@given(st.integers(0, 10 ** 6))
def test_pixel_subset_equals_full_frame(orc, seed):
    D, raw, tf, cam = case(seed)
    vol = volume(orc, raw, "u8", levels=2)
    params = {"lod_mode": 1, "bg": (0.1, 0.2, 0.3, 0.4)}
    full = orc.render(vol, cam, tf, params)
    pix = synth.pixel_subset(cam["w"], cam["h"], max(1, cam["w"] * cam["h"] // 3), seed)
    sub = orc.render(vol, cam, tf, params, pixels=pix)
    idx = pix[:, 1].astype(np.int64) * cam["w"] + pix[:, 0]
    np.testing.assert_array_equal(sub["rgba"], full["rgba"][idx])
    np.testing.assert_array_equal(sub["n"], full["n"][idx])


@settings(**SETTINGS)
@given(st.integers(0, 10 ** 6), st.permutations([0, 1, 2]))
def test_colour_channels_permute(orc, seed, perm):
    D, raw, tf, cam = case(seed)
    vol = volume(orc, raw, "u8")
    tfp = tf.copy()
    tfp[:, :3] = tf[:, perm]
    a = orc.render(vol, cam, tf, {})
    b = orc.render(vol, cam, tfp, {})
    np.testing.assert_array_equal(b["rgba"][:, :3], a["rgba"][:, perm])
    np.testing.assert_array_equal(b["rgba"][:, 3], a["rgba"][:, 3])


@settings(**SETTINGS)
@given(st.integers(0, 10 ** 6))
def test_increasing_opacity_makes_mop_and_mip_agree(orc, seed):
    """With TF opacity strictly increasing in the coordinate, the most opaque sample is the one
    of largest coordinate: maximum-opacity and maximum-intensity projection give the same image
    (Sec. V-A; the two keep their state in different forms)."""
    D, raw, tf, cam = case(seed)
    tf[:, 3] = np.linspace(0.01, 0.6, 256, dtype=np.float32)
    vol = volume(orc, raw, "u8", levels=2)
    params = {"lod_mode": 1, "bg": (0.2, 0.1, 0.4, 0.3)}
    mop = orc.render_max(vol, cam, tf, params, "mop")
    mip = orc.render_max(vol, cam, tf, params, "mip")
    np.testing.assert_allclose(mop["rgba"], mip["rgba"], rtol=0, atol=1e-12)


@settings(**SETTINGS)
@given(st.integers(0, 10 ** 6))
def test_level_step_on_level_zero_is_the_plain_render(orc, seed):
    """Level-scaled sampling changes nothing where every sample is on level 0 (step 2^0 dt,
    opacity to the power 2^0)."""
    D, raw, tf, cam = case(seed, "f32")
    vol = volume(orc, raw, "f32", levels=2)
    for params in ({"lod_mode": 0}, {"lod_mode": 1, "lod_bias": -30}):
        plain = orc.render(vol, cam, tf, params)
        ls = orc.render(vol, cam, tf, dict(params, flags=16))
        np.testing.assert_array_equal(ls["rgba"], plain["rgba"])
        np.testing.assert_array_equal(ls["n"], plain["n"])


@settings(**SETTINGS)
@given(st.integers(0, 10 ** 6), st.floats(-2.0, 2.0), st.floats(-2.0, 2.0))
def test_adjoint_is_linear_in_the_upstream_gradient(orc, seed, a, b):
    """The adjoint (gradients with respect to the TF and the voxels) is linear in dL/dI, and a
    zero dL/dI gives zero gradients."""
    D, raw, tf, cam = case(seed, "f32")
    vol = volume(orc, raw, "f32")
    n = cam["w"] * cam["h"]
    rng = np.random.default_rng(seed + 1)
    d1, d2 = rng.standard_normal((n, 4)), rng.standard_normal((n, 4))
    g1 = orc.render_grad(vol, cam, tf, {}, d1)
    g2 = orc.render_grad(vol, cam, tf, {}, d2)
    g = orc.render_grad(vol, cam, tf, {}, a * d1 + b * d2)
    for k in range(2):
        want = a * g1[k] + b * g2[k]
        scale = max(np.abs(g1[k]).max(), np.abs(g2[k]).max(), 1e-300)
        np.testing.assert_allclose(g[k], want, rtol=0, atol=1e-11 * scale * (1 + abs(a) + abs(b)))
    z = orc.render_grad(vol, cam, tf, {}, np.zeros((n, 4)))
    assert not z[0].any() and not z[1].any()


@settings(**SETTINGS)
@given(st.integers(0, 10 ** 6), st.integers(40, 120), st.integers(10, 60))
def test_tf_gradient_only_on_entries_the_samples_touch(orc, seed, lo, width):
    """A u8 volume with values in [lo, lo + width]: every TF lookup uses entries lo .. lo + width
    (the interpolation between entry i and i + 1 at coordinate i exactly reads entry i + 1 with
    weight 0), so dL/dtf is zero outside lo .. lo + width + 1."""
    D, _, tf, cam = case(seed)
    rng = np.random.default_rng(seed + 2)
    raw = rng.integers(lo, lo + width + 1, D[::-1], dtype=np.uint8)
    vol = volume(orc, raw, "u8")
    dI = rng.standard_normal((cam["w"] * cam["h"], 4))
    dtf, _ = orc.render_grad(vol, cam, tf, {}, dI)
    outside = np.ones(256, bool)
    outside[lo:lo + width + 2] = False
    assert not dtf[outside].any()
    assert dtf[~outside].any()
