"""Pins for the oracle's storage arithmetic: binary16 conversion, transcode, LOD downsample.

Each expected value comes from a formulation independent of oracle.c: numpy's own
float16 conversion, numpy reshape/pad box filters, and hand-worked small cases.
"""
import numpy as np
import pytest


def test_half_roundtrip_matches_numpy(orc):
    rng = np.random.default_rng(1)
    vals = np.concatenate([
        rng.uniform(-70000, 70000, 2000), rng.uniform(-1, 1, 2000), rng.uniform(0, 1e-4, 2000),
        rng.uniform(0, 6.2e-5, 500),  # subnormal halves
        np.array([0.0, -0.0, 1.0, 65504.0, 65519.99, 65520.0, 1e9, -1e9, 2.0 ** -24, 2.0 ** -25,
                  3 * 2.0 ** -26, 2.0 ** -14, 0.1, 1.0 / 3.0]),
    ]).astype(np.float32)
    # exact ties between two halves: mantissa + 0.5 ulp
    ties = (np.arange(1024, 2048, dtype=np.float64) + 0.5) * 2.0 ** -10
    vals = np.concatenate([vals, ties.astype(np.float32)])
    want = vals.astype(np.float16).view(np.uint16)
    got = np.array([orc.float_to_half(v) for v in vals], dtype=np.uint16)
    np.testing.assert_array_equal(got, want)


def test_half_to_double_all_finite(orc):
    bits = np.arange(0, 1 << 16, 37, dtype=np.uint16)
    want = bits.view(np.float16).astype(np.float64)
    got = np.array([orc.half_to_double(b) for b in bits])
    finite = np.isfinite(want)
    np.testing.assert_array_equal(got[finite], want[finite])


def test_u16_to_f16_definition(orc):
    u = np.arange(0, 65536, dtype=np.uint16)
    want = (u.astype(np.float32) / np.float32(65535.0)).astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(orc.u16_to_f16(u), want)


def test_level_dims(orc):
    assert orc.level_dims((128, 128, 128), 2) == [(128, 128, 128), (64, 64, 64)]
    assert orc.level_dims((1000, 7, 1), 4) == [(1000, 7, 1), (500, 4, 1), (250, 2, 1), (125, 1, 1)]
    assert orc.level_dims((4096,) * 3, 7)[-1] == (64, 64, 64)


def _box_numpy(a, dtype):
    """Independent 2x2x2 box filter: pad by edge replication to even dims, then take the eight
    strided child views in (dz, dy, dx) order."""
    Dz, Dy, Dx = a.shape
    pad = [(0, Dz % 2), (0, Dy % 2), (0, Dx % 2)]
    p = np.pad(a, pad, mode="edge")
    kids = [p[dz::2, dy::2, dx::2] for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    if dtype in ("u8", "u16"):
        s = sum(k.astype(np.int64) for k in kids)
        return ((s + 4) >> 3).astype(a.dtype)
    if dtype == "f32":
        acc = np.zeros(kids[0].shape, dtype=np.float32)
        for k in kids:
            acc = (acc + k).astype(np.float32)
        return (acc * np.float32(0.125)).astype(np.float32)
    # f16 bits
    acc = np.zeros(kids[0].shape, dtype=np.float32)
    for k in kids:
        acc = (acc + k.view(np.float16).astype(np.float32)).astype(np.float32)
    return (acc * np.float32(0.125)).astype(np.float16).view(np.uint16)


@pytest.mark.parametrize("dtype", ["u8", "u16", "f16", "f32"])
@pytest.mark.parametrize("shape", [(8, 8, 8), (7, 5, 9), (1, 3, 2), (33, 17, 65)])
def test_downsample_matches_independent_box(orc, dtype, shape):
    rng = np.random.default_rng(hash((dtype, shape)) % (1 << 32))
    if dtype == "u8":
        a = rng.integers(0, 256, shape, dtype=np.uint8)
    elif dtype == "u16":
        a = rng.integers(0, 65536, shape, dtype=np.uint16)
    elif dtype == "f32":
        a = rng.random(shape, dtype=np.float32)
    else:
        a = rng.random(shape).astype(np.float16).view(np.uint16)
    got = orc.downsample(a, dtype)
    want = _box_numpy(a, dtype)
    assert got.shape == tuple((s + 1) // 2 for s in shape)
    np.testing.assert_array_equal(got, want)


def test_downsample_hand_values(orc):
    # 2x2x2 u8 block 0..7: sum 28 -> (28 + 4) >> 3 = 4 (round half up of 3.5)
    a = np.arange(8, dtype=np.uint8).reshape(2, 2, 2)
    assert orc.downsample(a, "u8").item() == 4
    # 1 + 0*7 = 1 -> (1 + 4) >> 3 = 0; 4 -> (4+4)>>3 = 1 (0.5 rounds up)
    b = np.zeros((2, 2, 2), np.uint8); b[0, 0, 0] = 4
    assert orc.downsample(b, "u8").item() == 1
    b[0, 0, 0] = 3
    assert orc.downsample(b, "u8").item() == 0
    # odd edge: a 3-long axis; the coarse voxel 1 averages fine voxel 2 with itself
    c = np.array([[[10, 20, 30]]], dtype=np.uint16)
    np.testing.assert_array_equal(orc.downsample(c, "u16"), np.array([[[15, 30]]], np.uint16))


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_downsample_constant_and_conservation(orc, dtype):
    shape = (16, 12, 20)
    val = {"u8": 77, "u16": 40001, "f32": 0.375}[dtype]
    a = np.full(shape, val, dtype={"u8": np.uint8, "u16": np.uint16, "f32": np.float32}[dtype])
    assert np.all(orc.downsample(a, dtype) == a[::2, ::2, ::2])
    # even dims: 8 * mean of the coarse level equals the fine sum (float32 on dyadic values)
    if dtype == "f32":
        rng = np.random.default_rng(3)
        b = (rng.integers(0, 64, shape) / 64.0).astype(np.float32)
        assert orc.downsample(b, "f32").sum(dtype=np.float64) * 8 == pytest.approx(b.sum(dtype=np.float64), abs=0)


def _nearest_binary32(q):
    """The binary32 value nearest to the exact rational q >= 0 (ties to an even significand),
    found by exact rational arithmetic: no float division or conversion rounds anything here."""
    from fractions import Fraction
    if q == 0:
        return np.float32(0.0)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    assert Fraction(2) ** e <= q < Fraction(2) ** (e + 1) and e >= -126  # a normal number
    quantum = Fraction(2) ** (e - 23)
    m = q // quantum
    below, above = q - m * quantum, (m + 1) * quantum - q
    if above < below or (above == below and m % 2 == 1):
        m += 1
    value = m * quantum  # at most 24 significant bits: exact in float64 and in binary32
    out = np.float32(float(value))
    assert Fraction(float(out)) == value
    return out


def test_nearest_binary32_helper_by_hand():
    from fractions import Fraction
    assert _nearest_binary32(Fraction(1, 2)) == np.float32(0.5)
    # 1/3 = 0.0101...b: binary32 0x3eaaaaab (rounded up: the dropped bits are 1010... > half)
    assert _nearest_binary32(Fraction(1, 3)).view(np.uint32) == 0x3EAAAAAB
    # 1 + 2^-24 lies exactly halfway between 1 and 1 + 2^-23: ties to the even significand (1)
    assert _nearest_binary32(1 + Fraction(1, 2 ** 24)) == np.float32(1.0)
    assert _nearest_binary32(1 + Fraction(3, 2 ** 24)).view(np.uint32) == 0x3F800002


def test_u8_to_f32_every_code_is_u_over_255_rounded_once(orc):
    """orc_u8_to_f32 (the normalisation u / 255): all 256 codes against the correctly rounded
    binary32 of the exact quotient."""
    from fractions import Fraction
    u = np.arange(256, dtype=np.uint8)
    want = np.array([_nearest_binary32(Fraction(int(c), 255)) for c in u], dtype=np.float32)
    got = orc.u8_to_f32(u)
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
    assert got[255] == 1.0 and got[0] == 0.0
    # a quotient by 256, or a double rounding through a coarser type, would not match
    assert not np.array_equal(got, (u / 256.0).astype(np.float32))


def test_u16_to_f32_every_code_is_u_over_65535_rounded_once(orc):
    """orc_u16_to_f32 (the normalisation u / 65535): all 65536 codes against the correctly
    rounded binary32 of the exact quotient."""
    from fractions import Fraction
    u = np.arange(65536, dtype=np.uint16)
    want = np.array([_nearest_binary32(Fraction(int(c), 65535)) for c in u], dtype=np.float32)
    got = orc.u16_to_f32(u)
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
    assert got[65535] == 1.0 and got[0] == 0.0 and got[32768] > 0.5 > got[32767]


def test_u16_to_f16_is_binary16_of_the_pinned_quotient(orc):
    """The reduced-precision store: binary16 (nearest, ties to even) of the pinned binary32
    quotient, every code."""
    u = np.arange(65536, dtype=np.uint16)
    want = orc.u16_to_f32(u).astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(orc.u16_to_f16(u), want)
