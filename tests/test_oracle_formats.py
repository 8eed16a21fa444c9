"""Pins for the oracle's value formats and words (§4.2), independent of the oracle.

Each expected value is either derived by hand from the format definitions
(derivation in the comment beside it) or produced by a different
implementation (numpy's float16 and torch's bfloat16 conversions), or it is a
property that any correct rounding must have.
"""
import numpy as np
import pytest

import oracle as O

F16_CASES = [
    # value, binary16 bits; 1 sign, 5 exponent (bias 15), 10 fraction bits
    (1.0, 0x3C00),
    (-2.0, 0xC000),
    (65504.0, 0x7BFF),  # largest finite: (2 - 2^-10) * 2^15
    (65519.99, 0x7BFF),  # below the midpoint 65520 between 65504 and 65536
    (1.0 / 3.0, 0x3555),  # 0.0101010101|0101... -> fraction 0x155, rounded down
    (2.0 ** -24, 0x0001),  # smallest subnormal
    (2.0 ** -25, 0x0000),  # halfway between 0 and 2^-24: ties to even -> 0
    (3 * 2.0 ** -25, 0x0002),  # halfway between 1 and 2 units: ties to even -> 2
    (2.0 ** -14, 0x0400),  # smallest normal
    (1.0 + 2.0 ** -11, 0x3C00),  # halfway between 1 and 1 + 2^-10: even -> 1
    (1.0 + 3 * 2.0 ** -11, 0x3C02),  # halfway between 1+2^-10 and 1+2^-9: even
    (-0.0, 0x8000),
]


@pytest.mark.parametrize("v,bits", F16_CASES)
def test_f16_hand_values(v, bits):
    assert O.f16_bits(v) == bits


def test_f16_overflow_and_nonfinite():
    with pytest.raises(O.OracleError) as e:
        O.f16_bits(65520.0)  # ties to even rounds up to 65536: not representable
    assert e.value.code == O.ERR_RANGE
    with pytest.raises(O.OracleError) as e:
        O.f16_bits(float("inf"))
    assert e.value.code == O.ERR_NONFINITE


def test_f16_matches_numpy_on_random_and_midpoints():
    rng = np.random.default_rng(7)
    bits = rng.integers(0, 2 ** 32, size=60000, dtype=np.uint64).astype(np.uint32)
    v32 = bits.view(np.float32)
    v32 = v32[np.isfinite(v32) & (np.abs(v32) < 65504)]
    # every binary16 value and the exact midpoints between neighbours (ties)
    h = np.arange(0, 0x7BFF, dtype=np.uint16)
    hv = h.view(np.float16).astype(np.float64)
    mids = (hv[:-1] + hv[1:]) / 2
    cand = np.concatenate([v32.astype(np.float64), hv, -hv, mids, -mids,
                           np.nextafter(mids, 0), np.nextafter(mids, 1)])
    cand = cand[np.abs(cand) < 65504].astype(np.float32)  # numpy's cast takes float32
    ref = cand.astype(np.float16).view(np.uint16)
    got = np.array([O.f16_bits(float(c)) for c in cand], dtype=np.uint16)
    assert np.array_equal(got, ref)


def test_f16_value_all_patterns():
    h = np.arange(2 ** 16, dtype=np.uint32).astype(np.uint16)
    ref = h.view(np.float16).astype(np.float64)
    got = np.array([O.f16_value(int(x)) for x in h])
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.array_equal(np.isinf(got), np.isinf(ref))


# --------------------------------------------------------------------------
# E8MY (§4.2.2): 1 sign, 8 exponent, Y = 22 - D mantissa bits
# --------------------------------------------------------------------------
def f32_bits(v):
    return int(np.array(v, np.float32).view(np.uint32))


def test_e8m7_one_third():
    # 1/3 = 0x3EAAAAAB; keep 7 of 23 fraction bits: 0101010|1010...1011, the
    # first dropped bit is 1 and more follow -> round up to 0101011.
    assert O.e8my_bits(float(np.float32(1 / 3)), 15) == 0x3EAB0000


@pytest.mark.parametrize("v,D,bits", [
    # D = 15 (E8M7): grid 2^-7 on [1, 2)
    (1 + 2.0 ** -8, 15, 0x3F810000),  # exact tie between 1 and 1+2^-7: away -> up
    (-(1 + 2.0 ** -8), 15, 0xBF810000),  # away from zero for negatives too
    (1 + 3 * 2.0 ** -8, 15, 0x3F820000),  # tie between 1+2^-7 and 1+2^-6 -> away
    (2 - 2.0 ** -9, 15, 0x40000000),  # rounds up across the binade to 2.0
    # D = 22 (E8M0) keeps no fraction bits: 0.75 lies halfway between 0.5
    # and 1.0 and ties go away from zero -> 1.0
    (0.75, 22, 0x3F800000),
])
def test_e8my_ties_away(v, D, bits):
    assert O.e8my_bits(v, D) == bits


def test_e8my_subnormal_and_overflow():
    # D = 1: the grid in the subnormal range is 2^(D+1) = 4 steps of 2^-149
    assert O.e8my_bits(2.0 ** -149, 1) == 0  # 1/4 of a grid step -> 0
    assert O.e8my_bits(2.0 ** -148, 1) == 4  # exactly half a step: away -> 4 * 2^-149
    assert O.e8my_bits(-(2.0 ** -148), 1) == 0x80000004
    assert O.e8my_bits(-(2.0 ** -150), 1) == 0x80000000  # signed zero
    fmax = float(np.finfo(np.float32).max)  # (2 - 2^-23) * 2^127 rounds to 2^128
    with pytest.raises(O.OracleError) as e:
        O.e8my_bits(fmax, 1)
    assert e.value.code == O.ERR_RANGE
    # (2 - 2^-21) * 2^127 is the largest E8M21 value and maps to itself
    top = float(np.array(0x7F7FFFFC, np.uint32).view(np.float32))
    assert O.e8my_bits(top, 1) == 0x7F7FFFFC
    with pytest.raises(O.OracleError) as e:
        O.e8my_bits(float("nan"), 7)
    assert e.value.code == O.ERR_NONFINITE


def _random_f32(n, seed):
    rng = np.random.default_rng(seed)
    b = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    v = b.view(np.float32)
    return v[np.isfinite(v) & (np.abs(v) < 1e38)]


@pytest.mark.parametrize("D", [1, 2, 7, 11, 12, 15, 22])
def test_e8my_rounding_properties(D):
    """Any correct round-half-away to the E8MY grid: the low D+1 bits are clear,
    the error is at most half a grid step, exact halves go away from zero, and
    the map is monotone."""
    v = np.sort(_random_f32(3000, D).astype(np.float64))
    q = np.array([O.e8my_bits(float(x), D) for x in v], dtype=np.uint32)
    assert np.all(q & np.uint32((1 << (D + 1)) - 1) == 0)
    qv = q.view(np.float32).astype(np.float64)
    ex = np.frexp(v)[1]
    unit = np.ldexp(1.0, np.maximum(ex, -125) - 23 + D)
    err = np.abs(qv - v)
    assert np.all(err <= unit / 2)
    ties = err == unit / 2
    assert np.all(np.abs(qv[ties]) > np.abs(v[ties]))
    assert np.all(np.diff(qv) >= 0)


@pytest.mark.parametrize("D", [1, 7, 11, 15, 22])
def test_e8my_equals_integer_rounding(D):
    """Round half away on the FP32 magnitude bits: add half a step (2^D) and
    clear the low D+1 bits; the carry moves into the exponent by itself. This
    is a different route to the same result for every finite input that does
    not overflow, subnormals included."""
    v = _random_f32(20000, 100 + D)
    sub = (np.random.default_rng(D).integers(0, 2 ** 23, 2000, dtype=np.uint64)
           .astype(np.uint32)).view(np.float32)
    v = np.concatenate([v, sub, -sub])
    b = v.view(np.uint32).astype(np.uint64)
    mag = b & 0x7FFFFFFF
    ref = (b & 0x80000000) | ((mag + (1 << D)) & ~np.uint64((1 << (D + 1)) - 1))
    got = np.array([O.e8my_bits(float(x), D) for x in v], dtype=np.uint64)
    assert np.array_equal(got, ref)


def test_e8m7_matches_bfloat16_except_ties():
    """E8M7 (D = 15) has bfloat16's value set; torch rounds to nearest even,
    the paper rounds halves away from zero, so they agree off ties."""
    torch = pytest.importorskip("torch")
    v = _random_f32(20000, 3)
    v = v[np.abs(v) < 3e38]
    b = v.view(np.uint32)
    tie = (b & 0xFFFF) == 0x8000
    bf = torch.from_numpy(v.copy()).to(torch.bfloat16).view(torch.int16).numpy()
    ref = (bf.astype(np.uint16).astype(np.uint32)) << 16
    got = np.array([O.e8my_bits(float(x), 15) for x in v], dtype=np.uint32)
    assert np.array_equal(got[~tie], ref[~tie])
    vt = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8)], np.float32)
    gt = np.array([O.e8my_bits(float(x), 15) for x in vt], dtype=np.uint32)
    bt = torch.from_numpy(vt).to(torch.bfloat16).view(torch.int16).numpy()
    bt = bt.astype(np.uint16).astype(np.uint32) << 16
    assert gt[0] != bt[0] and gt[1] == bt[1] and gt[2] != bt[2]


# --------------------------------------------------------------------------
# words (§4.2.1): flag in bit 0
# --------------------------------------------------------------------------
@pytest.mark.parametrize("field,delta,word", [
    # FP16 4.0 = 0x4400 in bits 16..31, delta 1 in bits 1..15, flag 1
    (0x4400 << 16, 1, 0x44000003),
    (0xBC00 << 16, 0, 0xBC000001),  # -1.0, delta 0
    (0xBC00 << 16, 63, 0xBC00007F),  # -1.0, delta 63: (63 << 1) | 1 = 0x7F
])
def test_word_value_hand(field, delta, word):
    assert O.word_value(field, delta) == word
    assert O.unpack(word, 15) == (1, delta, field)


def test_word_dummy_and_padding():
    assert O.word_dummy(40000) == 0x00013880  # 40000 << 1 = 80000, flag 0
    assert O.unpack(0x00013880, 15) == (0, 40000, 0)
    assert O.unpack(0, 15) == (0, 0, 0)  # padding: no value, no delta
    assert O.unpack(0xFFFFFFFE, 7) == (0, 2 ** 31 - 1, 0)  # widest delta


@pytest.mark.parametrize("D", [1, 2, 7, 15, 22])
def test_unpack_inverts_pack(D):
    rng = np.random.default_rng(D)
    for _ in range(300):
        field = int(rng.integers(0, 2 ** 32)) & ~((1 << (D + 1)) - 1)
        d = int(rng.integers(0, 2 ** D))
        assert O.unpack(O.word_value(field, d), D) == (1, d, field)
        dd = int(rng.integers(0, 2 ** 31))
        assert O.unpack(O.word_dummy(dd), D) == (0, dd, 0)
