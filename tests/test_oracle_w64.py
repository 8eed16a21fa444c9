"""Pins for the oracle's 64-bit words (§4.2.1 with W = 64: flag bit, D delta
bits, V = 63 - D value bits; a dummy holds a 63-bit delta) and their E11MY
values (E8MY's rounding rule of §4.2.2 on binary64: 1 sign, 11 exponent,
Y = 51 - D mantissa bits). Hand-derived values and words, an exact rational
route and an integer route for the rounding, the layout shared with 32-bit
words, decoding, and the FP64 product against a CSR route and exact
integer arithmetic."""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I


def bits(v: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def e11my_rational(v: float, D: int):
    """E11MY value of v from exact rationals: the grid unit of v's binade
    (the smallest normal binade below it), half away from zero; None past
    the largest finite double."""
    if v == 0.0:
        return v
    m, ex = math.frexp(v)  # |v| in [2^(ex-1), 2^ex)
    ex = max(ex, -1021)
    unit = Fraction(2) ** (ex - 53 + D + 1)
    q = Fraction(v) / unit
    r = math.floor(abs(q) + Fraction(1, 2)) * unit
    if r >= Fraction(2) ** 1024:
        return None
    r = float(r)
    return -r if v < 0 else r


def e11my_integer(v: float, D: int):
    """The same rounding on the bit pattern: add half a unit of the D + 1
    dropped bits to the magnitude, clear them; an all-ones exponent is out of
    range."""
    b = bits(v)
    sign, mag = b & (1 << 63), b & ((1 << 63) - 1)
    mag = (mag + (1 << D)) & ~((2 << D) - 1)
    if (mag >> 52) == 0x7FF:
        return None
    return sign | mag


@pytest.mark.parametrize("v,D,expect", [
    (1.0, 11, 0x3FF0000000000000),
    (1.0 / 3.0, 11, 0x3FD5555555555000),       # dropped bits 0x555 < half: down
    (2.0 / 3.0, 11, 0x3FE5555555555000),       # 0x3FE5555555555555: same bits
    (1 + 2.0 ** -40, 11, 0x3FF0000000001000),  # Y = 40: the last kept bit, exact
    (1 + 2.0 ** -41, 11, 0x3FF0000000001000),  # a tie: away from zero
    (-(1 + 2.0 ** -41), 11, 0xBFF0000000001000),
    (1 + 2.0 ** -42, 11, 0x3FF0000000000000),  # below half: down
    (2 - 2.0 ** -41, 11, 0x4000000000000000),  # rounds up into the next binade
    (26.0, 31, 0x403A000000000000),            # Y = 20 holds 26 = 1.625 * 2^4
    (-0.0, 5, 0x8000000000000000),
])
def test_e11my_hand_values(v, D, expect):
    assert O.e11my_bits(v, D) == expect
    assert bits(O.e11my_value(expect)) == expect


def test_e11my_out_of_range_and_nonfinite():
    with pytest.raises(O.OracleError) as e:
        O.e11my_bits(np.finfo(np.float64).max, 11)  # rounds past the largest finite
    assert e.value.code == O.ERR_RANGE
    for bad in (float("inf"), float("nan")):
        with pytest.raises(O.OracleError) as e:
            O.e11my_bits(bad, 11)
        assert e.value.code == O.ERR_NONFINITE
    with pytest.raises(O.OracleError) as e:
        O.e11my_bits(1.0, 32)  # D outside [1, 31]
    assert e.value.code == O.ERR_ARG


@pytest.mark.parametrize("D", [1, 2, 11, 20, 31])
def test_e11my_equals_rational_and_integer_routes(D):
    rng = np.random.default_rng(D)
    # every binade's exponent field, random mantissas and signs, plus
    # subnormals, the edges of the range and constructed ties
    e = rng.integers(0, 2047, 6000).astype(np.uint64)
    mant = rng.integers(0, 1 << 52, 6000, dtype=np.uint64)
    sign = rng.integers(0, 2, 6000).astype(np.uint64) << np.uint64(63)
    pats = sign | (e << np.uint64(52)) | mant
    # exactly half a unit below the kept bits, in [1, 2)
    ties = (np.uint64(0x3FF0000000000000) | (rng.integers(0, 1 << (51 - D), 500, dtype=np.uint64)
                                             << np.uint64(D + 1)) | np.uint64(1 << D))
    edge = np.array([1, 2, (1 << 52) - 1, 1 << 52, 0x7FEFFFFFFFFFFFFF,
                     0x7FEFFFFFFFFFFFFF - (1 << (D + 1))], np.uint64)
    for p in np.concatenate([pats, ties, edge]):
        v = struct.unpack("<d", struct.pack("<Q", int(p)))[0]
        want = e11my_integer(v, D)
        rat = e11my_rational(v, D)
        assert (want is None) == (rat is None), hex(int(p))
        if want is None:
            with pytest.raises(O.OracleError):
                O.e11my_bits(v, D)
            continue
        got = O.e11my_bits(v, D)
        assert got == want, (hex(int(p)), hex(got), hex(want))
        assert O.e11my_value(got) == rat


@pytest.mark.parametrize("D", [1, 15, 28])
def test_fp32_values_survive_when_y_is_at_least_23(D):
    v = (I.uniform(3000, seed=D) * 1e3).astype(np.float32).astype(np.float64)
    field, deq = O.quantize_e11my(v, D)
    assert np.array_equal(deq, v)
    assert np.all(field & np.uint64((2 << D) - 1) == 0)


def test_words_by_hand():
    # one row, D = 2: a_00 = 1.0 (delta 0), a_05 = 2.0 (delta 5 >= 4: a
    # dummy of 5 first, then the value with delta 0), C = sigma = 1
    csr = I.CSR(n=1, m=6, rowptr=np.array([0, 2]), col=np.array([0, 5], np.int32),
                val=np.array([1.0, 2.0]))
    enc = O.encode64(csr, C=1, sigma=1, D=2, k_left=0)
    assert list(map(int, enc.pack)) == [0x3FF0000000000001, 5 << 1, 0x4000000000000001]
    assert (enc.n_words, enc.n_dummies, enc.n_pad) == (3, 1, 0)


@pytest.mark.parametrize("C,sigma,D", [(32, 256, 11), (8, 16, 2), (1, 1, 20), (32, 1, 22)])
def test_layout_equals_32_bit_words_and_decodes(C, sigma, D):
    # a 32-bit dummy already covers any column gap, so 64-bit words of the
    # same D have the same word counts, perm and offsets
    csr = I.random_csr(900, 70000, 0.003, seed=D, empty_rows=0.1, long_gaps=True)
    e64 = O.encode64(csr, C=C, sigma=sigma, D=D)
    e32 = O.encode(csr, C=C, sigma=sigma, D=D, fmt=O.FMT_E8MY)
    assert np.array_equal(e64.offset, e32.offset)
    assert np.array_equal(e64.perm, e32.perm)
    assert (e64.k_left, e64.n_dummies, e64.n_pad) == (e32.k_left, e32.n_dummies, e32.n_pad)
    assert e64.n_dummies > 0 or D > 16  # column gaps reach 70,000
    col, field, counts = O.decode64(e64, csr.rowptr)
    assert np.array_equal(col, csr.col)
    assert np.array_equal(field, e64.field)
    assert np.array_equal(counts, np.diff(csr.rowptr))


def test_spmv_equals_csr_route_and_exact_integer_product():
    csr = I.random_csr(1500, 1200, 0.01, seed=9, empty_rows=0.05, long_gaps=True)
    enc = O.encode64(csr, C=32, sigma=64, D=11)
    x = I.uniform(csr.m, seed=3).astype(np.float64)
    y = O.packsell64_spmv_f64(enc, x)
    ref = O.csr_spmv_fma_f64(csr, enc.deq, x)
    assert np.array_equal(y.view(np.uint64), ref.view(np.uint64))
    ys = O.packsell64_spmv_f64(enc, x, explicit=True)
    rows = (np.arange(enc.n) // enc.sigma) * enc.sigma + enc.perm
    assert np.array_equal(ys, y[rows])
    # integer values and x: every product and partial sum is exact in double
    rng = np.random.default_rng(4)
    iv = rng.integers(-1000, 1000, csr.nnz).astype(np.float64)
    ix = rng.integers(-1000, 1000, csr.m).astype(np.float64)
    ci = I.CSR(n=csr.n, m=csr.m, rowptr=csr.rowptr, col=csr.col, val=iv)
    ei = O.encode64(ci, C=32, sigma=64, D=11)
    dense = np.zeros((csr.n, csr.m), np.int64)
    rr = np.repeat(np.arange(csr.n), np.diff(csr.rowptr))
    dense[rr, csr.col] = iv.astype(np.int64)
    assert np.array_equal(O.packsell64_spmv_f64(ei, ix), (dense @ ix.astype(np.int64)).astype(np.float64))
