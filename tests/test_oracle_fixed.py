"""Pins for the oracle's fixed-point value format (an integer format: the
paper allows any V-bit value format, integer ones included, §4.2.1): a V-bit
two's-complement integer q per word, value q * 2^s with one exponent s per
matrix. Hand-derived exponents and fields, ties away from zero, an
independent numpy route for the rounding, and the value's error bound."""
import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I


def test_exponent_hand_values():
    # V = 16 (D = 15): q up to 32767. M = 4: 32767 * 2^-12 = 7.99.. >= 4 and
    # 32767 * 2^-13 = 3.99.. < 4, so s = -12
    assert O.fixed_exponent(4.0, 15) == -12
    # M = 26 (the 27-point diagonal): 32767 * 2^-10 = 31.99 >= 26 > 15.99
    assert O.fixed_exponent(26.0, 15) == -10
    # V = 24 (D = 7): q up to 8388607; M = 1: 8388607 * 2^-23 < 1, * 2^-22 >= 1
    assert O.fixed_exponent(1.0, 7) == -22
    assert O.fixed_exponent(0.0, 15) == 0


@pytest.mark.parametrize("v,D,s,field", [
    (4.0, 15, -12, 0x40000000),     # q = 16384 = 0x4000 in bits 16..31
    (-1.0, 15, -12, 0xF0000000),    # q = -4096 = 0xF000 (16-bit two's complement)
    (2.5 * 2 ** -12, 15, -12, 3 << 16),  # a tie: half away from zero -> 3
    (-2.5 * 2 ** -12, 15, -12, (0x10000 - 3) << 16),
    (0.5 * 2 ** -12, 15, -12, 1 << 16),
    (0.49 * 2 ** -12, 15, -12, 0),
])
def test_fixed_fields_hand_values(v, D, s, field):
    assert O.fixed_bits(v, D, s) == field
    assert O.word_value(field, 1) == field | 3


def test_overflow_and_nonfinite():
    with pytest.raises(O.OracleError) as e:
        O.fixed_bits(32767.5 * 2 ** -12, 15, -12)  # rounds to 32768
    assert e.value.code == O.ERR_RANGE
    with pytest.raises(O.OracleError) as e:
        O.fixed_bits(float("nan"), 15, 0)
    assert e.value.code == O.ERR_NONFINITE


@pytest.mark.parametrize("D", [1, 7, 11, 15, 22])
def test_fixed_quantisation_matches_numpy_route_and_bounds(D):
    V = 31 - D
    rng = np.random.default_rng(D)
    v = rng.standard_normal(5000) * 10.0 ** rng.uniform(-3, 3)
    field, deq, s = O.quantize_fixed(v, D)
    M = np.abs(v).max()
    top = 2.0 ** (V - 1) - 1
    assert top * 2.0 ** s >= M > top * 2.0 ** (s - 1)  # the smallest exponent that holds M
    # round half away from zero, as numpy's floor on the magnitude (numpy's own
    # rounding is half to even)
    q = np.sign(v) * np.floor(np.abs(np.ldexp(v, -s)) + 0.5)
    ref = ((q.astype(np.int64) % (1 << V)).astype(np.uint64) << np.uint64(D + 1)).astype(np.uint32)
    assert np.array_equal(field, ref)
    assert np.array_equal(deq, np.ldexp(q, s))
    assert np.all(np.abs(deq - v) <= 2.0 ** (s - 1))


def test_integer_matrix_is_exact_and_encodes():
    a = I.poisson5(64)
    field, deq, s = O.quantize_fixed(a.val, 15)
    assert np.array_equal(deq, a.val.astype(np.float64))
    e = O.encode(a, C=32, sigma=1, D=15, fmt=O.FMT_FIXED)
    assert e.n_words == 20352 and e.n_dummies == 0
    x = I.uniform(a.n, seed=1).astype(np.float64)
    assert np.array_equal(O.packsell_spmv_f64(e, x), O.csr_spmv_f64(a, a.val, x))
