"""Pins of the oracle's 16-bit words (W = 16, D = 7, E4M3 values), one of the
other word sizes the paper names (§4.2.1) but does not evaluate:
hand-derived E4M3 codes (ties both ways, subnormals, the overflow edge),
brute force against every finite E4M3 value, hand-computed words with the
15-bit dummy chain, and the decode round trip."""
import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I


@pytest.mark.parametrize("v,code", [
    (1.0, 0x38), (-1.0, 0xB8), (1.5, 0x3C), (448.0, 0x7E), (-448.0, 0xFE),
    (2.0 ** -6, 0x08), (2.0 ** -9, 0x01), (7 * 2.0 ** -9, 0x07), (0.0, 0x00), (-0.0, 0x80),
    (1 + 1 / 16, 0x38),       # tie between 1 (.000) and 1.125 (.001): to even, 1
    (1 + 3 / 16, 0x3A),       # tie between 1.125 (.001) and 1.25 (.010): to even, 1.25
    (464.0, 0x7E),            # tie between 448 and (unrepresentable) 480: to even, 448
    (2.0 ** -10, 0x00),       # half the smallest subnormal: tie to even, 0
    (3 * 2.0 ** -11, 0x01),   # 0.75 of it: up
    (15 * 2.0 ** -10, 0x08),  # 7.5 subnormal units: tie to even, 8 units = 2^-6
    (26.0, 0x5D), (-1.1, 0xB9),  # 26 = 1.625 * 2^4; 1.1 -> 1.125
])
def test_e4m3_hand_values(v, code):
    assert O.e4m3_bits(v) == code


@pytest.mark.parametrize("v", [465.0, 480.0, 1e6, -500.0])
def test_e4m3_overflow(v):
    with pytest.raises(O.OracleError):
        O.e4m3_bits(v)


@pytest.mark.parametrize("v", [float("nan"), float("inf"), float("-inf")])
def test_e4m3_nonfinite(v):
    with pytest.raises(O.OracleError):
        O.e4m3_bits(v)


def test_e4m3_every_code_round_trips():
    for c in range(256):
        if c & 0x7F == 0x7F:
            assert np.isnan(O.e4m3_value(c))
            continue
        assert O.e4m3_bits(O.e4m3_value(c)) == c or O.e4m3_value(c) == 0.0


def test_e4m3_nearest_by_brute_force():
    """Random magnitudes across the whole range: the code's value is the
    nearest finite E4M3 value, ties to the even code."""
    finite = sorted({O.e4m3_value(c) for c in range(128) if c != 0x7F})
    grid = np.array(finite)
    rng = np.random.default_rng(5)
    vals = np.concatenate([rng.uniform(0, 464, 3000), 2.0 ** rng.uniform(-12, 8.8, 3000)])
    for v in vals:
        q = O.e4m3_value(O.e4m3_bits(v))
        d = np.abs(grid - v)
        best = grid[d == d.min()]
        if best.size == 1:
            assert q == best[0]
        else:  # a tie: the candidate whose code is even
            assert q in best and O.e4m3_bits(q) % 2 == 0


def test_w16_dummy_chain_hand_words():
    """A gap of 70,000 with D = 7 and 15-bit dummy fields: dummies of 32767,
    32767 and 4466, then the value word with delta 0. One row, left offset 0."""
    csr = I.CSR(n=1, m=80000, rowptr=np.array([0, 2]), col=np.array([5, 70005], np.int32),
                val=np.array([1.0, -1.5], np.float32))
    e = O.encode16(csr, C=1, sigma=1, k_left=0)
    assert e.n_dummies == 3 and e.n_words == 5
    assert [int(w) for w in e.pack] == [(0x38 << 8) | (5 << 1) | 1, 32767 << 1, 32767 << 1,
                                        4466 << 1, (0xBC << 8) | 1]


@pytest.mark.parametrize("n,m,dens,C,sigma,gaps", [(300, 90000, 0.002, 32, 256, True),
                                                   (200, 500, 0.05, 8, 16, False),
                                                   (500, 70000, 0.001, 1, 1, True)])
def test_w16_layout_and_roundtrip(n, m, dens, C, sigma, gaps):
    csr = I.random_csr(n, m, dens, seed=n + C, empty_rows=0.1, long_gaps=gaps)
    e = O.encode16(csr, C=C, sigma=sigma)
    col, codes, counts = O.decode16(e, csr.rowptr)
    assert np.array_equal(counts, csr.row_lengths())
    assert np.array_equal(col, csr.col)
    assert np.array_equal(codes, e.codes)
    # widths and offsets follow the word counts (the same plan as 32-bit words)
    S = (n + C - 1) // C
    assert e.offset[-1] == e.n_words and e.offset.size == S + 1
    assert e.n_words == e.words.sum() + e.n_pad
