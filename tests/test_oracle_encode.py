"""Pins for the oracle's encoder and decoder (§3, §4.1, §4.3), independent of it.

Checks: hand-derived counts for the 5-point and 27-point matrices, the
paper's printed HPCG sizes (Table 2), the dummy rule of the §4.3 example,
Eq. 4 values, invariants of the sigma permutation and slice layout, dummy
counts recomputed from numpy deltas, and the decode round trip.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table2():
    rows = {}
    with open(os.path.join(GOLDEN, "paper_table2_hpcg.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, n, nnz = line.split()
                rows[name] = (int(n), int(nnz))
    return rows


def test_hpcg_sizes_closed_form_matches_table2():
    # 27-point stencil on nx*ny*nz: each axis contributes 3 nx - 2 neighbour
    # pairs (i, i') with |i - i'| <= 1, so nnz = (3nx-2)(3ny-2)(3nz-2)
    for name, (n, nnz) in _table2().items():
        x, y, z = (2 ** int(t) for t in name.split("_")[1:])
        assert x * y * z == n
        assert (3 * x - 2) * (3 * y - 2) * (3 * z - 2) == nnz


def test_stencil27_generator_small_boxes():
    for g in [(3, 3, 3), (5, 4, 3), (8, 8, 8)]:
        a = I.stencil27(g)
        assert a.nnz == (3 * g[0] - 2) * (3 * g[1] - 2) * (3 * g[2] - 2)


def test_hpcg_7_7_7_generator_matches_table2():
    n, nnz = _table2()["HPCG_7_7_7"]
    a = I.stencil27(128)
    assert (a.n, a.nnz) == (n, nnz)


@pytest.mark.parametrize("i,sigma,k,d", [
    # Eq. 4: d_i = floor(i/sigma)*sigma - k_left when k_left < floor(i/sigma)*sigma
    (0, 256, 64, 0), (255, 256, 64, 0), (256, 256, 64, 192), (511, 256, 64, 192),
    (512, 256, 64, 448), (256, 256, 300, 0), (512, 256, 300, 212),
    # sigma = 1 reduces Eq. 4 to Eq. 3: d_i = i - k_left when k_left < i
    (64, 1, 64, 0), (65, 1, 64, 1), (1000, 1, 64, 936),
])
def test_left_offset_eq4(i, sigma, k, d):
    assert O.left_offset(i, sigma, k) == d


@pytest.mark.parametrize("sigma", [1, 256])
def test_poisson5_64_counts(sigma):
    # n = 4096, nnz = 5n - 4*64; lower bandwidth 64 (the -L neighbour). Every
    # delta is at most 63 < 2^15, so no dummies. Slices of 32 rows cover half a
    # grid row: grid rows 0 and 63 have at most 4 nonzeros per cell (4 slices
    # of width 4), all other slices contain an interior cell (width 5):
    # N_w = 124 * 32 * 5 + 4 * 32 * 4 = 20352, i.e. 128 padding words.
    a = I.poisson5(64)
    e = O.encode(a, C=32, sigma=sigma, D=15, fmt=O.FMT_FP16)
    assert a.nnz == 20224
    assert e.k_left == 64
    assert (e.n_words, e.n_dummies, e.n_pad) == (20352, 0, 128)


def test_stencil27_128_counts_fp16():
    # k_left = 16513 = 128^2 + 128 + 1. D = 15: the largest gap (16126) and the
    # largest first delta fit in 15 bits, so no dummies. A sigma block of 256
    # rows is two grid lines; interior blocks hold 9nz-nonzero rows in every
    # slice, the two y-boundary blocks of a plane give 4 slices of width 9nz and
    # 4 of width 6nz (nz = 3 inside, 2 on the z faces):
    # N_w = 32*(62*8*9 + 2*(4*9 + 4*6)) * (126*3 + 2*2) = 56,034,816.
    a = I.stencil27(128)
    e = O.encode(a, C=32, sigma=256, D=15, fmt=O.FMT_FP16)
    assert e.k_left == 16513
    assert e.n_dummies == 0
    assert e.n_words == 32 * (62 * 8 * 9 + 2 * (4 * 9 + 4 * 6)) * (126 * 3 + 2 * 2)
    assert e.n_words == 56034816


def _deltas(csr, sigma, k_left):
    """First delta against Eq. 4's left offset, later ones against the previous
    column (Eq. 2), computed with numpy."""
    n = csr.n
    row = np.repeat(np.arange(n, dtype=np.int64), csr.row_lengths())
    col = csr.col.astype(np.int64)
    prev = np.empty_like(col)
    first = np.zeros(col.size, bool)
    first[csr.rowptr[:-1][csr.row_lengths() > 0]] = True
    base = (row // sigma) * sigma
    d0 = np.where(k_left < base, base - k_left, 0)
    prev[first] = d0[first]
    prev[~first] = np.concatenate([[0], col[:-1]])[~first]
    return col - prev, row


def test_dummy_example_of_section_4_3():
    # §4.3's example: D = 2, left offset 0; a delta of 4 does not fit in two
    # bits, so a dummy precedes that element and the element gets delta 0.
    # Row 0: columns 0, 3, 7 (deltas 0, 3, 4); row 1: column 5 (delta 5).
    csr = I.CSR(n=2, m=8, rowptr=np.array([0, 3, 4]), col=np.array([0, 3, 7, 5], np.int32),
                val=np.array([1.0, 2.0, 3.0, 4.0], np.float32))
    e = O.encode(csr, C=2, sigma=2, D=2, fmt=O.FMT_E8MY, k_left=0)
    assert e.k_left == 0 and e.n_dummies == 2
    assert list(e.words) == [4, 2]
    f = lambda v: O.e8my_bits(v, 2)
    # slice of 2 rows, width 4, column-major: p = j * C + l
    want = [f(1.0) | 1, O.word_dummy(5),  # j = 0: row 0 col 0; row 1 dummy to col 5
            f(2.0) | (3 << 1) | 1, f(4.0) | 1,  # j = 1: row 0 delta 3; row 1 delta 0
            O.word_dummy(4), 0,  # j = 2: row 0 dummy (gap 4); row 1 padding
            f(3.0) | 1, 0]  # j = 3: row 0 delta 0 after the dummy; padding
    assert [int(w) for w in e.pack] == want


def _check_layout(csr, e):
    n, C, s = csr.n, e.C, e.sigma
    # perm is a permutation inside every sigma block, sorted by stored words
    # (descending) and stable among equals
    orig = O.storage_rows(e)
    assert np.array_equal(np.sort(orig), np.arange(n))
    assert np.all(orig // s == np.arange(n) // s)
    w_st = e.words[orig]
    for b0 in range(0, n, s):
        blk = slice(b0, min(n, b0 + s))
        ws, os_ = w_st[blk], orig[blk]
        assert np.all(np.diff(ws) <= 0)
        eq = np.diff(ws) == 0
        assert np.all(np.diff(os_)[eq] > 0)
    # slice widths are the max stored words of their C rows
    S = (n + C - 1) // C
    pad = np.zeros(S * C, np.int64)
    pad[:n] = w_st
    widths = pad.reshape(S, C).max(axis=1)
    assert np.array_equal(np.diff(e.offset), C * widths)
    # word counts: nnz plus one dummy per delta that does not fit in D bits
    d, row = _deltas(csr, s, e.k_left)
    assert np.all(d >= 0)
    big = d >= (1 << e.D)
    assert e.n_dummies == int(big.sum())
    assert np.array_equal(e.words, csr.row_lengths() + np.bincount(row[big], minlength=n))
    assert e.n_pad == e.n_words - csr.nnz - e.n_dummies


def _roundtrip(csr, e):
    col, field, counts = O.decode(e, csr.rowptr)
    assert np.array_equal(counts, csr.row_lengths())
    assert np.array_equal(col, csr.col)
    assert np.array_equal(field, e.field)


CASES = [
    # n, m, density, C, sigma, D, fmt, empty-row fraction, long gaps
    (1, 1, 1.0, 32, 256, 15, O.FMT_FP16, 0.0, False),
    (37, 53, 0.2, 32, 256, 15, O.FMT_FP16, 0.1, False),
    (100, 100, 0.05, 4, 8, 1, O.FMT_E8MY, 0.2, True),
    (200, 70, 0.3, 8, 16, 2, O.FMT_E8MY, 0.0, True),
    (130, 400, 0.02, 32, 1, 7, O.FMT_E8MY, 0.3, True),
    (257, 257, 0.03, 32, 256, 11, O.FMT_E8MY, 0.05, False),
    (300, 90, 0.1, 1, 300, 3, O.FMT_E8MY, 0.0, True),
    (64, 5000, 0.01, 16, 32, 22, O.FMT_E8MY, 0.0, True),
]


@pytest.mark.parametrize("case", CASES)
def test_encode_layout_and_roundtrip(case):
    n, m, dens, C, sigma, D, fmt, empty, gaps = case
    csr = I.random_csr(n, m, dens, seed=n + m, empty_rows=empty, long_gaps=gaps)
    e = O.encode(csr, C=C, sigma=sigma, D=D, fmt=fmt)
    assert e.k_left == max(0, int(np.max(np.repeat(np.arange(n), csr.row_lengths())
                                         - csr.col, initial=0)))
    _check_layout(csr, e)
    _roundtrip(csr, e)


@pytest.mark.parametrize("D,fmt", [(15, O.FMT_FP16), (5, O.FMT_E8MY)])
def test_csr_order_layout(D, fmt):
    """C = 1, sigma = 1 is delta-value packing in CSR order: each slice is one
    row, so the pack is the rows' word sequences one after another (no
    padding) and the offsets are their running sums. The expected words are
    built here from numpy deltas (Eq. 2, Eq. 4) and the dummy rule (§4.3)."""
    csr = I.random_csr(120, 300, 0.05, seed=D, empty_rows=0.1, long_gaps=True)
    e = O.encode(csr, C=1, sigma=1, D=D, fmt=fmt)
    d, row = _deltas(csr, 1, e.k_left)
    want, counts = [], np.zeros(csr.n, np.int64)
    for p in range(csr.nnz):
        if d[p] >= (1 << D):
            want.append(O.word_dummy(int(d[p])))
            want.append(int(e.field[p]) | 1)
            counts[row[p]] += 2
        else:
            want.append(int(e.field[p]) | (int(d[p]) << 1) | 1)
            counts[row[p]] += 1
    assert e.n_pad == 0 and e.n_words == len(want)
    assert [int(w) for w in e.pack] == want
    assert np.array_equal(e.offset, np.concatenate([[0], np.cumsum(counts)]))


def test_empty_matrix_and_all_empty_rows():
    csr = I.CSR(n=5, m=7, rowptr=np.zeros(6, np.int64), col=np.zeros(0, np.int32),
                val=np.zeros(0, np.float32))
    e = O.encode(csr, C=4, sigma=2, D=15)
    assert e.n_words == 0 and list(e.offset) == [0, 0, 0]
    csr0 = I.CSR(n=0, m=0, rowptr=np.zeros(1, np.int64), col=np.zeros(0, np.int32),
                 val=np.zeros(0, np.float32))
    e0 = O.encode(csr0)
    assert e0.n_words == 0 and list(e0.offset) == [0]


def test_explicit_and_implicit_pack_identical():
    # the pack array does not depend on how y is ordered (reading of §3, §4.3)
    csr = I.random_csr(90, 90, 0.1, seed=3)
    e = O.encode(csr, C=8, sigma=32, D=7, fmt=O.FMT_E8MY)
    x = I.uniform(90, seed=4).astype(np.float64)
    y_impl = O.packsell_spmv_f64(e, x, explicit=False)
    y_expl = O.packsell_spmv_f64(e, x, explicit=True)
    assert np.array_equal(y_expl, y_impl[O.storage_rows(e)])


def test_encoder_rejects_bad_input():
    bad_sorted = I.CSR(n=1, m=5, rowptr=np.array([0, 2]), col=np.array([3, 1], np.int32),
                       val=np.ones(2, np.float32))
    with pytest.raises(O.OracleError) as e:
        O.encode(bad_sorted)
    assert e.value.code == O.ERR_UNSORTED
    dup = I.CSR(n=1, m=5, rowptr=np.array([0, 2]), col=np.array([1, 1], np.int32),
                val=np.ones(2, np.float32))
    with pytest.raises(O.OracleError):
        O.encode(dup)
    oob = I.CSR(n=1, m=5, rowptr=np.array([0, 1]), col=np.array([5], np.int32),
                val=np.ones(1, np.float32))
    with pytest.raises(O.OracleError) as e:
        O.encode(oob)
    assert e.value.code == O.ERR_RANGE
    big = I.CSR(n=1, m=5, rowptr=np.array([0, 1]), col=np.array([0], np.int32),
                val=np.array([1e5], np.float32))
    with pytest.raises(O.OracleError) as e:
        O.encode(big, fmt=O.FMT_FP16, D=15)
    assert e.value.code == O.ERR_RANGE
    # a k_left below the lower bandwidth would need a negative delta
    lower = I.CSR(n=3, m=3, rowptr=np.array([0, 1, 2, 3]), col=np.array([0, 0, 0], np.int32),
                  val=np.ones(3, np.float32))
    with pytest.raises(O.OracleError):
        O.encode(lower, sigma=1, k_left=0)


def test_irregular_generator_small_dense_rows():
    # small matrices whose Zipf row lengths reach m: every row must still hold
    # distinct sorted columns in range
    for seed in range(3):
        c = I.zipf_irregular(300, seed=seed, sigma_col=30.0)
        d = np.diff(c.col.astype(np.int64))
        first = np.zeros(c.nnz, bool)
        first[c.rowptr[:-1][c.row_lengths() > 0]] = True
        assert np.all(d[~first[1:]] > 0) and c.col.max() < c.m and c.col.min() >= 0
        assert O.check_csr(c) == 0


def test_poisson5_batch_generator_blocks_and_face_model():
    """The block-diagonal batch: each block equals its own system, and the
    values are the face model sum_f theta_f (e_u - e_v)(e_u - e_v)^T plus
    boundary terms, assembled here from the position arrays with numpy."""
    csr, parts = I.poisson5_varcoef_batch(6, seed=2, lmin=3, lmax=9)
    v = np.zeros(csr.nnz)
    np.add.at(v, parts["pos_uu"], parts["theta_f"])
    np.add.at(v, parts["pos_vv"], parts["theta_f"])
    np.add.at(v, parts["pos_uv"], -parts["theta_f"])
    np.add.at(v, parts["pos_vu"], -parts["theta_f"])
    np.add.at(v, parts["pos_b"], parts["theta_b"])
    assert np.allclose(v, csr.val, rtol=1e-15, atol=0)
    for sy in parts["systems"]:
        c = sy["csr"]
        r0, z0 = sy["row0"], sy["nz0"]
        assert c.n == sy["L"] ** 2
        assert np.array_equal(csr.rowptr[r0:r0 + c.n + 1] - z0, c.rowptr)
        assert np.array_equal(csr.col[z0:z0 + c.nnz] - r0, c.col)

