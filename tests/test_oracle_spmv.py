"""Pins for the oracle's SpMV definitions (Eq. 1, §4.4), independent of them:
dense brute force, a closed-form stencil product, the FP32 forward error
bound, and the transpose/SpMM identities against dense numpy products."""
import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I


def _dense(csr, val):
    A = np.zeros((csr.n, csr.m))
    row = np.repeat(np.arange(csr.n), csr.row_lengths())
    A[row, csr.col] = val
    return A


@pytest.mark.parametrize("seed,n,m,C,sigma,D,fmt", [
    (0, 33, 47, 32, 256, 15, O.FMT_FP16),
    (1, 64, 64, 8, 16, 2, O.FMT_E8MY),
    (2, 100, 30, 4, 1, 1, O.FMT_E8MY),
    (3, 17, 200, 16, 4, 7, O.FMT_E8MY),
])
def test_packsell_spmv_matches_dense(seed, n, m, C, sigma, D, fmt):
    csr = I.random_csr(n, m, 0.15, seed=seed, empty_rows=0.1, long_gaps=True)
    e = O.encode(csr, C=C, sigma=sigma, D=D, fmt=fmt)
    x = I.uniform(m, seed=seed + 10).astype(np.float64)
    ref = _dense(csr, e.deq) @ x
    assert np.allclose(O.packsell_spmv_f64(e, x), ref, rtol=1e-13, atol=1e-13)
    assert np.allclose(O.csr_spmv_f64(csr, e.deq, x), ref, rtol=1e-13, atol=1e-13)


def test_poisson5_closed_form():
    # y_(r,c) = 4 x_(r,c) - sum of the four neighbours (absent ones are 0);
    # 4 and -1 are exact in FP16, so quantisation changes nothing
    L = 64
    a = I.poisson5(L)
    e = O.encode(a, C=32, sigma=1, D=15, fmt=O.FMT_FP16)
    x = I.uniform(L * L, seed=0).astype(np.float64)
    g = np.pad(x.reshape(L, L), 1)
    ref = 4 * g[1:-1, 1:-1] - g[:-2, 1:-1] - g[2:, 1:-1] - g[1:-1, :-2] - g[1:-1, 2:]
    assert np.allclose(O.packsell_spmv_f64(e, x), ref.ravel(), rtol=0, atol=1e-15)


def test_fp32_fma_twin_within_error_bound():
    a = I.stencil27(16, seed=5)
    e = O.encode(a, C=32, sigma=256, D=11, fmt=O.FMT_E8MY)
    x = I.uniform(a.n, seed=6)
    y32 = O.csr_spmv_fma_f32(a, e.deq.astype(np.float32), x)
    exact = O.csr_spmv_f64(a, e.deq, x.astype(np.float64))
    bound = O.spmv_error_bound(a, e.deq, x, a.row_lengths())
    assert np.all(np.abs(y32 - exact) <= bound)
    # an exactly representable case: integer values, small integer x
    xi = np.rint(8 * x).astype(np.float32)
    vi = np.rint(e.deq).astype(np.float32)
    assert np.array_equal(O.csr_spmv_fma_f32(a, vi, xi),
                          O.csr_spmv_f64(a, vi, xi).astype(np.float32))


def test_fp32_fma_twin_single_rounding():
    # fma(1+2^-23, 1-2^-23, -1) = -2^-46 exactly; a separate multiply would
    # round the product to 1 and give 0
    csr = I.CSR(n=1, m=2, rowptr=np.array([0, 2]), col=np.array([0, 1], np.int32),
                val=np.array([-1.0, 1 + 2.0 ** -23], np.float32))
    x = np.array([1.0, 1 - 2.0 ** -23], np.float32)
    y = O.csr_spmv_fma_f32(csr, csr.val, x)
    assert y[0] == np.float32(-(2.0 ** -46))


def test_transpose_and_spmm_match_dense():
    csr = I.random_csr(40, 25, 0.2, seed=9)
    v = csr.val.astype(np.float64)
    A = _dense(csr, v)
    dy = I.uniform(40, seed=1).astype(np.float64)
    assert np.allclose(O.csr_spmv_t_f64(csr, v, dy), A.T @ dy, rtol=1e-13, atol=1e-13)
    X = np.random.default_rng(2).standard_normal((25, 5))
    assert np.allclose(O.csr_spmm_f64(csr, v, X), A @ X, rtol=1e-13, atol=1e-13)


def test_backward_error():
    csr = I.random_csr(30, 30, 0.3, seed=4)
    v = csr.val.astype(np.float64)
    x = I.uniform(30, seed=5).astype(np.float64)
    y = O.csr_spmv_f64(csr, v, x)
    assert O.backward_error(y, csr, v, x) == 0.0
    A = _dense(csr, v)
    y2 = y.copy()
    y2[3] += 1e-3
    want = 1e-3 / (np.abs(A).sum(axis=1).max() * np.abs(x).max())
    assert np.isclose(O.backward_error(y2, csr, v, x), want, rtol=1e-12)


@pytest.mark.parametrize("w", [8, 64, 512])
def test_error_bound_is_reached_on_a_row_of_ties(w):
    """A row 1, u, u, ..., u (u = 2^-24, w stored words, x = 1): every fused
    multiply-add 1 + u is an exact tie that rounds to even, i.e. back to 1, so
    the FP32 chain loses u at each of its w - 1 later steps. The error is
    (w - 1) u while sum |a_ij x_j| is about 1: the bound gamma_w * sum must
    hold, and must be within a factor of two of the error here (a bound off
    by a factor, or missing w, fails one of the two). 2^-24 is exact in FP16
    (its smallest subnormal) and in every E8MY."""
    u = 2.0 ** -24
    csr = I.CSR(n=1, m=w, rowptr=np.array([0, w], np.int64), col=np.arange(w, dtype=np.int32),
                val=np.array([1.0] + [u] * (w - 1)))
    e = O.encode(csr, C=32, sigma=1, D=15, fmt=O.FMT_FP16)
    assert np.array_equal(e.deq, csr.val)
    x = np.ones(w, np.float32)
    y32 = O.csr_spmv_fma_f32(csr, e.deq.astype(np.float32), x)
    exact = O.csr_spmv_f64(csr, e.deq, x.astype(np.float64))
    assert y32[0] == 1.0
    err = abs(float(y32[0]) - exact[0])
    assert err == (w - 1) * u
    bound = float(O.spmv_error_bound(csr, e.deq, x, np.array([w]))[0])
    assert err <= bound <= 2.0 * err
