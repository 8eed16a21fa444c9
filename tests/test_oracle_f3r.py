"""Pins for the oracle's F3R (§5.2.1) and its building blocks, against
independent references: numpy's dense solve, the minimal-residual property of
GMRES over the explicit Krylov subspace, the one-step solution of flexible
GMRES with an exact preconditioner, and closed forms of the Richardson
layer."""
import numpy as np
import pytest

import oracle as O
from oracle import solvers as S
from paper_2604_13433_gb300 import inputs as I


def _nonsym(n, seed):
    """A nonsymmetric, diagonally dominant sparse matrix, scaled to a unit
    diagonal (the symmetric scaling of §5.2)."""
    a = I.random_csr(n, n, 6.0 / n, seed=seed)
    d = np.zeros((n, n))
    d[np.repeat(np.arange(n), a.row_lengths()), a.col] = a.val
    d += np.diag(np.abs(d).sum(axis=1) + 1.0)
    g = 1.0 / np.sqrt(np.abs(np.diag(d)))
    d = g[:, None] * d * g[None, :]
    rows, cols = np.nonzero(d)
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int64)
    return I.CSR(n=n, m=n, rowptr=rowptr, col=cols.astype(np.int32), val=d[rows, cols]), d


def test_fgmres_full_steps_solve_exactly():
    a, d = _nonsym(40, 1)
    b = I.uniform(40, seed=2).astype(np.float64)
    z, est = S.fgmres_steps(lambda v: d @ v, b, 40, lambda v: v)
    assert np.allclose(z, np.linalg.solve(d, b), rtol=1e-10, atol=1e-12)
    assert est[-1] < 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_fgmres_minimises_the_residual_over_the_krylov_space(k):
    """With the identity preconditioner, k steps give the minimal residual
    over K_k(A, b) (computed here from the explicit Krylov basis), and the
    estimate |g_k| is that residual."""
    a, d = _nonsym(30, 3)
    b = I.uniform(30, seed=4).astype(np.float64)
    z, est = S.fgmres_steps(lambda v: d @ v, b, k, lambda v: v)
    K = np.stack([np.linalg.matrix_power(d, i) @ b for i in range(k)], axis=1)
    Q, _ = np.linalg.qr(K)
    c, *_ = np.linalg.lstsq(d @ Q, b, rcond=None)
    rmin = np.linalg.norm(b - d @ Q @ c)
    assert np.linalg.norm(b - d @ z) == pytest.approx(rmin, rel=1e-8)
    assert est[k] == pytest.approx(rmin, rel=1e-8)


def test_fgmres_with_an_exact_preconditioner_converges_in_one_step():
    a, d = _nonsym(25, 5)
    b = I.uniform(25, seed=6).astype(np.float64)
    z, est = S.fgmres_steps(lambda v: d @ v, b, 3, lambda v: np.linalg.solve(d, v),
                            stop=lambda e: e < 1e-12)
    assert len(est) == 2
    assert np.allclose(z, np.linalg.solve(d, b), rtol=1e-10, atol=1e-12)


def test_richardson_closed_forms():
    a, d = _nonsym(20, 7)
    r = I.uniform(20, seed=8).astype(np.float64)
    A = lambda v: d @ v
    assert np.allclose(S.richardson(A, r, 1, 0.5), 0.5 * r)
    assert np.allclose(S.richardson(A, r, 2), 2 * r - d @ r)
    assert np.allclose(S.richardson(A, r, 3), 3 * r - 3 * (d @ r) + d @ (d @ r))


@pytest.mark.parametrize("mixed", [False, True])
def test_f3r_converges_on_a_nonsymmetric_system(mixed):
    a, d = _nonsym(300, 9)
    b = I.uniform(300, seed=10, lo=0.0, hi=1.0).astype(np.float64)
    val16 = O.quantize(a.val, O.FMT_FP16, 15)[1]
    x, it, hist = S.f3r(a, b, val16=val16, m1=10, m2=4, m3=3, m4=2, tol=1e-10, mixed=mixed)
    assert np.linalg.norm(b - d @ x) / np.linalg.norm(b) < 1e-10
    assert it <= 12
    assert np.allclose(x, np.linalg.solve(d, b), rtol=1e-7, atol=1e-9)
