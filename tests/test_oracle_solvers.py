"""Pins for the oracle's solvers (§5.2.2) and adjoint gradients.

Independent references: dense solves (numpy.linalg), the closed-form
eigenvalues of the constant-coefficient 2-D Laplacian (CG convergence bound),
the equivalence of FCG with a one-step inner PCG to Jacobi PCG, one-step
convergence with an exact inner solve, and central finite differences.
"""
import numpy as np
import pytest

import oracle as O
from oracle import solvers as S
from paper_2604_13433_gb300 import inputs as I


def _dense(csr, val=None):
    val = csr.val if val is None else val
    A = np.zeros((csr.n, csr.m))
    A[np.repeat(np.arange(csr.n), csr.row_lengths()), csr.col] = val
    return A


def test_pcg_known_solution_and_dense():
    a, _ = I.poisson5_varcoef(20, seed=1)
    xs = I.normal(a.n, seed=2)
    b = O.csr_spmv_f64(a, a.val, xs)
    d = _dense(a)
    inv_diag = 1.0 / np.diag(d)
    x, it, hist = S.pcg(a, b, tol=1e-12, inv_diag=inv_diag)
    assert hist[-1] < 1e-12
    assert np.linalg.norm(b - d @ x) / np.linalg.norm(b) < 1e-12
    assert np.allclose(x, np.linalg.solve(d, b), rtol=1e-9, atol=1e-9)
    assert np.allclose(x, xs, rtol=1e-8, atol=1e-8)


def test_cg_iterations_within_chebyshev_bound():
    # 2-D Laplacian on L x L: eigenvalues 4 - 2cos(j pi/(L+1)) - 2cos(k pi/(L+1));
    # ||r_k|| / ||r_0|| <= 2 sqrt(kappa) ((sqrt(kappa)-1)/(sqrt(kappa)+1))^k
    L = 40
    a = I.poisson5(L, dtype=np.float64)
    t = np.pi / (L + 1)
    lmin, lmax = 4 - 4 * np.cos(t), 4 - 4 * np.cos(L * t)
    kappa = lmax / lmin
    tol = 1e-10
    sk = np.sqrt(kappa)
    bound = np.log(2 * sk / tol) / np.log((sk + 1) / (sk - 1))
    b = I.uniform(a.n, seed=3).astype(np.float64)
    x, it, hist = S.pcg(a, b, tol=tol)
    assert it <= np.ceil(bound)
    d = _dense(a)
    assert np.linalg.norm(b - d @ x) / np.linalg.norm(b) < tol


def test_pcg_a_norm_error_decreases():
    a, _ = I.poisson5_varcoef(12, seed=4)
    d = _dense(a)
    b = I.uniform(a.n, seed=5).astype(np.float64)
    xs = np.linalg.solve(d, b)
    errs = []
    for k in range(1, 30):
        x, _, _ = S.pcg(a, b, tol=0.0, maxit=k, inv_diag=1 / np.diag(d))
        e = x - xs
        errs.append(e @ d @ e)
    assert np.all(np.diff(errs) < 0)


def test_iocg_one_step_inner_equals_pcg():
    # With one inner PCG step from zero, z = alpha0 * M r: a positive multiple
    # of the Jacobi-preconditioned residual. FCG is invariant to the scale of
    # z, so its iterates are those of Jacobi PCG.
    a, _ = I.poisson5_varcoef(10, seed=6)
    d = _dense(a)
    M = 1 / np.diag(d)
    b = I.uniform(a.n, seed=7).astype(np.float64)

    def inner(r):
        z = M * r
        q = d @ z
        return ((r @ z) / (z @ q)) * z

    for k in (1, 5, 12):
        x1, _, _ = S.pcg(a, b, tol=0.0, maxit=k, inv_diag=M)
        x2, _, _ = S.iocg(a, b, None, tol=0.0, max_outer=k, inner=inner)
        assert np.allclose(x1, x2, rtol=1e-10, atol=1e-12)


def test_iocg_exact_inner_converges_in_one_step():
    a, _ = I.poisson5_varcoef(10, seed=8)
    d = _dense(a)
    b = I.uniform(a.n, seed=9).astype(np.float64)
    x, k, hist = S.iocg(a, b, None, tol=1e-12, max_outer=5,
                        inner=lambda r: np.linalg.solve(d, r))
    assert k == 1
    assert np.linalg.norm(b - d @ x) / np.linalg.norm(b) < 1e-12


@pytest.mark.parametrize("fmt,D", [(O.FMT_FP16, 15), (O.FMT_E8MY, 8)])
def test_iocg_mixed_precision_reaches_1e10(fmt, D):
    a = I.poisson7_varcoef(12, seed=10)
    b = I.uniform(a.n, seed=11).astype(np.float64)
    e = O.encode(a, C=32, sigma=256, D=D, fmt=fmt)
    x, k, hist = S.iocg(a, b, e.deq, m_in=20, tol=1e-10, max_outer=200)
    r = b - O.csr_spmv_f64(a, a.val, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-10
    assert k < 200


def _solve(csr, val, b):
    return np.linalg.solve(_dense(csr, val), b)


def test_adjoint_grads_match_finite_differences():
    L = 6
    a, faces = I.poisson5_varcoef(L, seed=12)
    b = I.uniform(a.n, seed=13).astype(np.float64)
    xt = I.normal(a.n, seed=14)
    theta = faces["theta"].copy()

    def assemble(th):
        v = np.zeros(a.nnz)
        F = faces["u"].size
        np.add.at(v, faces["pos_uu"], th[:F])
        np.add.at(v, faces["pos_vv"], th[:F])
        np.add.at(v, faces["pos_uv"], -th[:F])
        np.add.at(v, faces["pos_vu"], -th[:F])
        np.add.at(v, faces["pos_b"], th[F:])
        return v

    assert np.allclose(assemble(theta), a.val)

    def loss(th, bb):
        x = _solve(a, assemble(th), bb)
        return float(np.sum((x - xt) ** 2))

    x = _solve(a, a.val, b)
    g = 2 * (x - xt)
    lam, dval = S.adjoint_grads(a, x, g)
    # dL/db = lam = A^-T g (dense check, and FD)
    assert np.allclose(lam, np.linalg.solve(_dense(a).T, g), rtol=1e-9, atol=1e-11)
    gth = S.face_grads(faces, dval)
    rng = np.random.default_rng(15)
    for f in rng.choice(theta.size, 8, replace=False):
        h = 1e-6 * abs(theta[f])
        tp, tm = theta.copy(), theta.copy()
        tp[f] += h
        tm[f] -= h
        fd = (loss(tp, b) - loss(tm, b)) / (2 * h)
        assert np.isclose(gth[f], fd, rtol=1e-5, atol=1e-8)
    for i in rng.choice(a.n, 5, replace=False):
        h = 1e-6
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (loss(theta, bp) - loss(theta, bm)) / (2 * h)
        assert np.isclose(lam[i], fd, rtol=1e-5, atol=1e-8)


# --------------------------------------------------------------------------
# the inner solve of IO-CG (§5.2.2), pinned against independent references
# --------------------------------------------------------------------------
def _inner_case(seed):
    a, _ = I.poisson5_varcoef(6, seed=seed)  # 36 unknowns, SPD
    e = O.encode(a, C=32, sigma=256, D=15, fmt=O.FMT_FP16)
    d = _dense(a, e.deq)
    r = I.uniform(a.n, seed=seed + 1).astype(np.float64) * 3.0
    return a, e.deq, d, r


@pytest.mark.parametrize("jacobi", [False, True])
def test_inner_pcg_without_rounding_is_an_exact_solve(jacobi):
    """With the float32 rounding taken out and m_in = n, CG on an SPD system
    of n unknowns reaches the solution (finite termination, §5.2.2's CG):
    the result must equal the dense solve of q(A) z = r to rounding. A wrong
    alpha, beta or rescaling does not terminate at the solution."""
    a, deq, d, r = _inner_case(40)
    M = 1.0 / np.diag(d) if jacobi else None
    z = S.inner_pcg_f32(a, deq, r, a.n, inv_diag=M, dtype=np.float64)
    ref = np.linalg.solve(d, r)
    assert np.allclose(z, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_inner_pcg_iterates_follow_fp64_pcg(k):
    """Its first k iterates are those of the FP64 Jacobi PCG (pinned on its
    own above) started from zero on r / ||r||, scaled by ||r||, up to float32
    rounding; in double precision they agree to rounding of double."""
    a, deq, d, r = _inner_case(41)
    M = 1.0 / np.diag(d)
    s = np.linalg.norm(r)
    ref, _, _ = S.pcg(a, r / s, tol=0.0, maxit=k, inv_diag=M, val=deq)
    ref = ref * s
    z32 = S.inner_pcg_f32(a, deq, r, k, inv_diag=M)
    z64 = S.inner_pcg_f32(a, deq, r, k, inv_diag=M, dtype=np.float64)
    scale = np.abs(ref).max()
    assert np.abs(z64 - ref).max() <= 1e-12 * scale
    err32 = np.abs(z32 - ref).max()
    assert err32 <= 2e-5 * scale
    assert err32 > 0.0  # the float32 rounding is really simulated
