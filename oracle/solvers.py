"""Oracle solvers: Jacobi PCG, inner-outer CG and adjoints, in numpy.

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).

* :func:`pcg` - preconditioned CG in double precision with a Jacobi
  (diagonal) preconditioner; the FP64 PCG baseline of §5.2.2.
* :func:`iocg` - the inner-outer CG of §5.2.2: flexible CG in double
  precision whose preconditioner is ``m_in`` iterations of PCG run in single
  precision (simulated: every inner vector is stored as float32 and every inner
  dot product is accumulated in double) with the quantised matrix.
* :func:`adjoint_grads` - gradients of a loss of the solution of A x = b with
  respect to b and to the matrix entries on the sparsity pattern, from one
  adjoint solve A^T lam = dL/dx.

Readings where the paper is silent (§5.2.2 gives the scheme, not the details):
the outer method is flexible CG with truncation 1 (one previous direction,
Notay's FCG(1)); the inner solve starts from zero, takes exactly ``m_in``
iterations, and works on the outer residual divided by its 2-norm (scaled
back afterwards); convergence is declared on the true residual
||b - A x||_2 / ||b||_2 recomputed in double precision.
"""
from __future__ import annotations

import numpy as np

from . import csr_spmv_f64


def _dot(a, b) -> float:
    return float(np.dot(np.asarray(a, np.float64), np.asarray(b, np.float64)))


def pcg(A, b, x0=None, tol=1e-10, maxit=10000, inv_diag=None, val=None):
    """Jacobi-preconditioned CG in double precision.

    ``A`` is a CSR (values ``val`` or ``A.val``). Returns (x, iters, hist) with
    hist[k] = ||r_k||_2 / ||b||_2 of the recurrence residual; on reaching tol
    the true residual is recomputed, and the iteration continues from it if
    it is not yet below tol.
    """
    val = A.val if val is None else val
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    M = np.ones_like(b) if inv_diag is None else np.asarray(inv_diag, np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    r = b - csr_spmv_f64(A, val, x)
    z = M * r
    p = z.copy()
    rz = _dot(r, z)
    hist = [np.linalg.norm(r) / nb]
    it = 0
    while it < maxit:
        if hist[-1] < tol:
            rt = b - csr_spmv_f64(A, val, x)
            if np.linalg.norm(rt) / nb < tol:
                break
            r = rt
            z = M * r
            p = z.copy()
            rz = _dot(r, z)
        q = csr_spmv_f64(A, val, p)
        pq = _dot(p, q)
        if pq <= 0.0:
            raise FloatingPointError("pcg: p^T A p <= 0 (matrix not SPD)")
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / nb)
        z = M * r
        rz_new = _dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def inner_pcg_f32(A, deq, r, m_in, inv_diag=None, dtype=np.float32):
    """m_in PCG iterations on A z = r from z = 0 in simulated single precision.

    The right-hand side is r / ||r||_2 (rounded to float32); the result is
    scaled back by ||r||_2 in double. Vectors are float32, dot products are
    accumulated in double, scalars alpha and beta are rounded to float32 before
    they scale a vector, and A v is the quantised matrix applied in double and
    rounded to float32. ``dtype`` is the working precision of the vectors and
    scalars (float32 for the inner solve of §5.2.2; float64 takes the
    rounding out, so the same steps are plain CG in double precision).
    """
    dt = np.dtype(dtype).type
    s = float(np.linalg.norm(r))
    if s == 0.0:
        return np.zeros_like(r, dtype=np.float64)
    rr = (np.asarray(r, np.float64) / s).astype(dt)
    M = None if inv_diag is None else np.asarray(inv_diag, dt)
    xx = np.zeros_like(rr)
    z = rr if M is None else (M * rr).astype(dt)
    p = z.copy()
    rz = _dot(rr, z)
    for _ in range(m_in):
        if rz == 0.0:
            break
        q = csr_spmv_f64(A, deq, p).astype(dt)
        pq = _dot(p, q)
        if pq <= 0.0:
            break
        a = dt(rz / pq)
        xx = (xx + a * p).astype(dt)
        rr = (rr - a * q).astype(dt)
        z = rr if M is None else (M * rr).astype(dt)
        rz_new = _dot(rr, z)
        bta = dt(rz_new / rz)
        p = (z + bta * p).astype(dt)
        rz = rz_new
    return xx.astype(np.float64) * s


def iocg(A, b, deq, m_in=20, tol=1e-10, max_outer=1000, x0=None, inv_diag=None,
         val64=None, inner=None):
    """Inner-outer CG (§5.2.2): FCG(1) in double, preconditioned by m_in
    single-precision PCG iterations on the quantised matrix ``deq``.

    ``inner`` may replace the inner solve (a callable r -> z) for tests.
    Returns (x, outer_iters, hist) with hist[k] the outer recurrence relative
    residual after outer iteration k.
    """
    val64 = A.val if val64 is None else val64
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    r = b - csr_spmv_f64(A, val64, x)
    hist = [np.linalg.norm(r) / nb]
    p_prev = q_prev = None
    pq_prev = 0.0
    k = 0
    solve = inner if inner is not None else (lambda v: inner_pcg_f32(A, deq, v, m_in, inv_diag))
    while k < max_outer:
        if hist[-1] < tol:
            rt = b - csr_spmv_f64(A, val64, x)
            if np.linalg.norm(rt) / nb < tol:
                break
            r = rt
            p_prev = None
        z = solve(r)
        if p_prev is None:
            p = z
        else:
            p = z - (_dot(z, q_prev) / pq_prev) * p_prev
        q = csr_spmv_f64(A, val64, p)
        pq = _dot(p, q)
        if pq <= 0.0:
            raise FloatingPointError("iocg: p^T A p <= 0")
        alpha = _dot(p, r) / pq
        x += alpha * p
        r -= alpha * q
        k += 1
        hist.append(np.linalg.norm(r) / nb)
        p_prev, q_prev, pq_prev = p, q, pq
    return x, k, hist


def adjoint_grads(A, x, g, val=None, tol=1e-13, inv_diag=None):
    """For x = A^-1 b and a loss with dL/dx = g: lam = A^-T g (A symmetric
    here, so one PCG solve), dL/db = lam and dL/da_ij = -lam_i x_j on the
    pattern of A (CSR order)."""
    val = A.val if val is None else val
    lam, _, _ = pcg(A, g, tol=tol, maxit=100000, inv_diag=inv_diag, val=val)
    row = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    dval = -lam[row] * np.asarray(x, np.float64)[A.col]
    return lam, dval


def face_grads(faces, dval):
    """Chain dL/dA on the pattern to the face coefficients of
    A = sum_f theta_f (e_u - e_v)(e_u - e_v)^T + sum_b theta_b e_b e_b^T:
    dL/dtheta_f = dA_uu + dA_vv - dA_uv - dA_vu, dL/dtheta_b = dA_bb."""
    gf = (dval[faces["pos_uu"]] + dval[faces["pos_vv"]] - dval[faces["pos_uv"]]
          - dval[faces["pos_vu"]])
    gb = dval[faces["pos_b"]]
    return np.concatenate([gf, gb])


# --------------------------------------------------------------------------
# F3R (§5.2.1): three layers of flexible GMRES and an innermost Richardson
# --------------------------------------------------------------------------
# Readings where the paper is silent (it names the layers and which of them
# use the FP16 SpMV, and takes the rest from the solver's own paper): the
# outer layer is restarted FGMRES(m1) in double precision; layers 2 and 3 run
# exactly m2 and m3 FGMRES steps from zero; layer 4 runs m4 Richardson steps
# z <- z + omega (r - A z) from z = 0; the Jacobi preconditioner is the
# identity on symmetrically scaled matrices; Krylov bases by classical
# Gram-Schmidt; in the FP16-enabled form layers 2-4 keep their vectors in
# float32, layer 2 applies A with float32 values and layers 3-4 with the
# FP16-quantised values (each product rounded once to float32); dot products,
# Hessenberg entries and Givens rotations in double.

def _rnd(v, dt):
    """v rounded to the working precision dt (float32 or float64), as double."""
    return np.asarray(v, np.float64).astype(dt).astype(np.float64)


def fgmres_steps(apply_a, rhs, m, precond, dt=np.float64, stop=None):
    """Up to m steps of flexible GMRES from zero on A z = rhs (Saad's FGMRES:
    Arnoldi on the preconditioned directions z_j = M_j(v_j), the small
    least-squares problem min ||beta e_1 - H y|| by Givens rotations, z =
    sum_j y_j z_j). Vectors are kept in precision dt. ``stop(est)`` may end the
    loop early on the residual estimate |g_{j+1}|. Returns (z, estimates)."""
    rhs = _rnd(rhs, dt)
    beta = np.sqrt(_dot(rhs, rhs))
    if beta == 0.0:
        return np.zeros_like(rhs), [0.0]
    V = [_rnd(rhs / beta, dt)]
    Z = []
    H = np.zeros((m + 1, m))
    cs, sn = np.zeros(m), np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    est = [beta]
    k = 0
    for j in range(m):
        Z.append(_rnd(precond(V[j]), dt))
        w = _rnd(apply_a(Z[j]), dt)
        h = np.array([_dot(w, V[i]) for i in range(j + 1)])  # classical Gram-Schmidt
        w = _rnd(w - sum(h[i] * V[i] for i in range(j + 1)), dt)
        hn = np.sqrt(_dot(w, w))
        H[:j + 1, j] = h
        H[j + 1, j] = hn
        for i in range(j):  # earlier rotations on the new column
            a, bb = H[i, j], H[i + 1, j]
            H[i, j], H[i + 1, j] = cs[i] * a + sn[i] * bb, -sn[i] * a + cs[i] * bb
        r = np.hypot(H[j, j], H[j + 1, j])
        cs[j], sn[j] = (H[j, j] / r, H[j + 1, j] / r) if r > 0 else (1.0, 0.0)
        H[j, j], H[j + 1, j] = r, 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        V.append(_rnd(w * (1.0 / hn if hn > 0 else 0.0), dt))
        k = j + 1
        est.append(abs(g[j + 1]))
        if stop is not None and stop(abs(g[j + 1])):
            break
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):  # back substitution on the rotated H
        t = g[i] - H[i, i + 1:k] @ y[i + 1:k]
        y[i] = t / H[i, i] if H[i, i] != 0 else 0.0
    z = sum(y[i] * Z[i] for i in range(k))
    return np.asarray(z, np.float64), est


def richardson(apply_a, r, steps, omega=1.0, dt=np.float64):
    """``steps`` Richardson steps z <- z + omega (r - A z) from z = 0 (the
    first one gives z = omega r), vectors in precision dt."""
    r = _rnd(r, dt)
    z = _rnd(omega * r, dt)
    for _ in range(steps - 1):
        z = _rnd(z + omega * (r - _rnd(apply_a(z), dt)), dt)
    return z


def f3r(A, b, val16=None, m1=30, m2=8, m3=4, m4=2, omega=1.0, tol=1e-9, max_iters=300,
        x0=None, mixed=True):
    """F3R (§5.2.1). mixed=True: the FP16-enabled form (layer 2 with float32
    values and vectors, layers 3 and 4 with the FP16-quantised values
    ``val16`` and float32 vectors); mixed=False: every layer in double with
    A.val. Layer 1 stops on its residual estimate and confirms on the true
    residual (restarting from it otherwise). Returns (x, outer steps,
    estimates)."""
    b = np.asarray(b, np.float64)
    dt = np.float32 if mixed else np.float64
    v64 = np.asarray(A.val, np.float64)
    v32 = v64.astype(np.float32).astype(np.float64) if mixed else v64
    v16 = np.asarray(val16, np.float64) if mixed else v64
    a1 = lambda v: csr_spmv_f64(A, v64, v)
    a2 = lambda v: csr_spmv_f64(A, v32, v)
    a3 = lambda v: csr_spmv_f64(A, v16, v)
    layer4 = lambda r: richardson(a3, r, m4, omega, dt)
    layer3 = lambda r: _rnd(fgmres_steps(a3, r, m3, layer4, dt)[0], dt)
    layer2 = lambda r: fgmres_steps(a2, r, m2, layer3, dt)[0]
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, [0.0]
    it, hist = 0, []
    while it < max_iters:
        r = b - a1(x)
        if np.linalg.norm(r) / nb < tol:
            break
        left = max_iters - it
        z, est = fgmres_steps(a1, r, min(m1, left), layer2, np.float64,
                              stop=lambda e: e / nb < tol)
        x = x + z
        it += len(est) - 1
        hist += [e / nb for e in est[1:]]
    return x, it, hist
