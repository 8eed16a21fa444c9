"""Differentiation through PackSELL products and solves (a11), against the
oracle's FP64 adjoint formulas and central finite differences."""
import numpy as np
import pytest

import oracle as O
from oracle import solvers as S
from paper_2604_13433_gb300 import inputs as I

from _gpu import FMT, P, dev, need_gpu, torch

pytestmark = pytest.mark.gpu


def AG():
    P()
    from paper_2604_13433_gb300 import autograd
    return autograd


def _dense(csr, val):
    A = np.zeros((csr.n, csr.m))
    A[np.repeat(np.arange(csr.n), csr.row_lengths()), csr.col] = val
    return A


@pytest.mark.parametrize("fmt,D", [("fp16", 15), ("e8my", 5)])
def test_spmv_backward(fmt, D):
    need_gpu()
    ps, ag = P(), AG()
    csr = I.random_csr(300, 250, 0.03, seed=3, empty_rows=0.05, long_gaps=True)
    A = ps.packsell_encode_csr(csr, fmt=fmt, D=D, sigma=64, keep_rowptr=True)
    deq = O.encode(csr, C=32, sigma=64, D=D, fmt=FMT[fmt]).deq
    val = dev(csr.val).requires_grad_(True)
    x = dev(I.uniform(250, seed=4)).requires_grad_(True)
    w = I.uniform(300, seed=5)
    y = ag.spmv(A, x, val)
    (y * dev(w)).sum().backward()
    dense = _dense(csr, deq)
    dx_ref = dense.T @ w.astype(np.float64)
    assert np.allclose(x.grad.cpu().numpy(), dx_ref, rtol=1e-5, atol=1e-5)
    row = np.repeat(np.arange(300), csr.row_lengths())
    dval_ref = (w[row] * x.detach().cpu().numpy()[csr.col]).astype(np.float32)
    assert np.array_equal(val.grad.cpu().numpy(), dval_ref)


def _face_model(faces, csr):
    """theta -> CSR values of A = sum_f theta_f (e_u-e_v)(e_u-e_v)^T + boundary terms
    (the user's model, ordinary torch ops)."""
    F = faces["u"].size
    idx = {k: dev(faces[k]) for k in ("pos_uu", "pos_vv", "pos_uv", "pos_vu", "pos_b")}

    def assemble(theta):
        v = torch.zeros(csr.nnz, dtype=theta.dtype, device=theta.device)
        tf, tb = theta[:F], theta[F:]
        v = v.index_add(0, idx["pos_uu"], tf).index_add(0, idx["pos_vv"], tf)
        v = v.index_add(0, idx["pos_uv"], -tf).index_add(0, idx["pos_vu"], -tf)
        return v.index_add(0, idx["pos_b"], tb)

    return assemble


@pytest.mark.parametrize("m_in,fmt,D", [(0, "fp16", 15), (10, "fp16", 15), (10, "e8my", 9)])
def test_solve_gradients_match_oracle_and_fd(m_in, fmt, D):
    need_gpu()
    ag = AG()
    L = 10
    csr, faces = I.poisson5_varcoef(L, seed=11)
    b_h = I.uniform(csr.n, seed=12).astype(np.float64)
    xt_h = I.normal(csr.n, seed=13)
    assemble = _face_model(faces, csr)
    theta = dev(faces["theta"]).requires_grad_(True)
    b = dev(b_h).requires_grad_(True)
    rp, cl = dev(csr.rowptr), dev(csr.col)
    x = ag.solve(rp, cl, assemble(theta), b, m_in=m_in, fmt=fmt, D=D, rtol=1e-12)
    loss = ((x - dev(xt_h)) ** 2).sum()
    loss.backward()
    # oracle: dense solve, adjoint formulas
    A = _dense(csr, csr.val)
    xs = np.linalg.solve(A, b_h)
    g = 2 * (xs - xt_h)
    lam = np.linalg.solve(A.T, g)
    row = np.repeat(np.arange(csr.n), csr.row_lengths())
    dval = -lam[row] * xs[csr.col]
    dth_ref = S.face_grads(faces, dval)
    assert np.allclose(x.detach().cpu().numpy(), xs, rtol=1e-9, atol=1e-10)
    assert np.allclose(b.grad.cpu().numpy(), lam, rtol=1e-8, atol=1e-10)
    assert np.allclose(theta.grad.cpu().numpy(), dth_ref, rtol=1e-7, atol=1e-10)
    # central finite differences on a few faces (FP64 dense solves)
    th = faces["theta"]
    rng = np.random.default_rng(14)
    for f in rng.choice(th.size, 4, replace=False):
        h = 1e-6 * th[f]
        vals = []
        for sgn in (1, -1):
            t2 = th.copy()
            t2[f] += sgn * h
            v2 = assemble(dev(t2)).cpu().numpy()
            x2 = np.linalg.solve(_dense(csr, v2), b_h)
            vals.append(np.sum((x2 - xt_h) ** 2))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert np.isclose(theta.grad[f].item(), fd, rtol=1e-5, atol=1e-8)


def test_backward_entry_points():
    """packsell_spmv_backward and packsell_pcg_backward called directly: either
    output alone, agreement with the calls they compose, and the keep_rowptr
    requirement refused before anything is written."""
    need_gpu()
    ps = P()
    csr = I.random_csr(200, 180, 0.04, seed=21)
    A = ps.packsell_encode_csr(csr, fmt="fp16", keep_rowptr=True)
    x = dev(I.uniform(180, seed=22))
    dy = dev(I.uniform(200, seed=23))
    dx, dval = ps.packsell_spmv_backward(A, x, dy)
    dx_only, none1 = ps.packsell_spmv_backward(A, x, dy, need_dval=False)
    none2, dval_only = ps.packsell_spmv_backward(A, x, dy, need_dx=False)
    assert none1 is None and none2 is None
    assert torch.equal(dval, dval_only)
    row = np.repeat(np.arange(200), csr.row_lengths())
    dy_h, x_h = dy.cpu().numpy(), x.cpu().numpy()
    assert np.array_equal(dval.cpu().numpy(), (dy_h[row] * x_h[csr.col]).astype(np.float32))
    deq = O.encode(csr, C=32, sigma=256, D=15, fmt=O.FMT_FP16).deq
    dx_ref = _dense(csr, deq).T @ dy_h.astype(np.float64)
    for d in (dx, dx_only):  # atomic adds: compared within FP32 rounding
        assert np.allclose(d.cpu().numpy(), dx_ref, rtol=1e-5, atol=1e-5)
    B = ps.packsell_encode_csr(csr, fmt="fp16")  # no keep_rowptr
    with pytest.raises(ps.PackSELLError) as e:
        ps.packsell_spmv_backward(B, x, dy)
    assert e.value.code == 1

    a, _ = I.poisson5_varcoef(12, seed=24)
    A64 = ps.packsell_encode_csr(a, fmt="sell_f64", keep_rowptr=True)
    b = dev(I.uniform(a.n, seed=25).astype(np.float64))
    xs, _ = ps.packsell_pcg(A64, b, rtol=1e-12)
    g = dev(I.normal(a.n, seed=26))
    lam_ref, _ = ps.packsell_pcg(A64, g, rtol=1e-12)
    lam, dA, info = ps.packsell_pcg_backward(A64, xs, g, rtol=1e-12)
    assert info["status"] == "OK"
    assert torch.equal(lam, lam_ref)  # the same solve from zero
    assert torch.equal(dA, ps.packsell_pattern_outer_f64(A64, -1.0, lam_ref, xs))
    lam2, none3, _ = ps.packsell_pcg_backward(A64, xs, g, rtol=1e-12, need_dA=False)
    assert none3 is None and torch.equal(lam2, lam_ref)
    A64n = ps.packsell_encode_csr(a, fmt="sell_f64")  # no keep_rowptr
    with pytest.raises(ps.PackSELLError) as e:
        ps.packsell_pcg_backward(A64n, xs, g, rtol=1e-12)
    assert e.value.code == 1
