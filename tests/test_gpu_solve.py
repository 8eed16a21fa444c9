"""GPU solvers vs the oracle (§5.2.2), through the C ABI.

FP64 Jacobi PCG must reach the same iteration count as the oracle's FP64 PCG
(same arithmetic up to summation order) and the same solution; IO-CG with an
FP32 inner PCG on PackSELL/SELL matrices must reach a true relative residual
below 1e-10 with an outer iteration count within 10 % (at least 2) of the
oracle's simulated-precision IO-CG.
"""
import numpy as np
import pytest

import oracle as O
from oracle import solvers as S
from paper_2604_13433_gb300 import inputs as I

from _gpu import FMT, P, dev, need_gpu, torch

pytestmark = pytest.mark.gpu


def encode(csr, fmt, D=15, **kw):
    return P().packsell_encode_csr(csr, fmt=fmt, D=D, **kw)


def diag_of(csr):
    row = np.repeat(np.arange(csr.n), csr.row_lengths())
    d = np.zeros(csr.n)
    on = csr.col == row
    d[row[on]] = csr.val[on]
    return d


def close_count(a, b, rel=0.10, floor=2):
    return abs(a - b) <= max(floor, rel * max(a, b))


@pytest.mark.parametrize("graph", [True, False])
def test_pcg_fp64_matches_oracle(graph):
    need_gpu()
    ps = P()
    a, _ = I.poisson5_varcoef(48, seed=1)
    b = I.uniform(a.n, seed=2).astype(np.float64)
    M = 1.0 / diag_of(a)
    xo, ito, _ = S.pcg(a, b, tol=1e-10, inv_diag=M)
    A64 = encode(a, "sell_f64")
    x, info = ps.packsell_pcg(A64, dev(b), inv_diag=dev(M), rtol=1e-10, max_iters=2000,
                              use_graph=graph, history=True)
    assert info["relres_true"] < 1e-10
    assert abs(info["iters"] - ito) <= 2
    assert np.allclose(x.cpu().numpy(), xo, rtol=1e-7, atol=1e-9)
    h = np.array(info["hist"])
    assert h[0] == pytest.approx(1.0) and h[-1] < 1e-10


@pytest.mark.parametrize("fmt,D,m_in,sigma", [("fp16", 15, 20, 256), ("e8my", 8, 20, 256),
                                              ("e8my", 11, 50, 256), ("sell_f32", 15, 20, 256),
                                              ("sell_f32", 15, 20, 1), ("fp16", 15, 20, 1)])
def test_iocg_matches_oracle(fmt, D, m_in, sigma):
    """IO-CG against the oracle's simulated-precision IO-CG; the inner
    product runs the pipelined fused SpMV + dot for PackSELL and FP32 SELL
    alike (7-point rows), with and without the sigma permutation."""
    need_gpu()
    ps = P()
    a = I.poisson7_varcoef(16, seed=3)  # unit diagonal (symmetrically scaled)
    b = I.uniform(a.n, seed=4).astype(np.float64)
    deq = a.val if fmt == "sell_f32" else O.encode(a, D=D, fmt=FMT[fmt]).deq
    if fmt == "sell_f32":
        deq = a.val.astype(np.float32).astype(np.float64)
    xo, ko, _ = S.iocg(a, b, deq, m_in=m_in, tol=1e-10, max_outer=300)
    A64 = encode(a, "sell_f64")
    Ain = encode(a, fmt, D=D, sigma=sigma) if fmt != "sell_f32" else P().packsell_encode_csr(
        I.CSR(n=a.n, m=a.m, rowptr=a.rowptr, col=a.col, val=a.val.astype(np.float32)),
        fmt="sell_f32", sigma=sigma)
    x, info = ps.packsell_pcg(A64, dev(b), A_inner=Ain, m_in=m_in, rtol=1e-10, max_iters=300)
    assert info["relres_true"] < 1e-10
    assert close_count(info["iters"], ko), (info["iters"], ko)
    assert info["inner_iters"] == m_in * info["iters"]
    r = b - O.csr_spmv_f64(a, a.val, x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-10


def test_iocg_with_jacobi_and_known_solution():
    need_gpu()
    ps = P()
    a, _ = I.poisson5_varcoef(96, seed=5)  # unscaled: Jacobi inside the inner PCG
    xs = I.normal(a.n, seed=6)
    b = O.csr_spmv_f64(a, a.val, xs)
    M = 1.0 / diag_of(a)
    A64 = encode(a, "sell_f64")
    Ain = encode(a, "e8my", D=10)
    x, info = ps.packsell_pcg(A64, dev(b), A_inner=Ain, inv_diag=dev(M), m_in=30, rtol=1e-10,
                              max_iters=500)
    assert info["relres_true"] < 1e-10
    assert np.allclose(x.cpu().numpy(), xs, rtol=1e-6, atol=1e-6)


def test_solve_deterministic_and_workspace():
    need_gpu()
    ps = P()
    a = I.poisson7_varcoef(20, seed=7)
    b = dev(I.uniform(a.n, seed=8).astype(np.float64))
    A64, Ain = encode(a, "sell_f64"), encode(a, "fp16")
    x1, i1 = ps.packsell_pcg(A64, b, A_inner=Ain, m_in=20)
    x2, i2 = ps.packsell_pcg(A64, b, A_inner=Ain, m_in=20, use_graph=False)
    nb = ps.packsell_pcg_workspace_bytes(a.n, 20, False, 1000)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    x3, i3 = ps.packsell_pcg(A64, b, A_inner=Ain, m_in=20, workspace=ws)
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    assert i1["iters"] == i2["iters"] == i3["iters"]
    with pytest.raises(ps.PackSELLError) as e:
        ps.packsell_pcg(A64, b, A_inner=Ain, m_in=20, workspace=ws[: nb // 2])
    assert e.value.code == 1


def test_solve_statuses():
    need_gpu()
    ps = P()
    a = I.poisson7_varcoef(12, seed=9)
    b = dev(I.uniform(a.n, seed=10).astype(np.float64))
    A64 = encode(a, "sell_f64")
    x, info = ps.packsell_pcg(A64, b, rtol=1e-14, max_iters=3, check=False)
    assert info["status"] == "NOT_CONVERGED" and info["iters"] == 3
    neg = I.CSR(n=a.n, m=a.m, rowptr=a.rowptr, col=a.col, val=-a.val)  # negative definite
    with pytest.raises(ps.PackSELLError) as e:
        ps.packsell_pcg(encode(neg, "sell_f64"), b, max_iters=50)
    assert e.value.status == "BREAKDOWN"
    # zero right-hand side: converged at once with x = 0
    z = torch.zeros_like(b)
    x, info = ps.packsell_pcg(A64, z)
    assert info["iters"] == 0 and torch.count_nonzero(x) == 0
