"""Locality reordering (reverse Cuthill-McKee, §7's future work) through the
GPU path: the reordered matrix encodes, its SpMV is bit for bit the oracle's
twin of the permuted matrix, IO-CG on the reordered system gives the
original system's solution, and on power-law rows the reordering cuts SELL
padding at sigma = 256."""
import numpy as np
import pytest

import oracle as O
import oracle.solvers as S
from paper_2604_13433_gb300 import inputs as I

from _gpu import P, dev, need_gpu, torch

pytestmark = pytest.mark.gpu


def _permuted(ps, csr):
    perm = ps.packsell_reorder_rcm(csr.rowptr, csr.col)
    rp, cl, vl = ps.packsell_permute_csr(csr.rowptr, csr.col, csr.val, perm)
    return perm, I.CSR(n=csr.n, m=csr.m, rowptr=rp, col=cl, val=vl)


def test_reordered_spmv_and_iocg_solve_the_original_system():
    need_gpu()
    ps = P()
    a = I.poisson7_varcoef(20, seed=31)
    perm, b_csr = _permuted(ps, a)
    enc = O.encode(b_csr, C=32, sigma=256, D=15, fmt=O.FMT_FP16)
    B = ps.packsell_encode_csr(b_csr, fmt="fp16", D=15)
    x = I.uniform(a.n, seed=32)
    y = ps.packsell_spmv(B, dev(x)).cpu().numpy()
    twin = O.csr_spmv_fma_f32(b_csr, enc.deq.astype(np.float32), x)
    assert np.array_equal(y.view(np.uint32), twin.view(np.uint32))
    # solve with the reordered operators, then scatter back: the original solution
    rhs = I.uniform(a.n, seed=33).astype(np.float64)
    B64 = ps.packsell_encode_csr(b_csr, fmt="sell_f64")
    xr, info = ps.packsell_pcg(B64, dev(rhs[perm]), A_inner=B, m_in=20, rtol=1e-10, max_iters=300)
    assert info["relres_true"] < 1e-10
    xo = np.empty(a.n)
    xo[perm] = xr.cpu().numpy()
    r = rhs - O.csr_spmv_f64(a, a.val, xo)
    assert np.linalg.norm(r) / np.linalg.norm(rhs) < 1e-10


def test_reordering_cuts_sell_padding_on_power_law_rows():
    need_gpu()
    ps = P()
    a = I.zipf_irregular(50000, seed=34)
    perm, b_csr = _permuted(ps, a)
    A = ps.packsell_encode_csr(a, fmt="fp16", D=15, sigma=256)
    B = ps.packsell_encode_csr(b_csr, fmt="fp16", D=15, sigma=256)
    assert B.n_words < 0.7 * A.n_words
    enc = O.encode(b_csr, C=32, sigma=256, D=15, fmt=O.FMT_FP16)
    assert B.n_words == enc.n_words
    x = I.uniform(a.n, seed=35)
    y = ps.packsell_spmv(B, dev(x)).cpu().numpy()
    twin = O.csr_spmv_fma_f32(b_csr, enc.deq.astype(np.float32), x)
    assert np.array_equal(y.view(np.uint32), twin.view(np.uint32))
