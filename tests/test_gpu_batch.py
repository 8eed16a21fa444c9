"""Batched SpMV (one persistent launch over many matrices) vs per-matrix
packsell_spmv (same bits) and the oracle's FP32 twin."""
import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I

from _gpu import FMT, P, dev, need_gpu, torch

pytestmark = pytest.mark.gpu


def test_batch_matches_single_spmv_and_twin():
    need_gpu()
    ps = P()
    rng = np.random.default_rng(0)
    mats, csrs, xs, ys, specs = [], [], [], [], []
    for i in range(40):
        n = int(rng.integers(1, 3000))
        m = int(rng.integers(1, 3000))
        csr = I.random_csr(n, m, float(rng.uniform(0.001, 0.02)), seed=i, empty_rows=0.05,
                           long_gaps=bool(i % 2))
        fmt, D = ("fp16", 15) if i % 3 == 0 else ("e8my", int(rng.integers(1, 16)))
        sigma = [1, 32, 256, 1000][i % 4]
        A = ps.packsell_encode_csr(csr, fmt=fmt, D=D, sigma=sigma, explicit_perm=(i % 5 == 0))
        mats.append(A)
        csrs.append(csr)
        specs.append((fmt, D, sigma, i % 5 == 0))
        xs.append(dev(I.uniform(m, seed=100 + i)))
        ys.append(torch.full((n,), float("nan"), device="cuda"))
    # a large stencil too, so items split matrices
    big = I.stencil27(40, seed=1)
    mats.append(ps.packsell_encode_csr(big, fmt="e8my", D=11))
    csrs.append(big)
    specs.append(("e8my", 11, 256, False))
    xs.append(dev(I.uniform(big.m, seed=7)))
    ys.append(torch.empty(big.n, device="cuda"))
    B = ps.packsell_batch_create(mats, xs, ys)
    assert B.items >= len(mats)
    B.spmv()
    torch.cuda.synchronize()
    for A, csr, x, y, (fmt, D, sigma, expl) in zip(mats, csrs, xs, ys, specs):
        ref = ps.packsell_spmv(A, x)
        assert torch.equal(y.view(torch.int32), ref.view(torch.int32))
    # spot-check a few against the oracle twin
    for j in (0, 7, len(mats) - 1):
        fmt, D, sigma, expl = specs[j]
        enc = O.encode(csrs[j], C=32, sigma=sigma, D=D, fmt=FMT[fmt])
        twin = O.csr_spmv_fma_f32(csrs[j], enc.deq.astype(np.float32), xs[j].cpu().numpy())
        if expl:
            twin = twin[O.storage_rows(enc)]
        assert np.array_equal(ys[j].cpu().numpy().view(np.uint32), twin.view(np.uint32))


def _split_bound_check(y, csr, deq, X, words):
    X = np.asarray(X, np.float64).reshape(csr.m, -1)
    y = np.asarray(y, np.float64).reshape(csr.n, -1)
    ref = O.csr_spmm_f64(csr, deq, X)
    absref = O.csr_spmm_f64(csr, np.abs(deq), np.abs(X))
    w = np.maximum(np.asarray(words, np.float64), 1.0)[:, None]
    bound = (w * 2.0 ** -24 / (1 - w * 2.0 ** -24)) * absref
    bad = np.argwhere(~(np.abs(y - ref) <= bound))
    assert bad.size == 0, f"{len(bad)} entries beyond gamma_w, first {bad[:3].tolist()}"


def test_batch_mixes_slice_heights():
    """C = 32 and C = 1 (CSR order) matrices in one plan: the C = 32 ones give
    packsell_spmv's bits, the C = 1 ones (split rows) the bits of variant 14
    on the matrix alone, within gamma_w of the oracle; empty rows, sigma
    sorting and both orders among them."""
    need_gpu()
    ps = P()
    rng = np.random.default_rng(3)
    mats, csrs, xs, ys, encs = [], [], [], [], []
    for i in range(30):
        C = 1 if i % 2 else 32
        csr = (I.zipf_irregular(int(rng.integers(500, 6000)), seed=200 + i) if i % 3 == 0 else
               I.random_csr(int(rng.integers(1, 2500)), int(rng.integers(1, 2500)),
                            float(rng.uniform(0.001, 0.02)), seed=i, empty_rows=0.1, long_gaps=True))
        fmt, D = ("fp16", 15) if i % 4 < 2 else ("e8my", int(rng.integers(1, 16)))
        sigma = [1, 64, 1, 256][i % 4]
        expl = i % 5 == 0
        mats.append(ps.packsell_encode_csr(csr, fmt=fmt, D=D, C=C, sigma=sigma, explicit_perm=expl))
        encs.append(O.encode(csr, C=C, sigma=sigma, D=D, fmt=FMT[fmt]))
        csrs.append(csr)
        xs.append(dev(I.uniform(csr.m, seed=300 + i)))
        ys.append(torch.full((csr.n,), float("nan"), device="cuda"))
    B = ps.packsell_batch_create(mats, xs, ys)
    B.spmv()
    torch.cuda.synchronize()
    for A, csr, x, y, enc in zip(mats, csrs, xs, ys, encs):
        yv = y.cpu().numpy()
        if A.C == 32:
            ref = ps.packsell_spmv(A, x)
            assert torch.equal(y.view(torch.int32), ref.view(torch.int32))
            continue
        ps.packsell_set_spmv_variant(A, ps.SPMV_SPLIT)
        assert torch.equal(y.view(torch.int32), ps.packsell_spmv(A, x).view(torch.int32))
        if A.explicit_perm:
            yo = np.empty_like(yv)
            yo[O.storage_rows(enc)] = yv
            yv = yo
        _split_bound_check(yv, csr, enc.deq, x.cpu().numpy(), enc.words)


@pytest.mark.parametrize("k", [1, 4, 16, 64])
def test_batched_spmm_csr_order(k):
    """Batched SpMM over C = 1 matrices in one launch: every Y_i within
    gamma_w of the oracle's product; k = 1 takes the one-column form."""
    need_gpu()
    ps = P()
    batch = I.zipf_batch(24, seed=9, nmin=200, nmax=20000)
    mats, Xs, Ys, encs = [], [], [], []
    for j, c in enumerate(batch):
        fmt, D = ("fp16", 15) if j % 2 else ("e8my", 9)
        mats.append(ps.packsell_encode_csr(c, fmt=fmt, D=D, C=1, sigma=1))
        encs.append(O.encode(c, C=1, sigma=1, D=D, fmt=FMT[fmt]))
        Xs.append(dev(np.random.default_rng(j).uniform(-1, 1, (c.m, k)).astype(np.float32)))
        Ys.append(torch.full((c.n, k), float("nan"), device="cuda"))
    B = ps.packsell_batch_create_spmm(mats, Xs, Ys)
    B.spmm()
    torch.cuda.synchronize()
    for A, c, X, Y, enc in zip(mats, batch, Xs, Ys, encs):
        _split_bound_check(Y.cpu().numpy(), c, enc.deq, X.cpu().numpy(), enc.words)
        if k == 1:  # the SpMV's items and kernel: variant 14's bits
            ref = ps.packsell_spmv(A, X[:, 0].contiguous())
            assert torch.equal(Y[:, 0].contiguous().view(torch.int32), ref.view(torch.int32))
    with pytest.raises(ps.PackSELLError):  # an SpMM plan does not run as a batched SpMV
        ps._check(ps.lib().packsell_batch_spmv(B._h, None))


def test_batch_rejects_bad_matrices():
    need_gpu()
    ps = P()
    csr = I.random_csr(100, 100, 0.05, seed=1)
    A = ps.packsell_encode_csr(csr, fmt="sell_f32")
    x, y = dev(I.uniform(100, seed=1)), torch.empty(100, device="cuda")
    with pytest.raises(ps.PackSELLError):
        ps.packsell_batch_create([A], [x], [y])
    A8 = ps.packsell_encode_csr(csr, fmt="fp16", C=8)
    with pytest.raises(ps.PackSELLError):
        ps.packsell_batch_create([A8], [x], [y])
    A32 = ps.packsell_encode_csr(csr, fmt="fp16", C=32)
    X, Y = torch.zeros(100, 4, device="cuda"), torch.empty(100, 4, device="cuda")
    with pytest.raises(ps.PackSELLError):  # batched SpMM takes C = 1 matrices only
        ps.packsell_batch_create_spmm([A32], [X], [Y])
