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
