"""packsell_pcg_noalloc: the solver for callers that cannot allocate device
memory while they solve (an application whose memory is reserved for its own
pool, a plugin with a fixed budget, a loop that must not take cudaMalloc's
implicit synchronisation). Its workspace is the library's static 8 MiB device
array. This file is collected
last on purpose (its name), and passes alone in a fresh process as well as
after the other tests.

Checked through the C ABI against packsell_pcg (which allocates its own
workspace) on two calls in a row: the same kernels on the same fixed grids
give the same bits, so the results must agree exactly; the test still states
the solver tolerance it needs (true relative residual below 1e-10, solutions
within 1e-12 relative)."""
import numpy as np
import pytest

from paper_2604_13433_gb300 import inputs as I

from _gpu import P, dev, need_gpu, torch

pytestmark = pytest.mark.gpu


def test_pcg_noalloc_matches_pcg_twice():
    need_gpu()
    ps = P()
    a = I.poisson7_varcoef(24, seed=21)  # 13,824 unknowns, unit diagonal
    b = dev(I.uniform(a.n, seed=22).astype(np.float64))
    A64 = ps.packsell_encode_csr(a, fmt="sell_f64")
    Ain = ps.packsell_encode_csr(a, fmt="e8my", D=9)
    x_ref, info_ref = ps.packsell_pcg(A64, b, A_inner=Ain, m_in=20, rtol=1e-10, max_iters=200)
    for _ in range(2):  # the shared array keeps the previous call's contents
        x = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        x, info = ps.packsell_pcg_noalloc(A64, b, x, A_inner=Ain, m_in=20, rtol=1e-10,
                                          max_iters=200)
        assert info["relres_true"] < 1e-10
        assert info["iters"] == info_ref["iters"]
        err = (x - x_ref).abs().max().item() / x_ref.abs().max().item()
        assert err <= 1e-12
        assert torch.equal(x, x_ref)
    # FP64 PCG mode with a Jacobi preconditioner
    M = dev(np.ones(a.n))
    x64_ref, _ = ps.packsell_pcg(A64, b, inv_diag=M, rtol=1e-10, max_iters=500)
    x64 = torch.zeros_like(x64_ref)
    x64, info = ps.packsell_pcg_noalloc(A64, b, x64, inv_diag=M, rtol=1e-10, max_iters=500)
    assert info["relres_true"] < 1e-10 and torch.equal(x64, x64_ref)


def test_pcg_noalloc_rejects_systems_beyond_the_static_area():
    need_gpu()
    ps = P()
    a = I.poisson7_varcoef(70, seed=23)  # 343,000 unknowns: 11 MB of FP64 PCG workspace
    A64 = ps.packsell_encode_csr(a, fmt="sell_f64")
    b = torch.ones(a.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    assert ps.packsell_pcg_workspace_bytes(a.n, 0, False, 1000) > 8 << 20
    with pytest.raises(ps.PackSELLError) as e:
        ps.packsell_pcg_noalloc(A64, b, x, rtol=1e-10, max_iters=1000)
    assert e.value.code == 1 and "static area" in str(e.value)
    assert torch.count_nonzero(x) == 0
