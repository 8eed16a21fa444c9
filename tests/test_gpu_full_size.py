"""Parity at the full sizes of the benchmarked workloads, in the launch
configurations the bench times: the irregular 4M matrix (SpMV in both
layouts, sampled SpMM columns, the batch of 256), IO-CG on the 7-point
256^3 problem (true residual recomputed by the oracle) and the 512-system
differentiable solve (sampled systems against the oracle's adjoint).
Expected values come from the oracle only."""
import numpy as np
import pytest

import oracle as O
import oracle.solvers as S
from paper_2604_13433_gb300 import inputs as I

from _gpu import P, dev, need_gpu, torch

pytestmark = pytest.mark.gpu


def _twin(csr, fmt, D, x):
    field, deq = O.quantize(csr.val, fmt, D)
    return O.csr_spmv_fma_f32(csr, deq.astype(np.float32), x), deq


@pytest.fixture(scope="module")
def irr4m():
    """The bench's irregular 4M matrix, its FP16 values as the oracle
    quantises them, and the oracle's storage order (C = 32, sigma = 256)."""
    need_gpu()
    csr = I.zipf_irregular(4194304, seed=3)
    _, deq = O.quantize(csr.val, O.FMT_FP16, 15)
    rows = O.storage_rows(O.encode(csr, C=32, sigma=256, D=15, fmt=O.FMT_FP16))
    return csr, deq.astype(np.float32), rows


def test_irregular_4M_spmv_both_layouts(irr4m):
    """SELL slices (C = 32, sigma = 256, explicit order, tuned variant) and
    CSR order (C = 1, variant 11): every output row bitwise the twin; the
    split-row CSR kernel (variant 14, the bench's CSR-order default): every
    row within the gamma_w bound of the oracle's FP64 product."""
    ps = P()
    csr, deq32, rows = irr4m
    x = I.uniform(csr.m, seed=4)
    twin = O.csr_spmv_fma_f32(csr, deq32, x)
    xd = dev(x)
    A = ps.packsell_encode_csr(csr, fmt="fp16", D=15, explicit_perm=True)
    ps.packsell_tune_spmv(A, xd, reps=3)
    y = ps.packsell_spmv(A, xd).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), twin[rows].view(np.uint32))
    del A
    B = ps.packsell_encode_csr(csr, fmt="fp16", D=15, C=1, sigma=1)
    assert B.n_pad == 0
    for v in (ps.SPMV_ROWTHREAD, ps.SPMV_CSR):
        ps.packsell_set_spmv_variant(B, v)
        y = ps.packsell_spmv(B, xd).cpu().numpy()
        assert np.array_equal(y.view(np.uint32), twin.view(np.uint32)), f"variant {v}"
    ps.packsell_set_spmv_variant(B, ps.SPMV_SPLIT)
    y = ps.packsell_spmv(B, xd).cpu().numpy().astype(np.float64)
    enc_words = np.diff(ps.packsell_arrays(B)["offset"])  # C = 1: one row per slice
    ref = O.csr_spmv_f64(csr, deq32.astype(np.float64), x.astype(np.float64))
    bound = O.spmv_error_bound(csr, deq32.astype(np.float64), x, enc_words)
    bad = np.nonzero(~(np.abs(y - ref) <= bound))[0]
    assert bad.size == 0, f"variant 14: {bad.size} rows beyond the bound, first {bad[:5]}"
    ps.packsell_check_status(B)


@pytest.mark.parametrize("k,cols", [(4, (0, 3)), (16, (5,)), (64, (0, 31, 63))])
def test_irregular_4M_spmm_sampled_columns(irr4m, k, cols):
    """SpMM on the bench's matrix: sampled columns of Y are SpMVs with the
    matching column of X, bitwise the twin."""
    ps = P()
    csr, deq32, rows = irr4m
    Xh = np.random.default_rng(k).uniform(-1, 1, (csr.m, k)).astype(np.float32)
    A = ps.packsell_encode_csr(csr, fmt="fp16", D=15, explicit_perm=True)
    Y = ps.packsell_spmm(A, dev(Xh)).cpu().numpy()
    for q in cols:
        tw = O.csr_spmv_fma_f32(csr, deq32, np.ascontiguousarray(Xh[:, q]))
        assert np.array_equal(Y[:, q].view(np.uint32), tw[rows].view(np.uint32)), f"column {q}"


def test_batch_256_full_size():
    """The bench's batch of 256 irregular matrices in one launch: every
    matrix's y bitwise its twin."""
    need_gpu()
    ps = P()
    mats = I.zipf_batch(256, seed=5)
    As, xs, ys = [], [], []
    for i, c in enumerate(mats):
        As.append(ps.packsell_encode_csr(c, fmt="fp16", D=15))
        xs.append(dev(I.uniform(c.m, seed=100 + i)))
        ys.append(torch.empty(c.n, dtype=torch.float32, device="cuda"))
    B = ps.PackSELLBatch(As, xs, ys)
    B.spmv()
    torch.cuda.synchronize()
    for i, c in enumerate(mats):
        tw, _ = _twin(c, O.FMT_FP16, 15, xs[i].cpu().numpy())
        assert np.array_equal(ys[i].cpu().numpy().view(np.uint32), tw.view(np.uint32)), f"matrix {i}"


def test_iocg_7point_256_true_residual():
    """IO-CG (FP16 inner, m_in = 20, sigma = 1 as the bench's second setting)
    on n = 16.7M: the oracle's FP64 CSR product confirms ||b - A x|| / ||b||
    below 1e-10."""
    need_gpu()
    ps = P()
    csr = I.poisson7_varcoef(256, seed=0)
    b_h = I.uniform(csr.n, seed=1).astype(np.float64)
    rp, cl, vl = dev(csr.rowptr), dev(csr.col), dev(csr.val)
    A64 = ps.packsell_encode(rp, cl, vl, csr.n, csr.m, fmt="sell_f64", sigma=1)
    Ain = ps.packsell_encode(rp, cl, vl, csr.n, csr.m, fmt="fp16", D=15, sigma=1)
    x = torch.zeros(csr.n, dtype=torch.float64, device="cuda")
    _, info = ps.packsell_pcg(A64, dev(b_h), x, A_inner=Ain, m_in=20, rtol=1e-10,
                              max_iters=5000, check=False)
    assert info["status"] == "OK"
    xh = x.cpu().numpy()
    r = b_h - O.csr_spmv_f64(csr, csr.val.astype(np.float64), xh)
    assert np.linalg.norm(r) / np.linalg.norm(b_h) < 1e-10
    assert info["relres_true"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b_h), rel=1e-3)


@pytest.mark.parametrize("m_in,fmt,D", [(0, "fp16", 15), (20, "e8my", 11)])
def test_diff_solve_512_sampled_systems(m_in, fmt, D):
    """The bench's 512 block-diagonal systems, forward and backward. For the
    smallest, a middle and the largest system the oracle recomputes, in FP64,
    the block residuals of the solution and of the adjoint (each at most the
    whole system's 1e-10 stopping residual) and the chain from the adjoint
    and the solution to the face coefficients (to rounding); the solution is
    also close to the oracle's own FP64 PCG solve."""
    need_gpu()
    from paper_2604_13433_gb300 import autograd as ag

    csr, parts = I.poisson5_varcoef_batch(512, seed=6)
    n, nnz = csr.n, csr.nnz
    Pd = {k: dev(parts["pos_" + k]) for k in ("uu", "vv", "uv", "vu", "b")}
    Ff = parts["theta_f"].size
    th_h = np.concatenate([parts["theta_f"], parts["theta_b"]])
    theta = dev(th_h).requires_grad_(True)
    b_h = I.uniform(n, seed=7).astype(np.float64)
    xt_h = I.normal(n, seed=8)
    b = dev(b_h).requires_grad_(True)

    def assemble(th):
        v = torch.zeros(nnz, dtype=th.dtype, device=th.device)
        tf, tb = th[:Ff], th[Ff:]
        v = v.index_add(0, Pd["uu"], tf).index_add(0, Pd["vv"], tf)
        v = v.index_add(0, Pd["uv"], -tf).index_add(0, Pd["vu"], -tf)
        return v.index_add(0, Pd["b"], tb)

    rtol = 1e-10
    x = ag.solve(dev(csr.rowptr), dev(csr.col), assemble(theta), b, m_in=m_in, fmt=fmt, D=D,
                 rtol=rtol, max_iters=20000)
    ((x - dev(xt_h)) ** 2).sum().backward()
    xg, lam, gth = x.detach().cpu().numpy(), b.grad.cpu().numpy(), theta.grad.cpu().numpy()
    g = 2 * (xg - xt_h)
    nb_glob, ng_glob = np.linalg.norm(b_h), np.linalg.norm(g)
    sizes = [s["L"] for s in parts["systems"]]
    order = np.argsort(sizes, kind="stable")
    nf = [s["faces"]["u"].size for s in parts["systems"]]
    nbd = [s["faces"]["theta"].size - f for s, f in zip(parts["systems"], nf)]
    f0 = np.concatenate([[0], np.cumsum(nf)])
    b0 = Ff + np.concatenate([[0], np.cumsum(nbd)])
    for i in (order[0], order[len(order) // 2], order[-1]):
        sy = parts["systems"][i]
        c, faces = sy["csr"], sy["faces"]
        sl = slice(sy["row0"], sy["row0"] + c.n)
        a64 = c.val.astype(np.float64)
        r = b_h[sl] - O.csr_spmv_f64(c, a64, xg[sl])
        assert np.linalg.norm(r) <= 1.01 * rtol * nb_glob, f"system {i}: residual"
        ra = g[sl] - O.csr_spmv_f64(c, a64, lam[sl])
        assert np.linalg.norm(ra) <= 1.01 * rtol * ng_glob, f"system {i}: adjoint residual"
        row = np.repeat(np.arange(c.n), c.row_lengths())
        dth = S.face_grads(faces, -lam[sl][row] * xg[sl][c.col])
        gth_i = np.concatenate([gth[f0[i]:f0[i + 1]], gth[b0[i]:b0[i + 1]]])
        assert np.allclose(gth_i, dth, rtol=1e-10, atol=1e-12 * np.abs(dth).max()), \
            f"system {i}: dL/dtheta"
        xs, _, _ = S.pcg(c, b_h[sl], tol=1e-13, maxit=100000)
        assert np.linalg.norm(xg[sl] - xs) <= 1e-4 * np.linalg.norm(xs), f"system {i}: x"


def test_batch_256_csr_order_full_size():
    """The bench's batch of 256 in CSR order (C = 1) in one launch: every
    matrix's y is variant 14's on that matrix alone, bit for bit, and within
    the gamma_w bound of the oracle's FP64 product."""
    need_gpu()
    ps = P()
    mats = I.zipf_batch(256, seed=5)
    As, xs, ys = [], [], []
    for i, c in enumerate(mats):
        As.append(ps.packsell_encode_csr(c, fmt="fp16", D=15, C=1, sigma=1))
        xs.append(dev(I.uniform(c.m, seed=100 + i)))
        ys.append(torch.empty(c.n, dtype=torch.float32, device="cuda"))
    B = ps.PackSELLBatch(As, xs, ys)
    B.spmv()
    torch.cuda.synchronize()
    for i, c in enumerate(mats):
        single = ps.packsell_spmv(As[i], xs[i])
        assert torch.equal(ys[i].view(torch.int32), single.view(torch.int32)), f"matrix {i}"
        if i % 16 == 0:
            _, deq = O.quantize(c.val, O.FMT_FP16, 15)
            xh = xs[i].cpu().numpy().astype(np.float64)
            ref = O.csr_spmv_f64(c, deq, xh)
            bound = O.spmv_error_bound(c, deq, xh, np.diff(c.rowptr))
            y = ys[i].cpu().numpy().astype(np.float64)
            assert np.all(np.abs(y - ref) <= bound), f"matrix {i}"


@pytest.fixture(scope="module")
def st27():
    need_gpu()
    return I.stencil27(128, seed=0)


@pytest.mark.parametrize("fmt,D", [("fixed", 15), ("e8my", 11), ("sell_f16", 15)])
def test_headline_matrix_formats_full_size(st27, fmt, D):
    """The bench's format sweep on the 27-point 128^3 matrix (C = 32, sigma =
    256, explicit order, tuned variant): every row bitwise the FP32 twin of
    the format's values."""
    ps = P()
    csr = st27
    x = I.uniform(csr.m, seed=0)
    xd = dev(x)
    A = ps.packsell_encode_csr(csr, fmt=fmt, D=D, C=32, sigma=256, explicit_perm=True)
    if fmt != "sell_f16":
        ps.packsell_tune_spmv(A, xd, reps=3)
    y = ps.packsell_spmv(A, xd).cpu().numpy()
    if fmt == "fixed":
        enc = O.encode(csr, C=32, sigma=256, D=D, fmt=O.FMT_FIXED)
        deq = enc.deq
    else:
        qf = O.FMT_FP16 if fmt == "sell_f16" else O.FMT_E8MY
        enc = O.encode(csr, C=32, sigma=256, D=D, fmt=qf)
        deq = enc.deq
    twin = O.csr_spmv_fma_f32(csr, deq.astype(np.float32), x)
    rows = ps.packsell_storage_rows(A).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), twin[rows].view(np.uint32))


def test_headline_matrix_64_bit_words_full_size(st27):
    """The bench's FP64 pair on the 27-point 128^3 matrix: the 64-bit words
    (E11M40, D = 11) byte for byte the oracle's encoding and the FP64
    product bit for bit the oracle's stored-order chain."""
    ps = P()
    csr = st27
    enc = O.encode64(csr, C=32, sigma=256, D=11)
    A = ps.packsell_encode_csr(csr, fmt="w64_e11my", D=11, C=32, sigma=256, explicit_perm=True)
    arr = ps.packsell_arrays(A)
    assert np.array_equal(arr["offset"], enc.offset)
    assert np.array_equal(arr["pack"], enc.pack)
    x = I.uniform(csr.m, seed=0).astype(np.float64)
    y = ps.packsell_spmv_f64(A, dev(x)).cpu().numpy()
    want = O.packsell64_spmv_f64(enc, x, explicit=True)
    assert np.array_equal(y.view(np.uint64), want.view(np.uint64))
