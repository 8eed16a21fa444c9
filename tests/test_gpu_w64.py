"""64-bit PackSELL words (W = 64, §4.2.1; E11MY values, FP64 products) on
the GPU: the encoder's words byte for byte the oracle's (quantiser included,
over every binade, subnormals, ties and the top of the range), the FP64
product bit for bit the oracle's stored-order chain, the Jacobi diagonal, and
the solvers with the 64-bit matrix as their FP64 operator."""

import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I

from _gpu import P, assert_same_encoding, dev, need_gpu, torch

pytestmark = pytest.mark.gpu


def f64(csr):
    return I.CSR(n=csr.n, m=csr.m, rowptr=csr.rowptr, col=csr.col, val=csr.val.astype(np.float64))


@pytest.mark.parametrize("case,D,C,sigma,dtype", [
    ("random", 11, 32, 256, np.float64), ("random", 2, 8, 64, np.float32),
    ("random", 31, 32, 1, np.float64), ("stencil27", 20, 32, 256, np.float64),
    ("zipf", 11, 1, 1, np.float64), ("random", 1, 32, 65536, np.float64),
])
def test_w64_encoding_and_spmv_match_oracle(case, D, C, sigma, dtype):
    need_gpu()
    ps = P()
    csr = {"random": lambda: I.random_csr(2000, 20000, 0.003, seed=D, dtype=np.float64,
                                          empty_rows=0.05, long_gaps=True),
           "stencil27": lambda: I.stencil27(20, seed=D),
           "zipf": lambda: I.zipf_irregular(8000, seed=D)}[case]()
    csr = I.CSR(n=csr.n, m=csr.m, rowptr=csr.rowptr, col=csr.col, val=csr.val.astype(dtype))
    enc = O.encode64(csr, C=C, sigma=sigma, D=D)
    A = ps.packsell_encode_csr(csr, fmt="w64_e11my", D=D, C=C, sigma=sigma)
    assert A.format == ps.FMT_W64_E11MY
    assert_same_encoding(A, enc)
    x = I.uniform(csr.m, seed=3).astype(np.float64)
    y = ps.packsell_spmv_f64(A, dev(x)).cpu().numpy()
    want = O.packsell64_spmv_f64(enc, x)
    assert np.array_equal(y.view(np.uint64), want.view(np.uint64))
    assert np.array_equal(want.view(np.uint64), O.csr_spmv_fma_f64(csr, enc.deq, x).view(np.uint64))


def test_w64_explicit_perm_writes_storage_order():
    need_gpu()
    ps = P()
    csr = f64(I.random_csr(3000, 2000, 0.01, seed=6, empty_rows=0.1))
    enc = O.encode64(csr, C=32, sigma=256, D=11)
    A = ps.packsell_encode_csr(csr, fmt="w64_e11my", D=11, explicit_perm=True)
    x = I.uniform(csr.m, seed=2).astype(np.float64)
    y = ps.packsell_spmv_f64(A, dev(x)).cpu().numpy()
    assert np.array_equal(y, O.packsell64_spmv_f64(enc, x, explicit=True))


@pytest.mark.parametrize("D", [1, 11, 31])
def test_w64_quantiser_over_every_binade(D):
    """Values chosen over every exponent field (subnormals included), ties,
    and the top of the range; encoded as one column so each word is the
    value field plus the flag."""
    need_gpu()
    ps = P()
    rng = np.random.default_rng(D)
    n = 1 << 18
    e = rng.integers(0, 2047, n).astype(np.uint64)
    pats = (rng.integers(0, 2, n).astype(np.uint64) << np.uint64(63)) | (e << np.uint64(52)) | \
        rng.integers(0, 1 << 52, n, dtype=np.uint64)
    ties = np.uint64(0x3FF0000000000000) | (rng.integers(0, 1 << (51 - D), 4096, dtype=np.uint64)
                                           << np.uint64(D + 1)) | np.uint64(1 << D)
    pats = np.concatenate([pats, ties, np.array([1, 2, 0x000FFFFFFFFFFFFF, 0x0010000000000000,
                                                 0x8000000000000000], np.uint64)])
    v = pats.view(np.float64)
    top = (2.0 - 2.0 ** -(51 - D)) * 2.0 ** 1023  # the largest E11MY value
    v = v[np.abs(v) <= top]
    rows = I.CSR(n=v.size, m=1, rowptr=np.arange(v.size + 1, dtype=np.int64),
                 col=np.zeros(v.size, np.int32), val=v)
    A = ps.packsell_encode_csr(rows, fmt="w64_e11my", D=D, C=32, sigma=1)
    words = ps.packsell_arrays(A)["pack"]
    field, _ = O.quantize_e11my(v, D)
    assert np.array_equal(words[:v.size], field | np.uint64(1))
    assert not words[v.size:].any()  # the last slice's phantom rows: padding
    with pytest.raises(ps.PackSELLError) as err:  # rounds past the largest finite double
        ps.packsell_encode_csr(I.CSR(n=1, m=1, rowptr=np.array([0, 1]),
                                     col=np.zeros(1, np.int32),
                                     val=np.array([np.finfo(np.float64).max])),
                               fmt="w64_e11my", D=D)
    assert err.value.code == 4


def test_w64_inv_diag_and_refusals():
    need_gpu()
    ps = P()
    a = I.poisson7_varcoef(12, seed=2)
    a = I.CSR(n=a.n, m=a.m, rowptr=a.rowptr, col=a.col,
              val=a.val.astype(np.float32).astype(np.float64))  # exact at Y = 40
    W = ps.packsell_encode_csr(a, fmt="w64_e11my", D=11)
    S64 = ps.packsell_encode_csr(a, fmt="sell_f64")
    assert torch.equal(ps.packsell_inv_diag(W), ps.packsell_inv_diag(S64))
    x32 = dev(I.uniform(a.m, seed=1))
    for call in (lambda: ps.packsell_spmv(W, x32), lambda: ps.packsell_tune_spmv(W, x32),
                 lambda: ps.packsell_spmm(W, torch.zeros(a.m, 4, device="cuda")),
                 lambda: ps.packsell_spmv_transpose(W, x32)):
        with pytest.raises(ps.PackSELLError):
            call()
    with pytest.raises(ps.PackSELLError):
        ps.packsell_encode_csr(a, fmt="w64_e11my", D=32)


def test_iocg_with_a_64_bit_outer_operator():
    """IO-CG (§5.2.2) with the 64-bit words as the FP64 outer operator: 1e-10
    on the true residual of the original matrix, in the outer iterations of
    the SELL_F64 outer operator (the operators differ by E11M40 rounding)."""
    need_gpu()
    ps = P()
    a = I.poisson7_varcoef(24, seed=3)
    b = I.uniform(a.n, seed=4).astype(np.float64)
    Ain = ps.packsell_encode_csr(a, fmt="fp16", D=15)
    runs = {}
    for fmt in ("sell_f64", "w64_e11my"):
        A64 = ps.packsell_encode_csr(f64(a), fmt=fmt, D=11)
        x, info = ps.packsell_pcg(A64, dev(b), A_inner=Ain, m_in=20, rtol=1e-10, max_iters=300)
        r = b - O.csr_spmv_f64(a, a.val, x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(b) < 2e-10
        runs[fmt] = info["iters"]
    assert abs(runs["sell_f64"] - runs["w64_e11my"]) <= 1, runs


def test_f3r_with_64_bit_operators():
    """F3R (§5.2.1) with 64-bit words as the FP64 outer operator (FP16-F3R)
    and as every layer's operator (FP64-F3R): 1e-9 on the true residual."""
    need_gpu()
    ps = P()
    csr = I.diag_scaled(I.stencil27(20, seed=3))
    bh = I.uniform(csr.n, seed=5, lo=0.0, hi=1.0).astype(np.float64)
    rp, cl, vl = dev(csr.rowptr), dev(csr.col), dev(csr.val.astype(np.float64))
    W = ps.packsell_encode(rp, cl, vl, csr.n, csr.m, fmt="w64_e11my", D=11)
    A2 = ps.packsell_encode(rp, cl, vl, csr.n, csr.m, fmt="sell_f32")
    A3 = ps.packsell_encode(rp, cl, vl, csr.n, csr.m, fmt="fp16", D=15)
    opts = dict(m1=20, m2=6, m3=3, m4=2, rtol=1e-9, max_iters=200)
    for mats in ((W, A2, A3), (W, W, W)):
        x, info = ps.packsell_f3r(*mats, dev(bh), **opts)
        r = bh - O.csr_spmv_f64(csr, csr.val, x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(bh) < 2e-9
