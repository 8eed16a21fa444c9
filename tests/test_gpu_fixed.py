"""Fixed-point values (an integer value format, §4.2.1) on the GPU: the
encoder's exponent and words byte for byte the oracle's, the SpMV bit for
bit the oracle's FP32 twin of the decoded matrix, and an integer-valued
matrix exact."""
import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I

from _gpu import P, assert_same_encoding, dev, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case,D,C,sigma", [("random", 15, 32, 256), ("random", 7, 8, 64),
                                            ("stencil27", 11, 32, 256), ("stencil27", 22, 32, 1),
                                            ("zipf", 9, 1, 1)])
def test_fixed_encoding_and_spmv_match_oracle(case, D, C, sigma):
    need_gpu()
    ps = P()
    csr = {"random": lambda: I.random_csr(2000, 1800, 0.01, seed=D, empty_rows=0.05, long_gaps=True),
           "stencil27": lambda: I.stencil27(24, seed=D),
           "zipf": lambda: I.zipf_irregular(8000, seed=D)}[case]()
    enc = O.encode(csr, C=C, sigma=sigma, D=D, fmt=O.FMT_FIXED)
    A = ps.packsell_encode_csr(csr, fmt="fixed", D=D, C=C, sigma=sigma)
    assert A.value_exp == enc.value_exp
    assert_same_encoding(A, enc)
    x = I.uniform(csr.m, seed=3)
    y = ps.packsell_spmv(A, dev(x)).cpu().numpy()
    twin = O.csr_spmv_fma_f32(csr, enc.deq.astype(np.float32), x)
    assert np.array_equal(enc.deq.astype(np.float32).astype(np.float64), enc.deq)  # exact in FP32
    assert np.array_equal(y.view(np.uint32), twin.view(np.uint32))
    if C == 32:  # the row-prefetch kernel with programmatic launch: the same chain
        ps.packsell_set_spmv_variant(A, 13)
        y13 = ps.packsell_spmv(A, dev(x)).cpu().numpy()
        assert np.array_equal(y13.view(np.uint32), twin.view(np.uint32))
        ps.packsell_set_spmv_variant(A, 0)
        assert set(ps.packsell_tune_spmv(A, dev(x), reps=2)) == {1, 13}


def test_fixed_integer_matrix_is_exact():
    need_gpu()
    ps = P()
    a = I.poisson5(64)
    A = ps.packsell_encode_csr(a, fmt="fixed", D=15)
    xi = np.random.default_rng(4).integers(-50, 50, a.m).astype(np.float32)
    y = ps.packsell_spmv(A, dev(xi)).cpu().numpy()
    assert np.array_equal(y, O.csr_spmv_f64(a, a.val, xi.astype(np.float64)).astype(np.float32))


def test_fixed_refusals():
    need_gpu()
    ps = P()
    csr = I.random_csr(100, 100, 0.05, seed=1)
    with pytest.raises(ps.PackSELLError):
        ps.packsell_encode_csr(csr, fmt="fixed", D=5)  # q would not convert to FP32 exactly
    A = ps.packsell_encode_csr(csr, fmt="fixed", D=15)
    import torch
    with pytest.raises(ps.PackSELLError):
        ps.packsell_spmm(A, torch.zeros(100, 4, device="cuda"))
