"""16-bit PackSELL words (PACKSELL_FMT_W16_E4M3: W = 16, D = 7, FP8 E4M3
values) through the C ABI: the GPU encoder byte for byte against the
oracle's encode16 (multi-dummy chains, sigma sort, slices), the hardware
E4M3 rounding against the oracle's, error statuses, the SpMV bit for bit
against the FP32 twin on the E4M3 values, and the calls that refuse it."""
import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I

from _gpu import P, dev, need_gpu, torch

pytestmark = pytest.mark.gpu


def _encode(csr, **kw):
    return P().packsell_encode_csr(csr, fmt="w16_e4m3", D=7, **kw)


def _same(A, e):
    arr = P().packsell_arrays(A)
    assert A.k_left == e.k_left
    assert (A.n_words, A.n_dummies, A.n_pad) == (e.n_words, e.n_dummies, e.n_pad)
    assert np.array_equal(arr["offset"], e.offset)
    if A.sigma > 1:
        assert np.array_equal(arr["perm"], e.perm)
    bad = np.nonzero(arr["pack"] != e.pack)[0]
    assert bad.size == 0, f"{bad.size} words differ, first at {bad[:5]}"


@pytest.mark.parametrize("n,m,dens,C,sigma,gaps", [
    (300, 200000, 0.002, 32, 256, True),   # gaps past 2^15: dummy chains
    (1000, 1000, 0.01, 32, 4096, True),
    (500, 70000, 0.001, 1, 1, True),
    (257, 300, 0.05, 8, 16, False),
])
def test_w16_encode_matches_oracle(n, m, dens, C, sigma, gaps):
    need_gpu()
    csr = I.random_csr(n, m, dens, seed=n + m, empty_rows=0.05, long_gaps=gaps)
    csr.val[:] = np.clip(csr.val, -400, 400)
    _same(_encode(csr, C=C, sigma=sigma), O.encode16(csr, C=C, sigma=sigma))


def test_w16_encode_stencils():
    need_gpu()
    for csr in (I.stencil27(24, seed=2), I.poisson7_varcoef(14, seed=3)):  # float32, float64
        _same(_encode(csr), O.encode16(csr))


def test_e4m3_rounding_matches_oracle():
    """Ties both ways, subnormals, the 448/464 edge, random values across the
    range, in float32 and float64 inputs, as the diagonal of a matrix."""
    need_gpu()
    special = [1 + 1 / 16, 1 + 3 / 16, 464.0, 463.9, 448.5, 2.0 ** -10, 3 * 2.0 ** -11,
               15 * 2.0 ** -10, 2.0 ** -6, -1.1, 26.0, 0.0, -0.0, 1e-30, -7 * 2.0 ** -9]
    rng = np.random.default_rng(8)
    vals = np.concatenate([special, rng.uniform(-460, 460, 500),
                           rng.choice([-1, 1], 500) * 2.0 ** rng.uniform(-12, 8.8, 500)])
    n = vals.size
    for dt in (np.float32, np.float64):
        v = vals.astype(dt)
        csr = I.CSR(n=n, m=n, rowptr=np.arange(n + 1, dtype=np.int64),
                    col=np.arange(n, dtype=np.int32), val=v)
        _same(_encode(csr, sigma=1), O.encode16(csr, sigma=1))


def test_w16_errors():
    need_gpu()
    ps = P()
    one = lambda v: I.CSR(n=1, m=1, rowptr=np.array([0, 1]), col=np.array([0], np.int32),
                          val=np.array([v], np.float32))
    with pytest.raises(ps.PackSELLError, match="RANGE"):
        _encode(one(465.0))
    with pytest.raises(ps.PackSELLError, match="NONFINITE"):
        _encode(one(float("nan")))
    with pytest.raises(ps.PackSELLError, match="INVALID_ARG"):
        ps.packsell_encode_csr(one(1.0), fmt="w16_e4m3", D=15)


@pytest.mark.parametrize("explicit", [False, True])
def test_w16_spmv_matches_twin(explicit):
    need_gpu()
    ps = P()
    for csr in (I.stencil27(24, seed=4), I.random_csr(2000, 90000, 0.002, seed=5, empty_rows=0.1,
                                                      long_gaps=True)):
        e = O.encode16(csr)
        A = _encode(csr, explicit_perm=explicit)
        x = I.uniform(csr.m, seed=6)
        y = ps.packsell_spmv(A, dev(x)).cpu().numpy()
        twin = O.csr_spmv_fma_f32(csr, e.deq.astype(np.float32), x)
        if explicit:
            twin = twin[O.storage_rows(e)]
        assert np.array_equal(y.view(np.uint32), twin.view(np.uint32))
        times = ps.packsell_tune_spmv(A, dev(x), reps=2)
        assert set(times) == {1}


def test_w16_refused_calls():
    need_gpu()
    ps = P()
    csr = I.stencil27(8, seed=1)
    A = _encode(csr)
    x = dev(I.uniform(csr.m, seed=1))
    with pytest.raises(ps.PackSELLError):
        ps.packsell_spmm(A, torch.zeros(csr.m, 4, device="cuda"))
    with pytest.raises(ps.PackSELLError):
        ps.packsell_spmv_transpose(A, x)
    with pytest.raises(ps.PackSELLError):
        ps.PackSELLBatch([A], [x], [torch.empty(csr.n, device="cuda")])
