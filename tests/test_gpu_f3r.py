"""F3R (§5.2.1) on the GPU and the FP16 SELL format it is compared on.

- FP16 SELL SpMV: bit for bit the FP16 PackSELL thread-per-row SpMV and the
  oracle's FP32 twin (the same chain over the same FP16 values).
- PackSELL-F3R and FP16-SELL-F3R give the same iterates, bit for bit, and the
  same step counts (the paper's observation that they converge identically).
- FP16-F3R and FP64-F3R reach the tolerance on the true residual, in step
  counts close to the oracle's F3R with the same layers and precisions."""
import numpy as np
import pytest

import oracle as O
import oracle.solvers as S
from paper_2604_13433_gb300 import inputs as I

from _gpu import P, dev, need_gpu, torch

pytestmark = pytest.mark.gpu


scaled = I.diag_scaled  # the symmetric diagonal scaling of §5.2


def nonsym(n, seed):
    """A nonsymmetric diagonally dominant matrix with power-law-free random rows."""
    a = I.random_csr(n, n, 8.0 / n, seed=seed)
    row = np.repeat(np.arange(n), a.row_lengths())
    rs = np.bincount(row, np.abs(a.val.astype(np.float64)), n)
    keep = a.col != row
    rows = np.concatenate([row[keep], np.arange(n)])
    cols = np.concatenate([a.col[keep], np.arange(n)])
    vals = np.concatenate([a.val[keep].astype(np.float64), rs + 1.0])
    o = np.lexsort((cols, rows))
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int64)
    return scaled(I.CSR(n=n, m=n, rowptr=rowptr, col=cols[o].astype(np.int32), val=vals[o]))


@pytest.mark.parametrize("C,sigma", [(32, 256), (32, 1), (8, 64)])
def test_sell_f16_spmv_equals_packsell_fp16(C, sigma):
    need_gpu()
    ps = P()
    csr = I.random_csr(3000, 2500, 0.004, seed=C + sigma, empty_rows=0.05, long_gaps=True)
    x = dev(I.uniform(2500, seed=1))
    A16 = ps.packsell_encode_csr(csr, fmt="fp16", D=15, C=C, sigma=sigma)
    S16 = ps.packsell_encode_csr(csr, fmt="sell_f16", C=C, sigma=sigma)
    ps.packsell_set_spmv_variant(A16, ps.SPMV_ROWTHREAD)
    ya = ps.packsell_spmv(A16, x).cpu().numpy()
    ys = ps.packsell_spmv(S16, x).cpu().numpy()
    assert np.array_equal(ya.view(np.uint32), ys.view(np.uint32))
    deq = O.quantize(csr.val, O.FMT_FP16, 15)[1].astype(np.float32)
    twin = O.csr_spmv_fma_f32(csr, deq, x.cpu().numpy())
    assert np.array_equal(ys.view(np.uint32), twin.view(np.uint32))
    # the layout of FP32 SELL: same slots, 6 bytes each instead of 8
    assert S16.n_words == ps.packsell_encode_csr(csr, fmt="sell_f32", C=C, sigma=sigma).n_words


def _f3r_inputs(ps, csr, low_fmt):
    rp, cl = dev(csr.rowptr), dev(csr.col)
    vl = dev(csr.val.astype(np.float64))
    A1 = ps.packsell_encode(rp, cl, vl, csr.n, csr.m, fmt="sell_f64")
    if low_fmt == "fp64":
        return A1, A1, A1
    A2 = ps.packsell_encode(rp, cl, vl, csr.n, csr.m, fmt="sell_f32")
    A3 = ps.packsell_encode(rp, cl, vl, csr.n, csr.m, fmt=low_fmt, D=15)
    return A1, A2, A3


OPTS = dict(m1=20, m2=6, m3=3, m4=2, rtol=1e-9, max_iters=200)


@pytest.mark.parametrize("case", ["stencil27", "nonsym"])
def test_packsell_f3r_and_fp16_sell_f3r_iterate_identically(case):
    need_gpu()
    ps = P()
    csr = scaled(I.stencil27(24, seed=3)) if case == "stencil27" else nonsym(6000, 4)
    b = dev(I.uniform(csr.n, seed=5, lo=0.0, hi=1.0).astype(np.float64))
    xs, infos = [], []
    for fmt in ("fp16", "sell_f16"):
        A1, A2, A3 = _f3r_inputs(ps, csr, fmt)
        x, info = ps.packsell_f3r(A1, A2, A3, b, **OPTS)
        xs.append(x.cpu().numpy())
        infos.append(info)
    assert infos[0]["iters"] == infos[1]["iters"]
    assert np.array_equal(xs[0].view(np.uint64), xs[1].view(np.uint64))
    assert infos[0]["relres_true"] == infos[1]["relres_true"] < 1e-9
    r = b.cpu().numpy() - O.csr_spmv_f64(csr, csr.val, xs[0])
    assert np.linalg.norm(r) / np.linalg.norm(b.cpu().numpy()) < 1e-9


@pytest.mark.parametrize("case,mixed", [("stencil27", True), ("stencil27", False),
                                        ("nonsym", True), ("nonsym", False)])
def test_f3r_matches_oracle(case, mixed):
    need_gpu()
    ps = P()
    csr = scaled(I.stencil27(16, seed=6)) if case == "stencil27" else nonsym(3000, 7)
    bh = I.uniform(csr.n, seed=8, lo=0.0, hi=1.0).astype(np.float64)
    val16 = O.quantize(csr.val, O.FMT_FP16, 15)[1]
    xo, ko, _ = S.f3r(csr, bh, val16=val16, mixed=mixed, m1=OPTS["m1"], m2=OPTS["m2"],
                      m3=OPTS["m3"], m4=OPTS["m4"], tol=OPTS["rtol"], max_iters=OPTS["max_iters"])
    A1, A2, A3 = _f3r_inputs(ps, csr, "fp16" if mixed else "fp64")
    x, info = ps.packsell_f3r(A1, A2, A3, dev(bh), **OPTS)
    assert info["relres_true"] < 1e-9
    assert abs(info["iters"] - ko) <= max(1, ko // 5), (info["iters"], ko)
    assert np.allclose(x.cpu().numpy(), xo, rtol=1e-6, atol=1e-7 * np.abs(xo).max())
