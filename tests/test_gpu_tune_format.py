"""The format autotuner (packsell_tune_format): the slice height, sort block,
value format and delta bits it picks keep the SpMV's backward error (§5.1.2,
measured against the oracle's FP64 product of the unquantised matrix) under
the requested ceiling; its error bounds agree with the same bound computed by
the oracle's quantiser; and it picks CSR order for the power-law matrix and
SELL slices for the 27-point stencil."""
import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I

from _gpu import P, dev, need_gpu, torch

pytestmark = pytest.mark.gpu

FMTS = [("fp16", 15), ("e8my", 15), ("e8my", 11), ("e8my", 7), ("e8my", 3), ("e8my", 1)]


def _oracle_bound(csr, fmt, D):
    """(max_i sum|a - q(a)| + gamma_w max_i sum|q(a)|) / max_i sum|a|, w twice
    the longest row, from the oracle's quantiser; inf if a value overflows."""
    try:
        _, deq = O.quantize(csr.val, O.FMT_FP16 if fmt == "fp16" else O.FMT_E8MY, D)
    except O.OracleError:
        return float("inf")
    a = np.abs(csr.val.astype(np.float64))
    row = np.repeat(np.arange(csr.n), np.diff(csr.rowptr))
    E = np.bincount(row, np.abs(csr.val.astype(np.float64) - deq), csr.n).max()
    Q = np.bincount(row, np.abs(deq), csr.n).max()
    A = np.bincount(row, a, csr.n).max()
    w = 2.0 * max(int(np.diff(csr.rowptr).max()), 1)
    u = 2.0 ** -24
    return (E + w * u / (1 - w * u) * Q) / A


def _tune(ps, csr, ceiling):
    rp, cl, vl = dev(csr.rowptr), dev(csr.col), dev(csr.val)
    x = dev(I.uniform(csr.m, seed=11))
    params, trials = ps.packsell_tune_format(rp, cl, vl, csr.n, csr.m, ceiling, x, reps=5)
    return params, trials, (rp, cl, vl, x)


def _backward_error(ps, csr, params, tensors):
    rp, cl, vl, x = tensors
    A = ps.packsell_encode(rp, cl, vl, csr.n, csr.m, **params)
    y = ps.packsell_spmv(A, x).cpu().numpy().astype(np.float64)
    return O.backward_error(y, csr, csr.val.astype(np.float64), x.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("ceiling", [1e-3, 5.5e-4])
def test_tune_format_power_law_rows(ceiling):
    need_gpu()
    ps = P()
    csr = I.zipf_irregular(1 << 20, seed=17)
    params, trials, t = _tune(ps, csr, ceiling)
    assert params["C"] == 1 and params["sigma"] == 1, params  # CSR order: no SELL padding
    assert len(trials) == 18
    for fmt, D in FMTS:  # the kernel's bound equals the oracle's, for every format
        tr = [r for r in trials if r["fmt"] == fmt and r["D"] == D]
        ref = _oracle_bound(csr, fmt, D)
        assert all(abs(r["error"] - ref) <= 1e-9 * ref for r in tr), (fmt, D, tr[0]["error"], ref)
        assert all(r["admissible"] == (ref <= ceiling) for r in tr)
    timed = [r for r in trials if r["admissible"]]
    assert timed and all(r["ms"] > 0 for r in timed)
    best = min(timed, key=lambda r: r["ms"])
    assert (best["C"], best["sigma"], best["fmt"], best["D"]) == \
        (params["C"], params["sigma"], params["fmt"], params["D"])
    assert _backward_error(ps, csr, params, t) <= ceiling


def test_tune_format_stencil27():
    need_gpu()
    ps = P()
    csr = I.stencil27(128, seed=0)
    params, trials, t = _tune(ps, csr, 1e-3)
    assert params["C"] == 32, params  # rows of equal length: SELL slices
    assert _backward_error(ps, csr, params, t) <= 1e-3


def test_tune_format_refuses_an_unreachable_ceiling():
    need_gpu()
    ps = P()
    csr = I.random_csr(500, 500, 0.02, seed=3)
    with pytest.raises(ps.PackSELLError) as e:
        _tune(ps, csr, 1e-12)
    assert e.value.code == 4
