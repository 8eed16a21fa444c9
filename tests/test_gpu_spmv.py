"""GPU products vs the oracle (through the C ABI).

The thread-per-row SpMV sums each row in stored order with FP32 fused
multiply-adds, so it must equal the oracle's FP32 twin (csr_spmv_fma_f32 on
the quantised values) bit for bit; it is also held to the FP32 forward error
bound against the FP64 oracle on the same quantised values (§4.4, Eq. 1).
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I

from _gpu import FMT, P, dev, encode_gpu, need_gpu, torch

pytestmark = pytest.mark.gpu

# ||y - y_oracle||_inf / ||y_oracle||_inf for the stencil matrices (rows of at
# most 27 words: gamma_27 * sum|a x| / max|y| stays below it); every case is
# also held to the componentwise bound gamma_w * sum_j |q(a_ij) x_j|
REL_TOL = 1e-6


def check_spmv(csr, fmt, D, C=32, sigma=256, explicit=False, seed=0, rel_tol=None):
    packsell = P()
    enc = O.encode(csr, C=C, sigma=sigma, D=D, fmt=FMT[fmt])
    A = encode_gpu(csr, fmt=fmt, C=C, sigma=sigma, D=D, explicit_perm=explicit)
    x = I.uniform(csr.m, seed=seed)
    xd = dev(x)
    variants = [packsell.SPMV_ROWTHREAD]
    if C == 32 and fmt in ("fp16", "e8my"):
        variants += list(packsell.SPMV_PREFETCH) + list(packsell.SPMV_DUAL) + list(packsell.SPMV_STAGE)
        variants.append(packsell.SPMV_PDL)
    if C == 32 and csr.n > 0 and fmt in ("fp16", "e8my"):
        variants += list(packsell.SPMV_BULK_VARIANTS)
    if C == 1 and csr.n > 0 and fmt in ("fp16", "e8my"):
        variants.append(packsell.SPMV_CSR)
    if C == 32 and csr.n > 0 and fmt in ("fp16", "e8my") and A.max_width <= 16:
        variants.append(packsell.SPMV_PIPE)
    ys = []
    for v in variants:
        packsell.packsell_set_spmv_variant(A, v)
        ys.append(packsell.packsell_spmv(A, xd).cpu().numpy())
    packsell.packsell_check_status(A)
    twin = O.csr_spmv_fma_f32(csr, enc.deq.astype(np.float32), x)
    tw = twin[O.storage_rows(enc)] if explicit else twin
    bad = {v: int((yv.view(np.uint32) != tw.view(np.uint32)).sum()) for v, yv in zip(variants, ys)}
    assert not any(bad.values()), f"rows differing from the FP32 twin, per variant: {bad}"
    y = ys[-1]
    ref = O.csr_spmv_f64(csr, enc.deq, x.astype(np.float64))
    if explicit:
        rows = O.storage_rows(enc)
        twin, ref = twin[rows], ref[rows]
    assert np.array_equal(y.view(np.uint32), twin.view(np.uint32)), \
        f"{int((y != twin).sum())} rows differ from the FP32 twin"
    bound = O.spmv_error_bound(csr, enc.deq, x, enc.words)
    if explicit:
        bound = bound[O.storage_rows(enc)]
    assert np.all(np.abs(y - ref) <= bound)
    if rel_tol is not None and np.abs(ref).max() > 0:
        assert np.abs(y - ref).max() / np.abs(ref).max() <= rel_tol
    if C == 1 and csr.n > 0 and fmt in ("fp16", "e8my"):
        check_split(packsell, A, xd, ref, bound)
    return A, enc, x, y


def check_split(packsell, A, xd, ref, bound):
    """Variant 14 (split rows, CSR order) sums a row as a fixed tree, not the
    stored-order chain: every row within the gamma_w forward-error bound of
    the oracle's FP64 product on the same quantised values, and the same bits
    on a second run."""
    packsell.packsell_set_spmv_variant(A, packsell.SPMV_SPLIT)
    y1 = packsell.packsell_spmv(A, xd).cpu().numpy()
    y2 = packsell.packsell_spmv(A, xd).cpu().numpy()
    assert np.array_equal(y1.view(np.uint32), y2.view(np.uint32))
    err = np.abs(y1.astype(np.float64) - ref)
    bad = np.nonzero(~(err <= bound))[0]
    assert bad.size == 0, f"variant 14: {bad.size} rows beyond the bound, first {bad[:5]}"
    packsell.packsell_set_spmv_variant(A, packsell.SPMV_AUTO)


CASES = [
    (33, 47, 0.2, 32, 256, "fp16", 15),
    (1000, 1000, 0.01, 32, 256, "e8my", 11),
    (777, 1500, 0.02, 32, 64, "e8my", 2),
    (4099, 4099, 0.003, 32, 256, "e8my", 1),
    (300, 90, 0.1, 8, 16, "e8my", 5),
    (2000, 3000, 0.005, 64, 512, "fp16", 15),
    (130, 400, 0.02, 32, 1, "e8my", 7),
    (64, 5000, 0.01, 16, 32, "e8my", 22),
]


@pytest.mark.parametrize("case", CASES)
def test_spmv_random(case):
    need_gpu()
    n, m, dens, C, sigma, fmt, D = case
    csr = I.random_csr(n, m, dens, seed=n, empty_rows=0.1, long_gaps=True)
    check_spmv(csr, fmt, D, C, sigma)


@pytest.mark.parametrize("explicit", [False, True])
def test_spmv_poisson5_64(explicit):
    need_gpu()
    a = I.poisson5(64)
    A, enc, x, y = check_spmv(a, "fp16", 15, sigma=1, explicit=explicit, rel_tol=REL_TOL)
    if not explicit:  # closed form: 4 x_i minus the four neighbours
        g = np.pad(x.astype(np.float64).reshape(64, 64), 1)
        ref = 4 * g[1:-1, 1:-1] - g[:-2, 1:-1] - g[2:, 1:-1] - g[1:-1, :-2] - g[1:-1, 2:]
        assert np.allclose(y, ref.ravel(), rtol=0, atol=1e-5)


def test_spmv_wide_rows_cross_stages():
    """Rows wider than a shared-memory stage (1 to 3000 words) and empty
    slices between them: the bulk kernel carries a row across stages."""
    need_gpu()
    rng = np.random.default_rng(5)
    n, m = 2000, 8000
    lens = np.where(rng.random(n) < 0.02, rng.integers(500, 3000, n), rng.integers(0, 6, n))
    lens[200:300] = 0
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rowptr[1:])
    cols = np.concatenate([np.sort(rng.choice(m, l, replace=False)) for l in lens]).astype(np.int32)
    csr = I.CSR(n=n, m=m, rowptr=rowptr, col=cols,
                val=rng.standard_normal(cols.size).astype(np.float32))
    for fmt, D in (("fp16", 15), ("e8my", 4)):
        check_spmv(csr, fmt, D, sigma=64)


@pytest.mark.parametrize("fmt,D", [("fp16", 15), ("e8my", 15), ("e8my", 11), ("e8my", 7)])
def test_spmv_stencil27_48(fmt, D):
    need_gpu()
    check_spmv(I.stencil27(48, seed=3), fmt, D, rel_tol=REL_TOL)


@pytest.mark.parametrize("fmt,D,explicit", [("fp16", 15, True), ("e8my", 11, True),
                                            ("e8my", 7, False)])
def test_spmv_stencil27_128_full_size(fmt, D, explicit):
    """The 2.1M-row, 55.7M-nonzero HPCG_7_7_7 pattern at the benchmark's
    launch configuration (every warp walks many slices, E8MY adds dummies):
    all rows of every variant bitwise against the FP32 twin."""
    need_gpu()
    check_spmv(I.stencil27(128, seed=0), fmt, D, explicit=explicit, rel_tol=REL_TOL)


@pytest.mark.parametrize("fmt,D,sigma", [("fp16", 15, 256), ("e8my", 11, 256),
                                          ("e8my", 7, 100), ("fp16", 15, 1)])
def test_storage_rows_maps_explicit_to_original(fmt, D, sigma):
    """packsell_storage_rows equals the oracle's storage order, is a
    permutation, and scattering an explicit-perm product through it gives the
    implicit-perm product bit for bit. The 7-point matrix with E8MY dummies
    sorts differently from FP16 (dummy words count in the sort key)."""
    need_gpu()
    packsell = P()
    csr = I.poisson7_varcoef(20, seed=4)
    enc = O.encode(csr, C=32, sigma=sigma, D=D, fmt=FMT[fmt])
    Ae = encode_gpu(csr, fmt=fmt, sigma=sigma, D=D, explicit_perm=True)
    Ai = encode_gpu(csr, fmt=fmt, sigma=sigma, D=D, explicit_perm=False)
    rows = packsell.packsell_storage_rows(Ae)
    assert np.array_equal(rows.cpu().numpy(), O.storage_rows(enc))
    assert np.array_equal(np.sort(rows.cpu().numpy()), np.arange(csr.n))
    assert np.array_equal(packsell.packsell_storage_rows(Ai).cpu().numpy(), O.storage_rows(enc))
    x = dev(I.uniform(csr.m, seed=5))
    ye = packsell.packsell_spmv(Ae, x)
    yo = torch.empty_like(ye)
    yo[rows.long()] = ye
    yi = packsell.packsell_spmv(Ai, x)
    assert torch.equal(yo.view(torch.int32), yi.view(torch.int32))


def _lengths_csr(lengths, m, seed):
    """A CSR with the given row lengths (distinct random columns per row)."""
    rng = np.random.default_rng(seed)
    cols = [np.sort(rng.choice(m, size=L, replace=False)) for L in lengths]
    rowptr = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32) if sum(lengths) else np.zeros(0, np.int32)
    val = rng.uniform(-1, 1, int(rowptr[-1])).astype(np.float32)
    return I.CSR(n=len(lengths), m=m, rowptr=rowptr, col=col, val=val)


@pytest.mark.parametrize("fmt,D,sigma,explicit", [("fp16", 15, 1, False), ("e8my", 11, 1, True),
                                                  ("fp16", 15, 256, False), ("e8my", 3, 1, False),
                                                  ("e8my", 7, 100, True)])
def test_spmv_csr_order_zipf(fmt, D, sigma, explicit):
    """CSR-order packing (C = 1, variant 11) on power-law rows up to 4,096
    words: tiles of short rows and the long-row path, bitwise the twin."""
    need_gpu()
    csr = I.zipf_irregular(30000, seed=5)
    A, enc, x, y = check_spmv(csr, fmt, D, C=1, sigma=sigma, explicit=explicit)
    assert A.n_pad == 0


def test_spmv_csr_order_tile_edges():
    """Row lengths around the 256-word tile limit and the 64-row tile cap,
    empty rows, and rows with many dummies (D = 2)."""
    need_gpu()
    lengths = ([0, 1, 255, 256, 257, 0, 511, 512, 513, 3] + [4] * 70 + [0] * 40 +
               [256, 1, 1000, 2, 253, 254, 252, 1, 250, 3, 0, 0] + [1] * 700 + [0] * 300)
    csr = _lengths_csr(lengths, 5000, seed=1)
    for fmt, D in (("fp16", 15), ("e8my", 2)):
        check_spmv(csr, fmt, D, C=1, sigma=1)
    packsell = P()
    A = encode_gpu(csr, fmt="fp16", C=1, sigma=1)
    times = packsell.packsell_tune_spmv(A, dev(I.uniform(csr.m, seed=2)), reps=3)
    assert packsell.SPMV_CSR in times and packsell.SPMV_SPLIT in times
    assert 5 not in times  # C = 32 variants are skipped


def test_pipelined_variant_short_rows_only():
    """Variant 12 runs one round per row: offered for slices of at most 16
    words (7-point rows with their dummies), refused and skipped otherwise."""
    need_gpu()
    packsell = P()
    csr = I.poisson7_varcoef(24, seed=3)
    A, enc, x, y = check_spmv(csr, "fp16", 15, sigma=1)
    assert A.max_width <= 16
    times = packsell.packsell_tune_spmv(A, dev(x), reps=3)
    assert packsell.SPMV_PIPE in times
    B = encode_gpu(I.stencil27(16, seed=1), fmt="fp16")
    assert B.max_width > 16
    with pytest.raises(packsell.PackSELLError):
        packsell.packsell_set_spmv_variant(B, packsell.SPMV_PIPE)
    assert packsell.SPMV_PIPE not in packsell.packsell_tune_spmv(
        B, dev(I.uniform(B.m, seed=2)), reps=2)


def test_dependent_launch_chain():
    """Variant 13 loads its first words before it waits for the previous
    kernel of its stream. In a chain y_{k+1} = A y_k on one stream each
    product reads the vector the product before it has just written, and a
    torch kernel halves the vector between some of them; every step must
    equal the oracle's FP32 twin applied to the previous step, bit for bit."""
    need_gpu()
    packsell = P()
    csr = I.stencil27(24, seed=5)
    enc = O.encode(csr, C=32, sigma=256, D=15, fmt=FMT["fp16"])
    A = encode_gpu(csr, fmt="fp16", C=32, sigma=256, D=15)  # y in original row order
    packsell.packsell_set_spmv_variant(A, packsell.SPMV_PDL)
    deq = enc.deq.astype(np.float32)
    v = I.uniform(csr.m, seed=9)
    vd = dev(v)
    outs = []
    for k in range(8):
        if k % 3 == 2:
            vd = vd * 0.5  # exact in FP32
        vd = packsell.packsell_spmv(A, vd)
        outs.append(vd)
    packsell.packsell_check_status(A)
    for k, yd in enumerate(outs):
        if k % 3 == 2:
            v = v * np.float32(0.5)
        v = O.csr_spmv_fma_f32(csr, deq, v)
        y = yd.cpu().numpy()
        assert np.array_equal(y.view(np.uint32), v.view(np.uint32)), f"step {k}"


def test_spmv_column_range_limit():
    """m = 2^31 - 1 columns (the format's limit): deltas above 2^30 need the
    31-bit dummy, one row ends at column m - 1. x (8 GB) lives only on the
    device, filled from a formula; the oracle twin runs on the same matrix
    with its used columns renumbered 0.., which keeps every value, order and
    x value, so each row's fused multiply-add chain is the same."""
    need_gpu()
    packsell = P()
    m = 2 ** 31 - 1
    rng = np.random.default_rng(31)
    rows = []
    for i in range(64):
        L = int(rng.integers(0, 9))
        cols = np.sort(rng.choice(m - 1, size=L, replace=False)) if L else np.zeros(0, np.int64)
        if i % 7 == 0:
            cols = np.unique(np.append(cols, m - 1))
        if i % 5 == 0:
            cols = np.unique(np.append(cols, [0, 2 ** 30 + i]))
        rows.append(cols.astype(np.int64))
    rowptr = np.concatenate([[0], np.cumsum([r.size for r in rows])]).astype(np.int64)
    col = np.concatenate(rows).astype(np.int32)
    val = rng.uniform(-1, 1, col.size).astype(np.float32)
    csr = I.CSR(n=64, m=m, rowptr=rowptr, col=col, val=val)
    # x_c = ((c mod 1000) - 500) * 2^-9: exact in float32 on both sides (a
    # division by 500 is not: torch divides by a scalar through its reciprocal)
    xf = lambda c: ((c % 1000) - 500).astype(np.float32) * np.float32(2.0 ** -9)
    for fmt, D in (("fp16", 15), ("e8my", 11)):
        A = encode_gpu(csr, fmt=fmt, D=D)
        assert A.n_dummies > 0
        xd = torch.empty(m, dtype=torch.float32, device="cuda")
        step = 1 << 28
        for a in range(0, m, step):
            c = torch.arange(a, min(m, a + step), dtype=torch.int64, device="cuda")
            xd[a:a + c.numel()] = ((c % 1000) - 500).to(torch.float32) * (2.0 ** -9)
        used, inv = np.unique(col, return_inverse=True)
        xu = xd[torch.from_numpy(used).cuda()].cpu().numpy()
        assert np.array_equal(xu.view(np.uint32), xf(used.astype(np.int64)).view(np.uint32))
        y = packsell.packsell_spmv(A, xd).cpu().numpy()
        del xd
        small = I.CSR(n=64, m=used.size, rowptr=rowptr, col=inv.astype(np.int32), val=val)
        _, deq = O.quantize(val, FMT[fmt], D)
        twin = O.csr_spmv_fma_f32(small, deq.astype(np.float32), xf(used.astype(np.int64)))
        assert np.array_equal(y.view(np.uint32), twin.view(np.uint32))


@pytest.mark.parametrize("fmt,D,explicit", [("fp16", 15, False), ("fp16", 15, True),
                                             ("e8my", 11, False), ("e8my", 5, True)])
def test_spmv_x16_paper_configuration(fmt, D, explicit):
    """x and y in binary16 (the paper's FP16 SpMV, §5.1.1): y equals the FP32
    twin on the widened x, rounded to binary16 (nearest even), bit for bit."""
    need_gpu()
    packsell = P()
    for csr in (I.stencil27(20, seed=6), I.random_csr(900, 700, 0.01, seed=3, empty_rows=0.1,
                                                     long_gaps=True)):
        enc = O.encode(csr, D=D, fmt=FMT[fmt])
        A = encode_gpu(csr, fmt=fmt, D=D, explicit_perm=explicit)
        xh = np.random.default_rng(7).uniform(-2, 2, csr.m).astype(np.float16)
        y = packsell.packsell_spmv_x16(A, dev(xh)).cpu().numpy()
        twin = O.csr_spmv_fma_f32(csr, enc.deq.astype(np.float32), xh.astype(np.float32))
        want = twin.astype(np.float16)
        if explicit:
            want = want[O.storage_rows(enc)]
        assert np.array_equal(y.view(np.uint16), want.view(np.uint16))


def test_spmv_host_buffers():
    """packsell_spmv_host: host x in, host y out through caller-owned device
    buffers; equals packsell_spmv bit for bit; NULL buffers are refused."""
    need_gpu()
    packsell = P()
    csr = I.stencil27(16, seed=9)
    A = encode_gpu(csr, fmt="fp16")
    xh = torch.from_numpy(I.uniform(csr.m, seed=10)).pin_memory()
    yh = torch.empty(csr.n, dtype=torch.float32).pin_memory()
    xd = torch.empty(csr.m, device="cuda")
    yd = torch.empty(csr.n, device="cuda")
    packsell.packsell_spmv_host(A, xh, yh, xd, yd)
    torch.cuda.synchronize()
    ref = packsell.packsell_spmv(A, xh.cuda()).cpu()
    assert torch.equal(yh.view(torch.int32), ref.view(torch.int32))
    with pytest.raises(packsell.PackSELLError):
        packsell._check(packsell.lib().packsell_spmv_host(A.handle, None, yh.data_ptr(),
                                                          xd.data_ptr(), yd.data_ptr(), None))


@pytest.mark.parametrize("host", ["pinned", "pinned_offset", "pageable"])
def test_spmv_host_copy_paths(host):
    """Host buffers of every kind - pinned, pinned starting one float into its
    allocation, pageable - give packsell_spmv's bits, on sizes that are not
    multiples of 4, over repeated calls."""
    need_gpu()
    packsell = P()
    csr = I.random_csr(1001, 999, 0.01, seed=4, empty_rows=0.05)
    A = encode_gpu(csr, fmt="e8my", D=9)
    x = torch.from_numpy(I.uniform(csr.m, seed=5))
    if host == "pageable":
        xh, yh = x.clone(), torch.full((csr.n,), float("nan"))
    else:
        off = 1 if host == "pinned_offset" else 0
        xb = torch.empty(csr.m + off, dtype=torch.float32).pin_memory()
        yb = torch.full((csr.n + off,), float("nan"), dtype=torch.float32).pin_memory()
        xh, yh = xb[off:], yb[off:]
        xh.copy_(x)
    xd = torch.empty(csr.m, device="cuda")
    yd = torch.empty(csr.n, device="cuda")
    for _ in range(3):  # repeated calls reuse the buffers
        packsell.packsell_spmv_host(A, xh, yh, xd, yd)
    torch.cuda.synchronize()
    ref = packsell.packsell_spmv(A, x.cuda()).cpu()
    assert torch.equal(yh.view(torch.int32), ref.view(torch.int32))


def test_tune_spmv_picks_a_variant():
    need_gpu()
    packsell = P()
    csr = I.stencil27(24, seed=2)
    A = encode_gpu(csr, fmt="fp16")
    x = dev(I.uniform(csr.m, seed=1))
    times = packsell.packsell_tune_spmv(A, x, reps=5)
    # 11 needs C = 1 and 12 slices of at most 16 words
    assert set(times) == set(range(1, 11)) | {13} and all(t > 0 for t in times.values())
    y = packsell.packsell_spmv(A, x).cpu().numpy()  # variant 0 = tuned choice
    enc = O.encode(csr, fmt=O.FMT_FP16)
    twin = O.csr_spmv_fma_f32(csr, enc.deq.astype(np.float32), x.cpu().numpy())
    assert np.array_equal(y.view(np.uint32), twin.view(np.uint32))


def test_spmv_padding_dummies_do_not_touch_x():
    """Padding and dummy words read no x: NaN in x at columns no row uses
    (and at the dummy targets' neighbours) leaves y finite (§4.3 reading)."""
    need_gpu()
    packsell = P()
    csr = I.random_csr(200, 400, 0.02, seed=11, long_gaps=True)
    used = np.zeros(400, bool)
    used[csr.col] = True
    x = I.uniform(400, seed=2)
    x[~used] = np.nan
    A = encode_gpu(csr, fmt="e8my", D=3, C=32, sigma=32)
    assert A.n_dummies > 0 and A.n_pad > 0
    y = packsell.packsell_spmv(A, dev(x)).cpu().numpy()
    assert np.all(np.isfinite(y))


def test_sell_f32_and_f64():
    need_gpu()
    packsell = P()
    csr = I.random_csr(3000, 2500, 0.004, seed=4, empty_rows=0.05)
    x = I.uniform(2500, seed=5)
    A = encode_gpu(csr, fmt="sell_f32")
    y = packsell.packsell_spmv(A, dev(x)).cpu().numpy()
    twin = O.csr_spmv_fma_f32(csr, csr.val, x)
    assert np.array_equal(y.view(np.uint32), twin.view(np.uint32))
    B = encode_gpu(csr, fmt="sell_f64")
    y64 = packsell.packsell_spmv_f64(B, dev(x.astype(np.float64))).cpu().numpy()
    ref = O.csr_spmv_f64(csr, csr.val.astype(np.float64), x.astype(np.float64))
    assert np.allclose(y64, ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("fmt,D,k", [("fp16", 15, 1), ("e8my", 11, 4), ("e8my", 2, 16),
                                     ("fp16", 15, 64), ("sell_f32", 0, 5), ("fp16", 15, 3),
                                     ("e8my", 7, 32), ("fp16", 15, 100), ("sell_f32", 0, 130),
                                     ("e8my", 15, 136), ("fp16", 15, 8)])
def test_spmm(fmt, D, k):
    """Lane-group SpMM: k = 1 routes through the SpMV; k % 4 != 0 takes the
    scalar loads; k > 128 takes two passes. Every column equals the twin."""
    need_gpu()
    packsell = P()
    csr = I.random_csr(1500, 1200, 0.005, seed=k, empty_rows=0.05, long_gaps=True)
    A = encode_gpu(csr, fmt=fmt, D=D if D else 15)
    deq = csr.val.astype(np.float64) if fmt == "sell_f32" else O.encode(
        csr, D=D, fmt=FMT[fmt]).deq
    X = np.random.default_rng(k).uniform(-1, 1, (1200, k)).astype(np.float32)
    Y = packsell.packsell_spmm(A, dev(X)).cpu().numpy()
    ref = O.csr_spmm_f64(csr, deq, X.astype(np.float64))
    for r in range(k):  # each column is an SpMV: bitwise equal to the twin
        twin = O.csr_spmv_fma_f32(csr, deq.astype(np.float32), np.ascontiguousarray(X[:, r]))
        assert np.array_equal(Y[:, r].view(np.uint32), twin.view(np.uint32))
    assert np.abs(Y - ref).max() <= REL_TOL * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("fmt,D,k", [("fp16", 15, 3), ("e8my", 11, 8), ("fp16", 15, 64),
                                     ("fp16", 15, 100), ("e8my", 7, 4)])
def test_spmm_long_rows(fmt, D, k):
    """Rows of up to 4,096 words (slices wider than 32 words take the
    two-phase SpMM: columns of a round first, then gathers in batches)."""
    need_gpu()
    packsell = P()
    csr = I.zipf_irregular(20000, seed=k)
    A = encode_gpu(csr, fmt=fmt, D=D)
    assert A.max_width > 32
    X = np.random.default_rng(k).uniform(-1, 1, (csr.m, k)).astype(np.float32)
    Y = packsell.packsell_spmm(A, dev(X)).cpu().numpy()
    deq = O.encode(csr, D=D, fmt=FMT[fmt]).deq.astype(np.float32)
    for r in sorted({0, k // 2, k - 1}):
        twin = O.csr_spmv_fma_f32(csr, deq, np.ascontiguousarray(X[:, r]))
        assert np.array_equal(Y[:, r].view(np.uint32), twin.view(np.uint32)), f"column {r}"


@pytest.mark.parametrize("fmt,C,sigma,explicit,k", [("fp16", 32, 256, True, 16),
                                                     ("e8my", 8, 1, False, 12),
                                                     ("fp16", 1, 1, False, 32),
                                                     ("sell_f32", 16, 64, False, 24),
                                                     ("fp16", 32, 100, False, 64)])
def test_spmm_strided_layouts(fmt, C, sigma, explicit, k):
    """X and Y as column slices of wider arrays (ld = k + 3: scalar loads),
    other slice heights, no sorting, a non-power-of-two sigma, both orders."""
    need_gpu()
    packsell = P()
    csr = I.random_csr(900, 700, 0.01, seed=C + k, empty_rows=0.05, long_gaps=True)
    enc = None if fmt == "sell_f32" else O.encode(csr, C=C, sigma=sigma, D=11 if fmt == "e8my" else 15,
                                                  fmt=FMT[fmt])
    A = encode_gpu(csr, fmt=fmt, C=C, sigma=sigma, D=11 if fmt == "e8my" else 15,
                   explicit_perm=explicit)
    deq = csr.val.astype(np.float64) if enc is None else enc.deq
    Xw = np.random.default_rng(k).uniform(-1, 1, (700, k + 3)).astype(np.float32)
    Xd = dev(Xw)[:, 1:k + 1]
    Yd = torch.full((900, k + 3), float("nan"), device="cuda")
    packsell.packsell_spmm(A, Xd, Yd[:, 2:k + 2])
    Y = Yd.cpu().numpy()
    assert np.isnan(Y[:, :2]).all() and np.isnan(Y[:, k + 2:]).all()  # nothing written outside
    Y = Y[:, 2:k + 2]
    if explicit:
        Y = Y[np.argsort(O.storage_rows(O.encode(csr, C=C, sigma=sigma, D=15, fmt=O.FMT_FP16)))]
    if C == 1 and enc is not None:  # CSR order: the split-row SpMM, held to gamma_w
        assert_within_bound(Y, csr, deq, Xw[:, 1:k + 1], enc.words)
        return
    for r in range(k):
        twin = O.csr_spmv_fma_f32(csr, deq.astype(np.float32), np.ascontiguousarray(Xw[:, r + 1]))
        assert np.array_equal(Y[:, r].view(np.uint32), twin.view(np.uint32)), f"column {r}"


@pytest.mark.parametrize("fmt,sigma,explicit,k", [("fp16", 256, True, 8), ("e8my", 64, False, 12),
                                                  ("fp16", 1, False, 20), ("e8my", 256, True, 36),
                                                  ("fp16", 100, False, 64), ("fp16", 256, True, 64)])
def test_spmm_aligned_column_slices(fmt, sigma, explicit, k):
    """C = 32 with 16-byte-aligned column slices of wider arrays (ld = k + 8):
    the 16-byte gathers of the lane-group SpMM, in both row orders, with k
    not a multiple of a pass's column count (12, 20, 36). Every column equals
    the twin bit for bit and nothing outside Y's columns is written."""
    need_gpu()
    packsell = P()
    D = 11 if fmt == "e8my" else 15
    csr = I.random_csr(1000, 800, 0.012, seed=100 + k, empty_rows=0.05, long_gaps=True)
    enc = O.encode(csr, C=32, sigma=sigma, D=D, fmt=FMT[fmt])
    A = encode_gpu(csr, fmt=fmt, C=32, sigma=sigma, D=D, explicit_perm=explicit)
    Xw = np.random.default_rng(k).uniform(-1, 1, (800, k + 8)).astype(np.float32)
    Xd = dev(Xw)[:, 4:k + 4]
    Yd = torch.full((1000, k + 8), float("nan"), device="cuda")
    packsell.packsell_spmm(A, Xd, Yd[:, 4:k + 4])
    Y = Yd.cpu().numpy()
    assert np.isnan(Y[:, :4]).all() and np.isnan(Y[:, k + 4:]).all()
    Y = Y[:, 4:k + 4]
    if explicit:
        Y = Y[np.argsort(O.storage_rows(enc))]
    for r in range(k):
        twin = O.csr_spmv_fma_f32(csr, enc.deq.astype(np.float32), np.ascontiguousarray(Xw[:, r + 4]))
        assert np.array_equal(Y[:, r].view(np.uint32), twin.view(np.uint32)), f"column {r}"


def assert_within_bound(Y, csr, deq, X, words):
    """Every entry of Y (original row order) within gamma_w * sum_j |a_ij X_jq|
    of the oracle's FP64 product, w the stored words of the row."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    ref = O.csr_spmm_f64(csr, deq, X)
    absref = O.csr_spmm_f64(csr, np.abs(deq), np.abs(X))
    w = np.maximum(np.asarray(words, np.float64), 1.0)[:, None]
    u = 2.0 ** -24
    bound = (w * u / (1 - w * u)) * absref
    bad = np.argwhere(~(np.abs(Y.astype(np.float64) - ref) <= bound))
    assert bad.size == 0, f"{len(bad)} entries beyond gamma_w, first {bad[:3].tolist()}"


@pytest.mark.parametrize("fmt,D,sigma,k", [("fp16", 15, 1, 4), ("e8my", 11, 1, 16), ("fp16", 15, 256, 64),
                                           ("e8my", 5, 1, 3), ("fp16", 15, 1, 1), ("e8my", 3, 100, 8)])
def test_spmm_csr_order_split_rows(fmt, D, sigma, k):
    """SpMM on CSR-order matrices (C = 1) runs the split-row kernel: power-law
    rows up to 4,096 words (tiles and long rows), four columns per pass,
    every entry within gamma_w of the oracle, the same bits on a second run;
    k = 1 with a strided X takes the one-column form."""
    need_gpu()
    packsell = P()
    csr = I.zipf_irregular(20000, seed=40 + k)
    enc = O.encode(csr, C=1, sigma=sigma, D=D, fmt=FMT[fmt])
    A = encode_gpu(csr, fmt=fmt, D=D, C=1, sigma=sigma)
    X = np.random.default_rng(k).uniform(-1, 1, (csr.m, k)).astype(np.float32)
    if k == 1:  # a column of a wider array: not the SpMV route
        Xw = dev(np.repeat(X, 2, axis=1))
        Xd, Yd = Xw[:, :1], torch.empty(csr.n, 2, device="cuda")[:, :1]
    else:
        Xd, Yd = dev(X), torch.empty(csr.n, k, device="cuda")
    packsell.packsell_spmm(A, Xd, Yd)
    Y1 = Yd.cpu().numpy().copy()
    packsell.packsell_spmm(A, Xd, Yd)
    assert np.array_equal(Y1.view(np.uint32), Yd.cpu().numpy().view(np.uint32))
    assert_within_bound(Y1, csr, enc.deq, X, enc.words)


@pytest.mark.parametrize("fmt,D,sigma,k", [("fp16", 15, 1, 20), ("e8my", 7, 1, 36), ("fp16", 15, 64, 64),
                                           ("e8my", 11, 1, 100)])
def test_spmm_csr_order_wide_k(fmt, D, sigma, k):
    """CSR-order SpMM with 16 < k and 16-byte-aligned column slices (ld = k + 8;
    k = 100 takes two passes of 64 columns): the rows of a tile (at most 125
    words) are walked in stored order from the decoded table, so they equal
    the twin bit for bit; the longer rows, summed by lane groups and a
    butterfly, stay within gamma_w; nothing outside Y's columns is written."""
    need_gpu()
    packsell = P()
    csr = I.zipf_irregular(12000, seed=70 + k)
    enc = O.encode(csr, C=1, sigma=sigma, D=D, fmt=FMT[fmt])
    A = encode_gpu(csr, fmt=fmt, D=D, C=1, sigma=sigma)
    Xw = np.random.default_rng(k).uniform(-1, 1, (csr.m, k + 8)).astype(np.float32)
    Yd = torch.full((csr.n, k + 8), float("nan"), device="cuda")
    packsell.packsell_spmm(A, dev(Xw)[:, 4:k + 4], Yd[:, 4:k + 4])
    Yw = Yd.cpu().numpy()
    assert np.isnan(Yw[:, :4]).all() and np.isnan(Yw[:, k + 4:]).all()
    Y = Yw[:, 4:k + 4]
    X = Xw[:, 4:k + 4]
    assert_within_bound(Y, csr, enc.deq, X, enc.words)
    tile_rows = np.asarray(enc.words) <= 125
    assert tile_rows.sum() > 0.9 * csr.n and (~tile_rows).any()
    for r in sorted({0, 1, k // 2, k - 1}):
        twin = O.csr_spmv_fma_f32(csr, enc.deq.astype(np.float32), np.ascontiguousarray(X[:, r]))
        got = Y[:, r]
        assert np.array_equal(got[tile_rows].view(np.uint32), twin[tile_rows].view(np.uint32)), \
            f"column {r}"


@pytest.mark.parametrize("fmt,D", [("fp16", 15), ("e8my", 3), ("sell_f32", 15)])
def test_transpose_and_pattern_outer(fmt, D):
    need_gpu()
    packsell = P()
    csr = I.random_csr(700, 900, 0.01, seed=8, empty_rows=0.05, long_gaps=True)
    A = encode_gpu(csr, fmt=fmt, D=D, C=32, sigma=64, keep_rowptr=True)
    deq = csr.val.astype(np.float64) if fmt == "sell_f32" else O.encode(
        csr, C=32, sigma=64, D=D, fmt=FMT[fmt]).deq
    dy = I.uniform(700, seed=9)
    dx = packsell.packsell_spmv_transpose(A, dev(dy)).cpu().numpy()
    ref = O.csr_spmv_t_f64(csr, deq, dy.astype(np.float64))
    # FP32 products and atomic sums in any order: |error_j| <= gamma_(c_j + 1)
    # sum_i |a_ij dy_i| with c_j the nonzeros of column j
    absum = O.csr_spmv_t_f64(csr, np.abs(deq), np.abs(dy).astype(np.float64))
    cnt = np.bincount(csr.col, minlength=csr.m) + 1.0
    u = 2.0 ** -24
    assert np.all(np.abs(dx - ref) <= cnt * u / (1 - cnt * u) * absum)
    x = I.uniform(900, seed=10)
    out = packsell.packsell_pattern_outer(A, -1.0, dev(dy), dev(x)).cpu().numpy()
    row = np.repeat(np.arange(700), csr.row_lengths())
    want = (np.float32(-1.0) * dy[row]) * x[csr.col]
    assert np.array_equal(out.view(np.uint32), want.astype(np.float32).view(np.uint32))


@pytest.mark.parametrize("variant", [2, 3, 4, 9, 10])
def test_bounded_wait_runs_out_and_reports_timeout(variant):
    """The TMA-staged variants' waits for data are bounded. With the limit
    at 0 polls every first wait gives up: the kernel records
    PACKSELL_ERR_TIMEOUT in the matrix's status word, lets the copies it has
    issued land (the drain keeps the default limit) and returns, and the GPU
    stays usable; with the default limit restored the next launch gives the
    twin's bits again and the status word reads clean."""
    need_gpu()
    ps = P()
    csr = I.stencil27(24, seed=2)
    A = encode_gpu(csr, fmt="fp16", C=32, sigma=256)
    x = dev(I.uniform(csr.m, seed=3))
    ps.packsell_set_spmv_variant(A, variant)
    try:
        ps.packsell_set_wait_limit(0)
        ps.packsell_spmv(A, x)
        with pytest.raises(ps.PackSELLError) as e:
            ps.packsell_check_status(A)  # reads and clears the word
        assert e.value.code == 10  # PACKSELL_ERR_TIMEOUT
    finally:
        ps.packsell_set_wait_limit(-1)
    y = ps.packsell_spmv(A, x).cpu().numpy()
    ps.packsell_check_status(A)
    enc = O.encode(csr, C=32, sigma=256, D=15, fmt=O.FMT_FP16)
    twin = O.csr_spmv_fma_f32(csr, enc.deq.astype(np.float32), x.cpu().numpy())
    assert np.array_equal(y.view(np.uint32), twin.view(np.uint32))
