"""GPU encoder vs the oracle: offsets, perm and every packed word bit-exact
(§4.1-§4.3), plus error statuses and export/import (through the C ABI)."""
import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I

from _gpu import FMT, P, assert_same_encoding, dev, encode_gpu, need_gpu, torch

pytestmark = pytest.mark.gpu

CASES = [
    # n, m, density, C, sigma, fmt, D, empty-row fraction, long gaps
    (1, 1, 1.0, 32, 256, "fp16", 15, 0.0, False),
    (37, 53, 0.2, 32, 256, "fp16", 15, 0.1, False),
    (100, 100, 0.05, 4, 8, "e8my", 1, 0.2, True),
    (200, 70, 0.3, 8, 16, "e8my", 2, 0.0, True),
    (130, 400, 0.02, 32, 1, "e8my", 7, 0.3, True),
    (1000, 1000, 0.01, 32, 256, "e8my", 11, 0.05, True),
    (300, 90, 0.1, 1, 300, "e8my", 3, 0.0, True),
    (64, 5000, 0.01, 16, 32, "e8my", 22, 0.0, True),
    (2000, 3000, 0.005, 64, 512, "fp16", 15, 0.1, True),
    (5000, 5000, 0.002, 32, 4096, "e8my", 9, 0.02, True),
    (3000, 300, 0.02, 1024, 3000, "e8my", 5, 0.0, True),
    (70000, 70000, 0.0002, 32, 65536, "fp16", 15, 0.05, True),  # the largest sigma
]


@pytest.mark.parametrize("case", CASES)
def test_encode_matches_oracle(case):
    need_gpu()
    n, m, dens, C, sigma, fmt, D, empty, gaps = case
    csr = I.random_csr(n, m, dens, seed=n + 7 * m, empty_rows=empty, long_gaps=gaps)
    enc = O.encode(csr, C=C, sigma=sigma, D=D, fmt=FMT[fmt])
    A = encode_gpu(csr, fmt=fmt, C=C, sigma=sigma, D=D)
    assert_same_encoding(A, enc)


@pytest.mark.parametrize("fmt,D", [("fp16", 15), ("e8my", 15), ("e8my", 11), ("e8my", 7),
                                   ("e8my", 1)])
def test_encode_stencil27_32(fmt, D):
    need_gpu()
    csr = I.stencil27(32, seed=1)
    enc = O.encode(csr, C=32, sigma=256, D=D, fmt=FMT[fmt])
    assert_same_encoding(encode_gpu(csr, fmt=fmt, D=D), enc)


def test_encode_f64_values_match_oracle():
    need_gpu()
    csr = I.poisson7_varcoef(12, seed=2)  # float64 values
    for fmt, D in (("fp16", 15), ("e8my", 10), ("e8my", 1)):
        enc = O.encode(csr, C=32, sigma=256, D=D, fmt=FMT[fmt])
        assert_same_encoding(encode_gpu(csr, fmt=fmt, D=D), enc)


def test_encode_config1_and_empty():
    need_gpu()
    a = I.poisson5(64)
    for sigma in (1, 256):
        A = encode_gpu(a, C=32, sigma=sigma)
        assert (A.k_left, A.n_words, A.n_dummies, A.n_pad) == (64, 20352, 0, 128)
        assert_same_encoding(A, O.encode(a, C=32, sigma=sigma))
    e = I.CSR(n=5, m=7, rowptr=np.zeros(6, np.int64), col=np.zeros(0, np.int32),
              val=np.zeros(0, np.float32))
    A = encode_gpu(e, C=4, sigma=2)
    assert A.n_words == 0 and list(P().packsell_arrays(A)["offset"]) == [0, 0, 0]


def test_quantizer_exhaustive_sample():
    """Every FP32 exponent, many mantissas: GPU value fields equal the oracle's."""
    need_gpu()
    rng = np.random.default_rng(0)
    b = rng.integers(0, 2 ** 32, 400000, dtype=np.uint64).astype(np.uint32)
    v = b.view(np.float32)
    v = v[np.isfinite(v) & (np.abs(v) < 6e4)]
    v = np.concatenate([v, np.float32([0.0, -0.0, 2 ** -24, 2 ** -25, 3 * 2 ** -25, 65504.0])])
    nnz = v.size
    # one row per value so each value is stored as a word of its own
    csr = I.CSR(n=nnz, m=1, rowptr=np.arange(nnz + 1, dtype=np.int64),
                col=np.zeros(nnz, np.int32), val=v)
    for fmt, D in (("fp16", 15), ("e8my", 1), ("e8my", 7), ("e8my", 12), ("e8my", 22)):
        enc = O.encode(csr, C=32, sigma=1, D=D, fmt=FMT[fmt])
        A = encode_gpu(csr, fmt=fmt, C=32, sigma=1, D=D)
        assert_same_encoding(A, enc)


@pytest.mark.parametrize("kind", ["unsorted", "dup", "range", "fp16_overflow", "nan",
                                  "k_left", "e8my_overflow"])
def test_encode_errors(kind):
    need_gpu()
    packsell = P()
    rowptr, col, val, kw = np.array([0, 2]), np.array([1, 3], np.int32), \
        np.ones(2, np.float32), {}
    code = {"unsorted": 2, "dup": 2, "range": 4, "fp16_overflow": 4, "nan": 3, "k_left": 1,
            "e8my_overflow": 4}[kind]
    if kind == "unsorted":
        col = np.array([3, 1], np.int32)
    elif kind == "dup":
        col = np.array([2, 2], np.int32)
    elif kind == "range":
        col = np.array([1, 5], np.int32)
    elif kind == "fp16_overflow":
        val = np.array([1.0, 70000.0], np.float32)
    elif kind == "nan":
        val = np.array([1.0, np.nan], np.float32)
    elif kind == "k_left":
        rowptr, col, val = np.array([0, 1, 2]), np.array([1, 0], np.int32), np.ones(2, np.float32)
        kw = {"k_left": 0, "sigma": 1}
    elif kind == "e8my_overflow":
        val = np.array([1.0, np.finfo(np.float32).max], np.float32)
        kw = {"fmt": "e8my", "D": 1}
    n = rowptr.size - 1
    with pytest.raises(packsell.PackSELLError) as e:
        packsell.packsell_encode(dev(rowptr.astype(np.int64)), dev(col), dev(val), n, 5, **kw)
    assert e.value.code == code


def test_export_import_roundtrip_and_corruption():
    need_gpu()
    packsell = P()
    csr = I.random_csr(500, 600, 0.02, seed=5, long_gaps=True)
    A = encode_gpu(csr, fmt="e8my", D=4, C=32, sigma=64)
    blob = packsell.packsell_export(A)
    B = packsell.packsell_import(blob)
    assert (B.n, B.m, B.nnz, B.n_words, B.k_left) == (A.n, A.m, A.nnz, A.n_words, A.k_left)
    x = dev(I.uniform(600, seed=1))
    assert torch.equal(packsell.packsell_spmv(A, x), packsell.packsell_spmv(B, x))
    # a dummy word whose delta jumps past the last column must be rejected
    hdr = len(blob) - 4 * A.n_words
    words = np.frombuffer(blob, np.uint32, A.n_words, hdr).copy()
    words[int(np.nonzero(words & 1)[0][0])] = np.uint32(0x7FFFFFFE)
    with pytest.raises(packsell.PackSELLError) as e:
        packsell.packsell_import(blob[:hdr] + words.tobytes())
    assert e.value.code == 9
    with pytest.raises(packsell.PackSELLError):
        packsell.packsell_import(blob[: len(blob) // 2])
    # a header whose widest slice disagrees with the offsets (the kernels size
    # their rounds by it): int32 at byte 96 of the header
    assert int(np.frombuffer(blob, np.int32, 1, 96)[0]) == A.max_width
    bad = bytearray(blob)
    bad[96:100] = np.int32(1).tobytes()
    with pytest.raises(packsell.PackSELLError) as e:
        packsell.packsell_import(bytes(bad))
    assert e.value.code == 9


@pytest.mark.gpu
@pytest.mark.parametrize("fmt,D", [("fp16", 15), ("e8my", 9), ("fixed", 11), ("w16_e4m3", 7),
                                   ("sell_f16", 15), ("sell_f32", 15), ("sell_f64", 15),
                                   ("w64_e11my", 11)])
def test_export_import_roundtrip_every_format(fmt, D):
    """Every storage format survives export and import: the same arrays,
    the same fixed-point exponent and the same product bits."""
    need_gpu()
    ps = P()
    csr = I.random_csr(700, 900, 0.02, seed=D, empty_rows=0.05, long_gaps=True)
    A = encode_gpu(csr, fmt=fmt, D=D, C=32, sigma=64)
    B = ps.packsell_import(ps.packsell_export(A))
    assert (B.format, B.n_words, B.nnz, B.value_exp) == (A.format, A.n_words, A.nnz, A.value_exp)
    a, b = ps.packsell_arrays(A), ps.packsell_arrays(B)
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    if fmt in ("sell_f64", "w64_e11my"):
        x = dev(I.uniform(900, seed=2).astype(np.float64))
        assert torch.equal(ps.packsell_spmv_f64(A, x), ps.packsell_spmv_f64(B, x))
    else:
        x = dev(I.uniform(900, seed=2))
        assert torch.equal(ps.packsell_spmv(A, x), ps.packsell_spmv(B, x))


@pytest.mark.gpu
def test_import_rejects_sell_f16_slot_after_padding():
    """FP16 SELL pads a row with column -1 and its product stops at the
    first -1: a stored column after one, or one more stored column than
    nnz, is a corrupt blob."""
    need_gpu()
    ps = P()
    C = 32
    csr = I.random_csr(300, 300, 0.03, seed=3, empty_rows=0.1)
    A = encode_gpu(csr, fmt="sell_f16", C=C, sigma=1)
    blob = ps.packsell_export(A)
    off = ps.packsell_arrays(A)["offset"]
    cols_at = len(blob) - 4 * A.n_words
    cols = np.frombuffer(blob, np.int32, A.n_words, cols_at).copy()
    assert ps.packsell_import(blob).nnz == A.nnz
    # a row's last stored slot q followed by padding at q + C, same slice
    slice_end = np.repeat(off[1:], np.diff(off))
    q = np.nonzero((cols[:-C] >= 0) & (cols[C:] == -1) & (np.arange(A.n_words - C) + C <
                                                           slice_end[:-C]))[0][0]
    swapped = cols.copy()
    swapped[q], swapped[q + C] = -1, cols[q]  # same count, wrong order
    extra = cols.copy()
    extra[q + C] = 0  # one stored column too many
    for bad in (swapped, extra):
        with pytest.raises(ps.PackSELLError) as e:
            ps.packsell_import(blob[:cols_at] + bad.tobytes())
        assert e.value.code == 9


def _device_words(ptr, count):
    """A torch view (int32) of a matrix's device word array."""
    class _View:
        pass
    v = _View()
    v.__cuda_array_interface__ = {"shape": (count,), "typestr": "<i4", "data": (ptr, False),
                                  "version": 3}
    return torch.as_tensor(v, device="cuda")


@pytest.mark.gpu
def test_validate_finds_corrupted_words():
    """packsell_validate decodes the matrix on the device: a word whose delta
    runs past the last column, and a padding word turned into a value, are
    CORRUPT; the restored matrix validates again. (No product runs on the
    corrupted matrix.)"""
    need_gpu()
    ps = P()
    csr = I.random_csr(500, 600, 0.02, seed=5, long_gaps=True)
    A = encode_gpu(csr, fmt="e8my", D=4, C=32, sigma=64)
    ps.packsell_validate(A)
    words = _device_words(A.info.pack, A.n_words)
    arr = ps.packsell_arrays(A)["pack"]
    assert np.array_equal(words.cpu().numpy().view(np.uint32), arr)
    first_value = int(np.nonzero(arr & 1)[0][0])
    first_pad = int(np.nonzero(arr == 0)[0][0])
    for at, bad, why in ((first_value, 0x7FFFFFFE, "bad word"),  # a dummy of 2^30 - 1
                         (first_pad, 0x3F800001, "do not match nnz")):  # 1.0, delta 0
        keep = int(words[at].item())
        words[at] = bad
        torch.cuda.synchronize()
        with pytest.raises(ps.PackSELLError) as e:
            ps.packsell_validate(A)
        assert e.value.code == 9 and why in str(e.value), str(e.value)
        words[at] = keep
        torch.cuda.synchronize()
        ps.packsell_validate(A)
