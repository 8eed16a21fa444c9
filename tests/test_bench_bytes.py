"""bench.py's algorithmic bytes per SpMV (the roofline's numerator) against
the arrays the oracle's encoder produces, and the headline's figure from the
hand-derived word count of the 27-point 128^3 matrix (CPU only)."""
import importlib.util
import os
from types import SimpleNamespace

import numpy as np
import pytest

import oracle as O
from paper_2604_13433_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_bytes_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _matrix(enc, explicit, fmt):
    """The fields of a PackSELLMatrix that the byte count reads."""
    pb = 0 if enc.sigma == 1 else (1 if enc.sigma <= 256 else 2)
    return SimpleNamespace(n=enc.n, m=enc.m, n_words=int(enc.pack.size),
                           n_slices=enc.offset.size - 1, perm_bytes=pb,
                           explicit_perm=explicit, format=fmt)


@pytest.mark.parametrize("explicit", [False, True])
@pytest.mark.parametrize("sigma", [1, 256, 1024])
def test_bytes_are_the_encoded_arrays(explicit, sigma):
    b = _bench()
    csr = I.stencil27(12, seed=1)
    perm = 0 if (explicit or sigma == 1) else csr.n * (1 if sigma <= 256 else 2)
    vectors = 4 * csr.m + 4 * csr.n  # x read once, y written once (FP32)
    enc = O.encode(csr, C=32, sigma=sigma, D=15, fmt=O.FMT_FP16)
    assert b.spmv_bytes(_matrix(enc, explicit, 1), False) == \
        enc.pack.nbytes + enc.offset.astype(np.int64).nbytes + perm + vectors
    e16 = O.encode16(csr, C=32, sigma=sigma)
    assert e16.pack.dtype == np.uint16
    assert b.spmv_bytes(_matrix(e16, explicit, 5), False) == \
        e16.pack.nbytes + e16.offset.astype(np.int64).nbytes + perm + vectors
    # 64-bit words: FP64 x and y
    e64 = O.encode64(csr, C=32, sigma=sigma, D=11)
    assert e64.pack.dtype == np.uint64
    assert b.spmv_bytes(_matrix(e64, explicit, 8), False) == \
        e64.pack.nbytes + e64.offset.astype(np.int64).nbytes + perm + 2 * vectors


def test_headline_bytes():
    # 27-point 128^3, C = 32, D = 15, explicit order: 146,688 x 382 = 56,034,816
    # words (the hand-derived count the oracle is pinned to), 65,536 slices
    b = _bench()
    n = 128 ** 3
    A = SimpleNamespace(n=n, m=n, n_words=146_688 * 382, n_slices=n // 32, perm_bytes=1,
                        explicit_perm=True, format=1)
    assert b.spmv_bytes(A, False) == 241_440_776
