"""Shared helpers for the GPU parity tests."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")

FMT = {"fp16": O.FMT_FP16, "e8my": O.FMT_E8MY}


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def P():
    from paper_2604_13433_gb300 import build, packsell
    build.build()
    return packsell


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def encode_gpu(csr, fmt="fp16", **kw):
    return P().packsell_encode_csr(csr, fmt=fmt, **kw)


def assert_same_encoding(A, enc):
    """GPU encoding vs oracle encoding: offsets, perm and words bit-exact."""
    arr = P().packsell_arrays(A)
    assert A.k_left == enc.k_left
    assert (A.n_words, A.n_dummies, A.n_pad) == (enc.n_words, enc.n_dummies, enc.n_pad)
    assert np.array_equal(arr["offset"], enc.offset)
    if A.sigma > 1:
        assert np.array_equal(arr["perm"], enc.perm)
    if "pack" in arr:
        bad = np.nonzero(arr["pack"] != enc.pack)[0]
        assert bad.size == 0, f"{bad.size} words differ, first at {bad[:5]}"
