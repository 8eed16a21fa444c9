"""Run in a child process by test_gpu_checks.py, with PACKSELL_CHECKS=1: the
bounds-check build of the library (libpacksell_checks.so).

1. On valid matrices every checked product gives the thread-per-row twin's
   bits (or the split rows' bound) and packsell_check_status reports OK.
2. One word of an encoded matrix is rewritten so that its column decodes to
   m, one past the end of x; every checked product then skips that gather
   and packsell_check_status reports PACKSELL_ERR_CHECK with index m. The
   column is exactly m, so even an unchecked gather would stay inside x's
   allocation (torch rounds it up to 512 bytes).
Prints "checks ok" on success."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2604_13433_gb300 import build, inputs as I  # noqa: E402

assert os.environ.get("PACKSELL_CHECKS") == "1"
build.build(checks=True)
from paper_2604_13433_gb300 import packsell as ps  # noqa: E402

assert ps.lib().packsell_checks_build() == 1


def words_view(A):
    class _V:
        pass
    v = _V()
    v.__cuda_array_interface__ = {"shape": (A.n_words,), "typestr": "<i4",
                                  "data": (A.info.pack, False), "version": 3}
    return torch.as_tensor(v, device="cuda")


def status():
    code = ps.lib().packsell_check_status(A_handle[0], None)
    return code, ps.lib().packsell_last_error().decode()


A_handle = [None]


def run_all(A, x, m):
    """Every product the library has for this layout; returns the outputs."""
    out = {}
    if A.C == 32:
        for v in (1, 5, 7, 13) + ((12,) if A.max_width <= 16 else ()):
            ps.packsell_set_spmv_variant(A, v)
            out[f"v{v}"] = ps.packsell_spmv(A, x).clone()
        ps.packsell_set_spmv_variant(A, 0)
        out["spmm"] = ps.packsell_spmm(A, x[:, None].repeat(1, 4).contiguous()).clone()
        out["transpose"] = ps.packsell_spmv_transpose(
            A, torch.ones(A.n, device="cuda")).clone()
    else:
        for v in (11, 14):
            ps.packsell_set_spmv_variant(A, v)
            out[f"v{v}"] = ps.packsell_spmv(A, x).clone()
        ps.packsell_set_spmv_variant(A, 0)
        for k in (4, 20):  # the split-row SpMM and, above k = 16, the table walk
            out[f"spmm{k}"] = ps.packsell_spmm(A, x[:, None].repeat(1, k).contiguous()).clone()
        y = torch.empty(A.n, device="cuda")
        B = ps.PackSELLBatch([A], [x], [y])
        B.spmv()
        out["batch"] = y.clone()
    torch.cuda.synchronize()
    return out


for C in (32, 1):
    csr = I.random_csr(700, 600, 0.02, seed=11 + C, empty_rows=0.05)
    m = csr.m
    A = ps.packsell_encode_csr(csr, fmt="fp16", D=15, C=C, sigma=1)
    A_handle[0] = A.handle
    enc = O.encode(csr, C=C, sigma=1, D=15, fmt=O.FMT_FP16)
    x = torch.from_numpy(I.uniform(m, seed=3)).cuda()
    twin = O.csr_spmv_fma_f32(csr, enc.deq.astype(np.float32), x.cpu().numpy())
    good = run_all(A, x, m)
    assert status() == (0, ""), status()
    key = "v1" if C == 32 else "v11"  # the stored-order chains: the twin's bits
    assert np.array_equal(good[key].cpu().numpy().view(np.uint32), twin.view(np.uint32))
    if C == 1:  # rows of at most 125 words: the table walk's stored-order chain
        assert np.array_equal(good["spmm20"][:, 7].cpu().numpy().view(np.uint32), twin.view(np.uint32))

    # rewrite a row's last value word so that it decodes to column m
    words = words_view(A)
    arr = ps.packsell_arrays(A)["pack"]
    row = int(np.argmax(np.diff(csr.rowptr)))  # a row with values (sigma = 1: storage row)
    last_col = int(csr.col[csr.rowptr[row + 1] - 1])
    k, l = row // C, row % C
    s0 = int(enc.offset[k])
    slots = [s0 + j * C + l for j in range((int(enc.offset[k + 1]) - s0) // C)]
    at = max(p for p in slots if arr[p] & 1)
    d_old = (int(arr[at]) >> 1) & 0x7FFF
    d_new = d_old + (m - last_col)
    assert d_new < (1 << 15)
    new_word = (int(arr[at]) & ~(0x7FFF << 1)) | (d_new << 1)
    words[at] = np.array(new_word, np.uint32).view(np.int32).item()
    torch.cuda.synchronize()
    run_all(A, x, m)
    code, msg = status()
    assert code == 11 and f"first index {m})" in msg, (code, msg)
    # one product at a time: each checked kernel reports its own skip
    for name in list(good):
        if name.startswith("v"):
            ps.packsell_set_spmv_variant(A, int(name[1:]))
            ps.packsell_spmv(A, x)
            torch.cuda.synchronize()
            code, msg = status()
            assert code == 11, (C, name, code, msg)
    ps.packsell_set_spmv_variant(A, 0)
    for name in list(good):
        if name.startswith("spmm") and name != "spmm":
            k = int(name[4:])
            ps.packsell_spmm(A, x[:, None].repeat(1, k).contiguous())
            torch.cuda.synchronize()
            code, msg = status()
            assert code == 11 and f"first index {m})" in msg, (C, name, code, msg)
    # restore the word: no skips again
    words[at] = np.array(int(arr[at]), np.uint32).view(np.int32).item()
    torch.cuda.synchronize()
    run_all(A, x, m)
    assert status() == (0, ""), status()
print("checks ok")
