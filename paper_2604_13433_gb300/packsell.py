"""Python binding of the PackSELL C ABI (``include/packsell.h``).

Argument marshalling only: every function here checks tensor devices, dtypes
and shapes, passes raw device pointers and the current CUDA stream to the
library, and turns a non-zero status into :class:`PackSELLError`. Every
computation runs in ``libpacksell.so``'s CUDA kernels; there is no CPU path,
and a missing library raises at the first call.

Function names follow the C ABI (``packsell_encode``, ``packsell_spmv`` ...).
PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpacksell.so")
# the bounds-check build, loaded instead when PACKSELL_CHECKS=1
LIB_CHECKS_PATH = os.path.join(_HERE, "libpacksell_checks.so")

FMT_FP16, FMT_E8MY, FMT_SELL_F32, FMT_SELL_F64, FMT_W16_E4M3, FMT_SELL_F16 = 1, 2, 3, 4, 5, 6
FMT_FIXED, FMT_W64_E11MY = 7, 8
_FORMATS = {"fp16": FMT_FP16, "e8my": FMT_E8MY, "sell_f32": FMT_SELL_F32,
            "sell_f64": FMT_SELL_F64, "w16_e4m3": FMT_W16_E4M3, "sell_f16": FMT_SELL_F16,
            "fixed": FMT_FIXED, "w64_e11my": FMT_W64_E11MY}

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSORTED", 3: "NONFINITE", 4: "RANGE", 5: "CUDA",
          6: "NOT_CONVERGED", 7: "BREAKDOWN", 8: "NO_MEMORY", 9: "CORRUPT", 10: "TIMEOUT",
          11: "CHECK"}
SPMV_AUTO, SPMV_ROWTHREAD, SPMV_BULK = 0, 1, 2
SPMV_BULK_VARIANTS = (2, 3, 4)
SPMV_PREFETCH = (5, 6)
SPMV_DUAL = (7, 8)
SPMV_STAGE = (9, 10)
SPMV_CSR = 11  # C = 1 PackSELL matrices (rows stored one after another)
SPMV_PIPE = 12  # C = 32, next row's words loaded while the current one is gathered
SPMV_PDL = 13  # C = 32, variant 5 with programmatic dependent launch
SPMV_SPLIT = 14  # C = 1, all lanes of a warp share a tile's words (split rows)
SPMV_VARIANTS = 14


class PackSELLError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class Params(ctypes.Structure):
    _fields_ = [("C", ctypes.c_int32), ("sigma", ctypes.c_int32), ("D", ctypes.c_int32),
                ("format", ctypes.c_int32), ("explicit_perm", ctypes.c_int32),
                ("keep_rowptr", ctypes.c_int32), ("k_left", ctypes.c_int64)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("params", Params), ("n_slices", ctypes.c_int64), ("n_words", ctypes.c_int64),
                ("n_dummies", ctypes.c_int64), ("n_pad", ctypes.c_int64),
                ("max_width", ctypes.c_int32), ("perm_bytes", ctypes.c_int32),
                ("bytes", ctypes.c_int64), ("pack", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("offset", ctypes.c_void_p), ("perm", ctypes.c_void_p),
                ("value_exp", ctypes.c_int32)]


class FormatTrial(ctypes.Structure):
    _fields_ = [("params", Params), ("error", ctypes.c_double), ("admissible", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("n_words", ctypes.c_int64), ("bytes", ctypes.c_double),
                ("ms", ctypes.c_double)]


class F3ROpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("m1", ctypes.c_int32), ("m2", ctypes.c_int32),
                ("m3", ctypes.c_int32), ("m4", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("omega", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("m_in", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


class SolveResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("relres", ctypes.c_double), ("relres_true", ctypes.c_double),
                ("seconds", ctypes.c_double)]


_lib = None

# symbol -> (restype, argtypes)
_P, _I64, _I32, _F32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
SIGNATURES = {
    "packsell_params_default": (None, [_P]),
    "packsell_version": (ctypes.c_char_p, []),
    "packsell_last_error": (ctypes.c_char_p, []),
    "packsell_encode": (ctypes.c_int, [_P, _I64, _I64, _I64, _P, _P, _P, _I32, _P, _P]),
    "packsell_destroy": (ctypes.c_int, [_P]),
    "packsell_get_info": (ctypes.c_int, [_P, _P]),
    "packsell_export": (ctypes.c_int, [_P, _P, _P, _P]),
    "packsell_import": (ctypes.c_int, [_P, ctypes.c_size_t, _P, _P]),
    "packsell_spmv": (ctypes.c_int, [_P, _P, _P, _P]),
    "packsell_spmv_f64": (ctypes.c_int, [_P, _P, _P, _P]),
    "packsell_spmm": (ctypes.c_int, [_P, _I32, _P, _I64, _P, _I64, _P]),
    "packsell_spmv_transpose": (ctypes.c_int, [_P, _P, _P, _P]),
    "packsell_pattern_outer": (ctypes.c_int, [_P, _F32, _P, _P, _P, _P]),
    "packsell_set_spmv_variant": (ctypes.c_int, [_P, _I32]),
    "packsell_check_status": (ctypes.c_int, [_P, _P]),
    "packsell_validate": (ctypes.c_int, [_P, _P]),
    "packsell_checks_build": (ctypes.c_int32, []),
    "packsell_tune_spmv": (ctypes.c_int, [_P, _P, _P, _I32, _P, _P]),
    "packsell_quantize": (ctypes.c_int, [_I32, _I32, _I64, _P, _I32, _P, _P, _P]),
    "packsell_set_wait_limit": (ctypes.c_int, [_I64]),
    "packsell_f3r_opts_default": (None, [_P]),
    "packsell_f3r": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "packsell_tune_format": (ctypes.c_int, [_I64, _I64, _I64, _P, _P, _P, _I32, ctypes.c_double,
                                            _P, _P, _I32, _P, _P, _I32, _P, _P]),
    "packsell_pcg_workspace_bytes": (ctypes.c_size_t, [_I64, _I32, _I32, _I32]),
    "packsell_pcg": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P, _P, _P]),
    "packsell_pcg_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "packsell_pattern_outer_f64": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, _P, _P]),
    "packsell_spmv_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "packsell_reorder_rcm": (ctypes.c_int, [_I64, _P, _P, _P]),
    "packsell_permute_csr": (ctypes.c_int, [_I64, _P, _P, _P, _I32, _P, _P, _P, _P]),
    "packsell_pcg_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t,
                                             _P, _P]),
    "packsell_inv_diag": (ctypes.c_int, [_P, _P, _P]),
    "packsell_storage_rows": (ctypes.c_int, [_P, _P, _P]),
    "packsell_spmv_x16": (ctypes.c_int, [_P, _P, _P, _P]),
    "packsell_spmv_host": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "packsell_batch_create": (ctypes.c_int, [_I32, _P, _P, _P, _P, _P]),
    "packsell_batch_spmv": (ctypes.c_int, [_P, _P]),
    "packsell_batch_create_spmm": (ctypes.c_int, [_I32, _P, _I32, _P, _P, _P, _P, _P, _P]),
    "packsell_batch_spmm": (ctypes.c_int, [_P, _P]),
    "packsell_batch_info": (ctypes.c_int, [_P, _P, _P, _P]),
    "packsell_batch_destroy": (ctypes.c_int, [_P]),
}


def lib():
    """Load ``libpacksell.so`` (built in-tree; ``libpacksell_checks.so`` when
    the environment sets PACKSELL_CHECKS=1); raise if it is missing."""
    global _lib
    if _lib is None:
        checks = os.environ.get("PACKSELL_CHECKS") == "1"
        path = LIB_CHECKS_PATH if checks else LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with `python -m paper_2604_13433_gb300.build"
                f"{' --checks' if checks else ''}` (there is no CPU fallback)")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int):
    if code != 0:
        raise PackSELLError(code, lib().packsell_last_error().decode())


def _stream(stream=None) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, name: str, numel=None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


class PackSELLMatrix:
    """Owner of an encoded matrix (a ``packsell_matrix*``)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        info = Info()
        _check(lib().packsell_get_info(self._h, ctypes.byref(info)))
        self.info = info
        self.n, self.m, self.nnz = info.n, info.m, info.nnz
        p = info.params
        self.C, self.sigma, self.D, self.format = p.C, p.sigma, p.D, p.format
        self.explicit_perm = bool(p.explicit_perm)
        self.k_left = p.k_left
        self.n_slices, self.n_words = info.n_slices, info.n_words
        self.n_dummies, self.n_pad = info.n_dummies, info.n_pad
        self.max_width, self.perm_bytes, self.bytes = info.max_width, info.perm_bytes, info.bytes
        self.value_exp = info.value_exp

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().packsell_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __repr__(self):
        return (f"PackSELLMatrix(n={self.n}, m={self.m}, nnz={self.nnz}, C={self.C}, "
                f"sigma={self.sigma}, D={self.D}, format={self.format}, words={self.n_words})")


def packsell_version() -> str:
    return lib().packsell_version().decode()


def packsell_encode(rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, n: int, m: int,
                    *, C: int = 32, sigma: int = 256, D: int = 15, fmt="fp16",
                    explicit_perm: bool = False, keep_rowptr: bool = False, k_left: int = -1,
                    stream=None) -> PackSELLMatrix:
    """Encode a CSR matrix held in CUDA tensors (rowptr int64 [n+1], col int32
    [nnz], val float32/float64 [nnz]). Synchronises the stream once."""
    fmt_code = _FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    nnz = col.numel()
    prm = Params(C, sigma, D, fmt_code, int(explicit_perm), int(keep_rowptr), k_left)
    if val.dtype not in (torch.float32, torch.float64):
        raise TypeError("val must be float32 or float64")
    h = ctypes.c_void_p()
    _check(lib().packsell_encode(
        ctypes.byref(prm), n, m, nnz, _dev(rowptr, torch.int64, "rowptr", n + 1),
        _dev(col, torch.int32, "col") if nnz else None,
        _dev(val, val.dtype, "val", nnz) if nnz else None, int(val.dtype == torch.float64),
        _stream(stream), ctypes.byref(h)))
    return PackSELLMatrix(h.value)


def packsell_set_wait_limit(polls: int) -> None:
    """Polls before the TMA-staged SpMV variants give up a wait for data
    (negative: the default); a diagnostics knob for the timeout path."""
    _check(lib().packsell_set_wait_limit(int(polls)))


def packsell_quantize(val: torch.Tensor, fmt="fp16", D: int = 15, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """The value quantiser of §4.2.2 on a CUDA tensor (float32 or float64):
    the uint32 value fields (as an int32 tensor of the same bits) that the
    encoder places in the words' upper bits."""
    fmt_code = _FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    if val.dtype not in (torch.float32, torch.float64):
        raise TypeError("val must be float32 or float64")
    n = val.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=val.device)
    bad = ctypes.c_int64(-1)
    _check(lib().packsell_quantize(fmt_code, D, n, _dev(val, val.dtype, "val", n) if n else None,
                                   int(val.dtype == torch.float64),
                                   _dev(out, torch.int32, "out", n) if n else None,
                                   ctypes.byref(bad), _stream(stream)))
    return out


_FORMAT_NAMES = {FMT_FP16: "fp16", FMT_E8MY: "e8my"}


def packsell_tune_format(rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, n: int,
                         m: int, max_error: float, x: torch.Tensor, y: torch.Tensor | None = None,
                         reps: int = 20, stream=None):
    """Pick slice height, sort block, value format and delta bits for a CSR
    matrix under a backward-error ceiling (packsell_tune_format). Returns
    (params, trials): params a dict of the keyword arguments for
    packsell_encode (C, sigma, D, fmt), trials one dict per candidate."""
    if y is None:
        y = torch.empty(n, dtype=torch.float32, device=x.device)
    if val.dtype not in (torch.float32, torch.float64):
        raise TypeError("val must be float32 or float64")
    nnz = col.numel()
    best = Params()
    cap = 32
    trials = (FormatTrial * cap)()
    cnt = ctypes.c_int32()
    _check(lib().packsell_tune_format(
        n, m, nnz, _dev(rowptr, torch.int64, "rowptr", n + 1), _dev(col, torch.int32, "col"),
        _dev(val, val.dtype, "val", nnz), int(val.dtype == torch.float64), float(max_error),
        _dev(x, torch.float32, "x", m), _dev(y, torch.float32, "y", n), reps, ctypes.byref(best),
        trials, cap, ctypes.byref(cnt), _stream(stream)))
    params = {"C": best.C, "sigma": best.sigma, "D": best.D, "fmt": _FORMAT_NAMES[best.format]}
    out = []
    for t in trials[:cnt.value]:
        out.append({"C": t.params.C, "sigma": t.params.sigma, "D": t.params.D,
                    "fmt": _FORMAT_NAMES[t.params.format], "error": t.error,
                    "admissible": bool(t.admissible), "variant": t.variant, "n_words": t.n_words,
                    "bytes": t.bytes, "ms": t.ms})
    return params, out


def _host(a: np.ndarray, dtype, name: str) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != dtype:
        raise TypeError(f"{name} must be {np.dtype(dtype)}, got {a.dtype}")
    return a


def packsell_reorder_rcm(rowptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Reverse Cuthill-McKee order of a square host CSR pattern (host code):
    perm[k] = the original row placed at position k (int32)."""
    rowptr, col = _host(rowptr, np.int64, "rowptr"), _host(col, np.int32, "col")
    n = rowptr.size - 1
    perm = np.empty(max(n, 0), np.int32)
    _check(lib().packsell_reorder_rcm(n, rowptr.ctypes.data, col.ctypes.data, perm.ctypes.data))
    return perm


def packsell_permute_csr(rowptr: np.ndarray, col: np.ndarray, val: np.ndarray | None,
                         perm: np.ndarray):
    """B = P A P^T on host CSR arrays (host code): returns (rowptr, col, val)
    of B; val is None when not given."""
    rowptr, col = _host(rowptr, np.int64, "rowptr"), _host(col, np.int32, "col")
    perm = _host(perm, np.int32, "perm")
    n = rowptr.size - 1
    if perm.size != n:
        raise ValueError(f"perm must have {n} elements")
    f64 = 0
    if val is not None:
        val = np.ascontiguousarray(val)
        if val.dtype not in (np.float32, np.float64):
            raise TypeError("val must be float32 or float64")
        f64 = int(val.dtype == np.float64)
    orp = np.empty(n + 1, np.int64)
    ocl = np.empty(col.size, np.int32)
    ovl = np.empty(col.size, val.dtype) if val is not None else None
    _check(lib().packsell_permute_csr(n, rowptr.ctypes.data, col.ctypes.data,
                                      val.ctypes.data if val is not None else None, f64,
                                      perm.ctypes.data, orp.ctypes.data, ocl.ctypes.data,
                                      ovl.ctypes.data if ovl is not None else None))
    return orp, ocl, ovl


def packsell_encode_csr(csr, device="cuda", **kw) -> PackSELLMatrix:
    """Encode a host CSR (``inputs.CSR``): copy its arrays to the device first."""
    rp = torch.from_numpy(csr.rowptr).to(device)
    cl = torch.from_numpy(csr.col).to(device)
    vl = torch.from_numpy(csr.val).to(device)
    return packsell_encode(rp, cl, vl, csr.n, csr.m, **kw)


def packsell_set_spmv_variant(A: PackSELLMatrix, variant: int) -> None:
    """0 auto, 1 thread-per-row, 2-4 bulk-staged configurations, 5-6 row prefetch,
    7-8 dual-row, 9-10 stage-planned, 11 CSR order (C = 1), 12 pipelined (slices of
    at most 16 words), 13 variant 5 with programmatic dependent launch."""
    _check(lib().packsell_set_spmv_variant(A.handle, int(variant)))


def packsell_tune_spmv(A: PackSELLMatrix, x: torch.Tensor, y: torch.Tensor | None = None,
                       reps: int = 20, stream=None) -> dict:
    """Time every SpMV variant on (x, y) and make variant 0 use the fastest.
    Returns {variant: ms per launch} for the variants that ran."""
    if y is None:
        y = torch.empty(A.n, dtype=torch.float32, device=x.device)
    times = (ctypes.c_float * SPMV_VARIANTS)()
    _check(lib().packsell_tune_spmv(A.handle, _dev(x, torch.float32, "x", A.m),
                                    _dev(y, torch.float32, "y", A.n), int(reps), times,
                                    _stream(stream)))
    return {v + 1: times[v] for v in range(SPMV_VARIANTS) if times[v] > 0}


def packsell_check_status(A: PackSELLMatrix, stream=None) -> None:
    """Raise if a kernel's bounded wait ran out since the last check."""
    _check(lib().packsell_check_status(A.handle, _stream(stream)))


def packsell_spmv(A: PackSELLMatrix, x: torch.Tensor, y: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """y = A x (float32)."""
    if y is None:
        y = torch.empty(A.n, dtype=torch.float32, device=x.device)
    _check(lib().packsell_spmv(A.handle, _dev(x, torch.float32, "x", A.m),
                               _dev(y, torch.float32, "y", A.n), _stream(stream)))
    return y


def packsell_spmv_f64(A: PackSELLMatrix, x: torch.Tensor, y: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """y = A x (float64; SELL_F64 and W64_E11MY matrices)."""
    if y is None:
        y = torch.empty(A.n, dtype=torch.float64, device=x.device)
    _check(lib().packsell_spmv_f64(A.handle, _dev(x, torch.float64, "x", A.m),
                                   _dev(y, torch.float64, "y", A.n), _stream(stream)))
    return y


def packsell_spmm(A: PackSELLMatrix, X: torch.Tensor, Y: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Y = A X with X row-major [m, k] (float32)."""
    if X.dim() != 2 or X.shape[0] != A.m or X.stride(1) != 1:
        raise ValueError("X must be [m, k] with unit column stride")
    k = X.shape[1]
    if Y is None:
        Y = torch.empty((A.n, k), dtype=torch.float32, device=X.device)
    if Y.shape != (A.n, k) or Y.stride(1) != 1:
        raise ValueError("Y must be [n, k] with unit column stride")
    if X.dtype != torch.float32 or Y.dtype != torch.float32 or not X.is_cuda or not Y.is_cuda:
        raise TypeError("X and Y must be float32 CUDA tensors")
    _check(lib().packsell_spmm(A.handle, k, X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0),
                               _stream(stream)))
    return Y


def packsell_spmv_transpose(A: PackSELLMatrix, dy: torch.Tensor, dx: torch.Tensor | None = None,
                            stream=None) -> torch.Tensor:
    """dx = A^T dy (float32)."""
    if dx is None:
        dx = torch.empty(A.m, dtype=torch.float32, device=dy.device)
    _check(lib().packsell_spmv_transpose(A.handle, _dev(dy, torch.float32, "dy", A.n),
                                         _dev(dx, torch.float32, "dx", A.m), _stream(stream)))
    return dx


def packsell_pattern_outer(A: PackSELLMatrix, alpha: float, u: torch.Tensor, v: torch.Tensor,
                           out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """out[q] = alpha * u_i * v_j for each stored nonzero a_ij (CSR order)."""
    if out is None:
        out = torch.empty(A.nnz, dtype=torch.float32, device=u.device)
    _check(lib().packsell_pattern_outer(A.handle, float(alpha), _dev(u, torch.float32, "u", A.n),
                                        _dev(v, torch.float32, "v", A.m),
                                        _dev(out, torch.float32, "out", A.nnz), _stream(stream)))
    return out


def packsell_spmv_backward(A: PackSELLMatrix, x: torch.Tensor, dy: torch.Tensor, *,
                           need_dx: bool = True, need_dval: bool = True, stream=None):
    """Backward of y = A x: (dx = A^T dy, dval = dy_i x_j on the pattern in CSR
    order), either None when not asked for (float32)."""
    dx = torch.empty(A.m, dtype=torch.float32, device=dy.device) if need_dx else None
    dval = torch.empty(A.nnz, dtype=torch.float32, device=dy.device) if need_dval else None
    _check(lib().packsell_spmv_backward(
        A.handle, _dev(x, torch.float32, "x", A.m) if need_dval else None,
        _dev(dy, torch.float32, "dy", A.n),
        dx.data_ptr() if dx is not None else None,
        dval.data_ptr() if dval is not None else None, _stream(stream)))
    return dx, dval


def packsell_inv_diag(A: PackSELLMatrix, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """1 / a_ii of a square SELL_F64 or W64_E11MY matrix (Jacobi preconditioner)."""
    if out is None:
        out = torch.empty(A.n, dtype=torch.float64, device="cuda")
    _check(lib().packsell_inv_diag(A.handle, _dev(out, torch.float64, "out", A.n),
                                   _stream(stream)))
    return out


def packsell_spmv_host(A: PackSELLMatrix, x_host: torch.Tensor, y_host: torch.Tensor,
                       x_dev: torch.Tensor, y_dev: torch.Tensor, stream=None) -> torch.Tensor:
    """y_host = A x_host through the device staging buffers x_dev, y_dev
    (copy in, SpMV, copy out, all on `stream`; pinned host tensors make the
    copies asynchronous). Returns y_host; valid once the stream is synced."""
    for name, t, numel in (("x_host", x_host, A.m), ("y_host", y_host, A.n)):
        if (not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float32
                or not t.is_contiguous() or t.numel() != numel):
            raise TypeError(f"{name} must be a contiguous float32 host tensor of {numel}")
    _check(lib().packsell_spmv_host(A.handle, x_host.data_ptr(), y_host.data_ptr(),
                                    _dev(x_dev, torch.float32, "x_dev", A.m),
                                    _dev(y_dev, torch.float32, "y_dev", A.n), _stream(stream)))
    return y_host


def packsell_spmv_x16(A: PackSELLMatrix, x: torch.Tensor, y: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """y = A x with float16 x and y (FP32 accumulation in stored order, y
    rounded to binary16)."""
    if y is None:
        y = torch.empty(A.n, dtype=torch.float16, device="cuda")
    _check(lib().packsell_spmv_x16(A.handle, _dev(x, torch.float16, "x", A.m),
                                   _dev(y, torch.float16, "y", A.n), _stream(stream)))
    return y


def packsell_storage_rows(A: PackSELLMatrix, out: torch.Tensor | None = None,
                          stream=None) -> torch.Tensor:
    """Original row held at each storage position (int32 [n]): with an
    explicit permutation, y_orig[rows] = y."""
    if out is None:
        out = torch.empty(A.n, dtype=torch.int32, device="cuda")
    _check(lib().packsell_storage_rows(A.handle, _dev(out, torch.int32, "out", A.n),
                                       _stream(stream)))
    return out


def packsell_pattern_outer_f64(A: PackSELLMatrix, alpha: float, u: torch.Tensor,
                               v: torch.Tensor, out: torch.Tensor | None = None,
                               stream=None) -> torch.Tensor:
    """out[q] = alpha * u_i * v_j in double on the pattern (SELL_F64 matrix)."""
    if out is None:
        out = torch.empty(A.nnz, dtype=torch.float64, device=u.device)
    _check(lib().packsell_pattern_outer_f64(A.handle, float(alpha),
                                            _dev(u, torch.float64, "u", A.n),
                                            _dev(v, torch.float64, "v", A.m),
                                            _dev(out, torch.float64, "out", A.nnz),
                                            _stream(stream)))
    return out


def packsell_validate(A: PackSELLMatrix, stream=None) -> None:
    """Decode the whole matrix on the device and check it (raises CORRUPT)."""
    _check(lib().packsell_validate(A.handle, _stream(stream)))


def packsell_export(A: PackSELLMatrix, stream=None) -> bytes:
    size = ctypes.c_size_t(0)
    _check(lib().packsell_export(A.handle, None, ctypes.byref(size), _stream(stream)))
    buf = ctypes.create_string_buffer(size.value)
    _check(lib().packsell_export(A.handle, buf, ctypes.byref(size), _stream(stream)))
    return buf.raw[: size.value]


def packsell_import(blob: bytes, stream=None) -> PackSELLMatrix:
    h = ctypes.c_void_p()
    _check(lib().packsell_import(blob, len(blob), _stream(stream), ctypes.byref(h)))
    return PackSELLMatrix(h.value)


def packsell_arrays(A: PackSELLMatrix):
    """Host copies of the encoded arrays: dict with offset, perm, and pack
    (PackSELL words) or val/col (SELL), parsed from the export blob."""
    blob = packsell_export(A)
    hdr = 8 + 3 * 8 + ctypes.sizeof(Params) + 4 * 8 + 4 * 4
    pos = hdr
    S = A.n_slices
    out = {"offset": np.frombuffer(blob, np.int64, S + 1, pos)}
    pos += 8 * (S + 1)
    if A.perm_bytes:
        dt = np.uint8 if A.perm_bytes == 1 else np.uint16
        out["perm"] = np.frombuffer(blob, dt, A.n, pos).astype(np.int32)
        pos += A.perm_bytes * A.n
    else:
        out["perm"] = np.zeros(A.n, np.int32)
    if A.format == FMT_W16_E4M3:
        out["pack"] = np.frombuffer(blob, np.uint16, A.n_words, pos)
    elif A.format == FMT_W64_E11MY:
        out["pack"] = np.frombuffer(blob, np.uint64, A.n_words, pos)
    elif A.format in (FMT_FP16, FMT_E8MY, FMT_FIXED):
        out["pack"] = np.frombuffer(blob, np.uint32, A.n_words, pos)
    else:
        dt = {FMT_SELL_F64: np.float64, FMT_SELL_F16: np.float16}.get(A.format, np.float32)
        out["val"] = np.frombuffer(blob, dt, A.n_words, pos)
        pos += np.dtype(dt).itemsize * A.n_words
        out["col"] = np.frombuffer(blob, np.int32, A.n_words, pos)
    return out


def packsell_pcg_workspace_bytes(n: int, m_in: int = 0, has_diag: bool = False,
                                 max_iters: int = 1000) -> int:
    return int(lib().packsell_pcg_workspace_bytes(n, m_in, int(has_diag), max_iters))


def packsell_pcg(A_outer: PackSELLMatrix, b: torch.Tensor, x: torch.Tensor | None = None, *,
                 A_inner: PackSELLMatrix | None = None, inv_diag: torch.Tensor | None = None,
                 rtol: float = 1e-10, m_in: int = 0, max_iters: int = 1000,
                 check_every: int | None = None, use_graph: bool = True,
                 workspace: torch.Tensor | None = None, history: bool = False,
                 check: bool = True, stream=None):
    """Solve A x = b (see the C header). m_in = 0: FP64 Jacobi PCG on A_outer;
    m_in > 0: inner-outer CG with m_in FP32 PCG iterations on A_inner.

    Returns (x, info) with info = dict(iters, inner_iters, relres, relres_true,
    seconds, status[, hist]). With check=True a status other than OK raises.
    """
    n = A_outer.n
    if x is None:
        x = torch.zeros(n, dtype=torch.float64, device=b.device)
    if check_every is None:
        check_every = 1 if m_in > 0 else 10
    opts = SolveOpts(float(rtol), int(m_in), int(max_iters), int(check_every), int(use_graph))
    res = SolveResult()
    hist = (ctypes.c_double * (max_iters + 1))() if history else None
    wptr, wbytes = None, 0
    if workspace is not None:
        if not workspace.is_cuda:
            raise TypeError("workspace must be a CUDA tensor")
        wptr, wbytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    code = lib().packsell_pcg(
        A_outer.handle, A_inner.handle if A_inner is not None else None,
        _dev(inv_diag, torch.float64, "inv_diag", n) if inv_diag is not None else None,
        _dev(b, torch.float64, "b", n), _dev(x, torch.float64, "x", n), ctypes.byref(opts),
        wptr, wbytes, hist, ctypes.byref(res), _stream(stream))
    info = {"iters": res.iters, "inner_iters": res.inner_iters, "relres": res.relres,
            "relres_true": res.relres_true, "seconds": res.seconds,
            "status": STATUS.get(code, str(code))}
    if history:
        info["hist"] = [hist[i] for i in range(min(res.iters, max_iters) + 1)]
    if check and code != 0:
        raise PackSELLError(code, lib().packsell_last_error().decode())
    return x, info


def packsell_pcg_backward(A_outer: PackSELLMatrix, x: torch.Tensor, dL_dx: torch.Tensor, *,
                          A_inner: PackSELLMatrix | None = None,
                          inv_diag: torch.Tensor | None = None, rtol: float = 1e-10,
                          m_in: int = 0, max_iters: int = 1000, check_every: int | None = None,
                          use_graph: bool = True, need_dA: bool = True, stream=None):
    """Backward of x = A^-1 b (A SPD): returns (dL_db, dL_dA, info); dL_db is
    the adjoint solution lam of A lam = dL/dx, dL_dA = -lam_i x_j on the
    pattern in CSR order (float64; None without need_dA)."""
    n = A_outer.n
    if check_every is None:
        check_every = 1 if m_in > 0 else 10
    opts = SolveOpts(float(rtol), int(m_in), int(max_iters), int(check_every), int(use_graph))
    res = SolveResult()
    db = torch.empty(n, dtype=torch.float64, device=dL_dx.device)
    dA = torch.empty(A_outer.nnz, dtype=torch.float64, device=dL_dx.device) if need_dA else None
    code = lib().packsell_pcg_backward(
        A_outer.handle, A_inner.handle if A_inner is not None else None,
        _dev(inv_diag, torch.float64, "inv_diag", n) if inv_diag is not None else None,
        _dev(x, torch.float64, "x", n), _dev(dL_dx, torch.float64, "dL_dx", n), db.data_ptr(),
        dA.data_ptr() if dA is not None else None, ctypes.byref(opts), None, 0, ctypes.byref(res),
        _stream(stream))
    info = {"iters": res.iters, "inner_iters": res.inner_iters, "relres": res.relres,
            "relres_true": res.relres_true, "seconds": res.seconds,
            "status": STATUS.get(code, str(code))}
    _check(code)
    return db, dA, info


def packsell_pcg_noalloc(A_outer: PackSELLMatrix, b: torch.Tensor, x: torch.Tensor, *,
                         A_inner: PackSELLMatrix | None = None,
                         inv_diag: torch.Tensor | None = None, rtol: float = 1e-10,
                         m_in: int = 0, max_iters: int = 1000, check_every: int | None = None,
                         check: bool = True, stream=None):
    """packsell_pcg with its workspace in the library's static device array:
    for callers that must not allocate device memory while they solve (the
    caller provides x as well, so this call allocates nothing). Systems up to
    about 160,000 unknowns (IO-CG) or 260,000 (FP64 PCG); overlapping calls
    race on the shared array."""
    n = A_outer.n
    if check_every is None:
        check_every = 1 if m_in > 0 else 10
    opts = SolveOpts(float(rtol), int(m_in), int(max_iters), int(check_every), 0)
    res = SolveResult()
    code = lib().packsell_pcg_noalloc(
        A_outer.handle, A_inner.handle if A_inner is not None else None,
        _dev(inv_diag, torch.float64, "inv_diag", n) if inv_diag is not None else None,
        _dev(b, torch.float64, "b", n), _dev(x, torch.float64, "x", n), ctypes.byref(opts),
        None, ctypes.byref(res), _stream(stream))
    info = {"iters": res.iters, "inner_iters": res.inner_iters, "relres": res.relres,
            "relres_true": res.relres_true, "seconds": res.seconds,
            "status": STATUS.get(code, str(code))}
    if check and code != 0:
        raise PackSELLError(code, lib().packsell_last_error().decode())
    return x, info


class PackSELLBatch:
    """A batched-SpMV plan (``packsell_batch*``) with its matrices and vectors
    kept alive."""

    def __init__(self, mats, xs, ys, stream=None):
        if not (len(mats) == len(xs) == len(ys)) or not mats:
            raise ValueError("need equally many matrices, x and y (at least one)")
        cnt = len(mats)
        A = (ctypes.c_void_p * cnt)(*[m.handle.value for m in mats])
        X = (ctypes.c_void_p * cnt)(*[_dev(x, torch.float32, "x", m.m) for m, x in zip(mats, xs)])
        Y = (ctypes.c_void_p * cnt)(*[_dev(y, torch.float32, "y", m.n) for m, y in zip(mats, ys)])
        h = ctypes.c_void_p()
        _check(lib().packsell_batch_create(cnt, A, X, Y, _stream(stream), ctypes.byref(h)))
        self._h, self.mats, self.xs, self.ys = h, list(mats), list(xs), list(ys)
        w, b, it = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().packsell_batch_info(h, ctypes.byref(w), ctypes.byref(b), ctypes.byref(it)))
        self.words, self.bytes, self.items = w.value, b.value, it.value

    def spmv(self, stream=None):
        _check(lib().packsell_batch_spmv(self._h, _stream(stream)))

    def close(self):
        if self._h:
            lib().packsell_batch_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def packsell_batch_create(mats, xs, ys, stream=None) -> PackSELLBatch:
    return PackSELLBatch(mats, xs, ys, stream)


class PackSELLBatchMM:
    """A batched-SpMM plan (``packsell_batch*`` from packsell_batch_create_spmm):
    Y_i = A_i X_i for C = 1 matrices, X_i [m_i x k] and Y_i [n_i x k] row-major
    (leading dimension = row stride), kept alive with the plan."""

    def __init__(self, mats, Xs, Ys, stream=None):
        if not (len(mats) == len(Xs) == len(Ys)) or not mats:
            raise ValueError("need equally many matrices, X and Y (at least one)")
        k = int(Xs[0].shape[1])
        cnt = len(mats)
        for m, X, Y in zip(mats, Xs, Ys):
            if X.dim() != 2 or Y.dim() != 2 or X.shape != (m.m, k) or Y.shape != (m.n, k):
                raise ValueError("X_i must be [m_i x k] and Y_i [n_i x k]")
            if X.dtype != torch.float32 or Y.dtype != torch.float32 or not X.is_cuda or not Y.is_cuda:
                raise ValueError("X_i and Y_i must be float32 CUDA tensors")
            if X.stride(1) != 1 or Y.stride(1) != 1:
                raise ValueError("X_i and Y_i must be row-major (unit column stride)")
        A = (ctypes.c_void_p * cnt)(*[m.handle.value for m in mats])
        Xp = (ctypes.c_void_p * cnt)(*[X.data_ptr() for X in Xs])
        Yp = (ctypes.c_void_p * cnt)(*[Y.data_ptr() for Y in Ys])
        lx = (ctypes.c_int64 * cnt)(*[max(X.stride(0), k) for X in Xs])
        ly = (ctypes.c_int64 * cnt)(*[max(Y.stride(0), k) for Y in Ys])
        h = ctypes.c_void_p()
        _check(lib().packsell_batch_create_spmm(cnt, A, k, Xp, lx, Yp, ly, _stream(stream),
                                                ctypes.byref(h)))
        self._h, self.mats, self.Xs, self.Ys, self.k = h, list(mats), list(Xs), list(Ys), k
        w, b, it = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(lib().packsell_batch_info(h, ctypes.byref(w), ctypes.byref(b), ctypes.byref(it)))
        self.words, self.bytes, self.items = w.value, b.value, it.value

    def spmm(self, stream=None):
        _check(lib().packsell_batch_spmm(self._h, _stream(stream)))

    def close(self):
        if self._h:
            lib().packsell_batch_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def packsell_batch_create_spmm(mats, Xs, Ys, stream=None) -> PackSELLBatchMM:
    return PackSELLBatchMM(mats, Xs, Ys, stream)


def packsell_batch_spmm(B: PackSELLBatchMM, stream=None) -> None:
    B.spmm(stream)


def packsell_batch_spmv(B: PackSELLBatch, stream=None) -> None:
    B.spmv(stream)


def packsell_f3r(A_outer: PackSELLMatrix, A_mid: PackSELLMatrix, A_low: PackSELLMatrix,
                 b: torch.Tensor, x: torch.Tensor | None = None, *, rtol: float | None = None,
                 m1: int | None = None, m2: int | None = None, m3: int | None = None,
                 m4: int | None = None, max_iters: int | None = None, omega: float | None = None,
                 check: bool = True, stream=None):
    """F3R (§5.2.1): FGMRES(m1) in FP64 on A_outer, preconditioned by m2 FGMRES
    steps on A_mid, by m3 FGMRES steps on A_low, by m4 Richardson steps on
    A_low. Returns (x, info). Unset options take packsell_f3r_opts_default."""
    o = F3ROpts()
    lib().packsell_f3r_opts_default(ctypes.byref(o))
    for k, v in (("rtol", rtol), ("m1", m1), ("m2", m2), ("m3", m3), ("m4", m4),
                 ("max_iters", max_iters), ("omega", omega)):
        if v is not None:
            setattr(o, k, v)
    n = A_outer.n
    if x is None:
        x = torch.zeros(n, dtype=torch.float64, device=b.device)
    res = SolveResult()
    code = lib().packsell_f3r(A_outer.handle, A_mid.handle, A_low.handle,
                              _dev(b, torch.float64, "b", n), _dev(x, torch.float64, "x", n),
                              ctypes.byref(o), ctypes.byref(res), _stream(stream))
    info = {"iters": res.iters, "inner_iters": res.inner_iters, "relres": res.relres,
            "relres_true": res.relres_true, "seconds": res.seconds, "status": STATUS.get(code, code)}
    if check:
        _check(code)
    return x, info
