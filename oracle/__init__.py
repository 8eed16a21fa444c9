"""PackSELL oracle: plain, slow, obviously correct CPU reference.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may import this package. It never imports the CUDA
library or its binding, and the library never imports it.

The bit-exact format work (value quantisation, words, encoding, decoding) and
the SpMV definitions live in ``packsell_oracle.c`` (plain C, built by
:func:`build`); this module marshals numpy arrays into it. The solvers
(Jacobi PCG, inner-outer CG, adjoints) are in :mod:`oracle.solvers`.

Citations are to the paper's sections and equations (arXiv 2604.13433):
§3 SELL and its sigma permutation, §4.1 delta encoding (Eq. 2, Eq. 3),
§4.2 word structure and value formats, §4.3 dummies, padding and Eq. 4,
§4.4 PackSELL SpMV, §5.1.2 backward error, §5.2.2 inner-outer CG.

Parity status of each function is stated in its docstring; every function
here is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "packsell_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FMT_FP16 = 1
FMT_E8MY = 2
FMT_FIXED = 7  # fixed point: a V-bit two's-complement integer times 2^s (one s per matrix)
FMT_W64_E11MY = 8  # 64-bit words, binary64 values with Y = 51 - D mantissa bits

OK, ERR_ARG, ERR_UNSORTED, ERR_NONFINITE, ERR_RANGE = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -ffp-contract=off so no FMA is implied)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, u32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        L.orc_f16_bits.argtypes = [ctypes.c_double, P]
        L.orc_f16_value.argtypes = [ctypes.c_uint16]
        L.orc_f16_value.restype = ctypes.c_double
        L.orc_e8my_bits.argtypes = [ctypes.c_double, ctypes.c_int, P]
        L.orc_word_value.argtypes = [u32, u32]
        L.orc_word_value.restype = u32
        L.orc_word_dummy.argtypes = [u32]
        L.orc_word_dummy.restype = u32
        L.orc_unpack.argtypes = [u32, ctypes.c_int, P, P, P]
        L.orc_lower_bandwidth.argtypes = [i64, P, P]
        L.orc_lower_bandwidth.restype = i64
        L.orc_left_offset.argtypes = [i64, i64, i64]
        L.orc_left_offset.restype = i64
        L.orc_check_csr.argtypes = [i64, i64, P, P]
        L.orc_encode_plan.argtypes = [i64, i64, P, P, i32, i32, i32, i64, P, P, P, P]
        L.orc_encode_fill.argtypes = [i64, P, P, P, i32, i32, i32, i64, P, P, P]
        L.orc_decode.argtypes = [i64, i32, i32, i32, i64, P, P, P, P, P, P, P]
        L.orc_e4m3_bits.argtypes = [ctypes.c_double, P]
        L.orc_e4m3_value.argtypes = [ctypes.c_uint8]
        L.orc_e4m3_value.restype = ctypes.c_double
        L.orc_encode_plan_w.argtypes = [i64, i64, P, P, i32, i32, i32, i32, i64, P, P, P, P]
        L.orc_encode16_fill.argtypes = [i64, P, P, P, i32, i32, i64, P, P, P]
        L.orc_decode16.argtypes = [i64, i32, i32, i64, P, P, P, P, P, P, P]
        L.orc_csr_spmv_f64.argtypes = [i64, P, P, P, P, P]
        L.orc_csr_spmv_fma_f32.argtypes = [i64, P, P, P, P, P]
        L.orc_csr_spmv_t_f64.argtypes = [i64, i64, P, P, P, P, P]
        L.orc_csr_spmm_f64.argtypes = [i64, i64, P, P, P, P, i64, P, i64]
        L.orc_packsell_spmv_f64.argtypes = [i64, i32, i32, i32, i32, i64, P, P, P, P, P,
                                            ctypes.c_int, i32]
        L.orc_quantize.argtypes = [i64, P, i32, i32, P, P, P]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_fixed_exponent.argtypes = [ctypes.c_double, ctypes.c_int]
        L.orc_fixed_exponent.restype = ctypes.c_int
        L.orc_fixed_bits.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, P]
        L.orc_fixed_value.argtypes = [u32, ctypes.c_int, ctypes.c_int]
        L.orc_fixed_value.restype = ctypes.c_double
        L.orc_quantize_fixed.argtypes = [i64, P, i32, P, P, P, P]
        u64 = ctypes.c_uint64
        L.orc_e11my_bits.argtypes = [ctypes.c_double, ctypes.c_int, P]
        L.orc_e11my_value.argtypes = [u64]
        L.orc_e11my_value.restype = ctypes.c_double
        L.orc_quantize_e11my.argtypes = [i64, P, i32, P, P, P]
        L.orc_encode64_fill.argtypes = [i64, P, P, P, i32, i32, i32, i64, P, P, P]
        L.orc_decode64.argtypes = [i64, i32, i32, i32, i64, P, P, P, P, P, P, P]
        L.orc_packsell64_spmv_f64.argtypes = [i64, i32, i32, i32, i64, P, P, P, P, P,
                                              ctypes.c_int]
        L.orc_csr_spmv_fma_f64.argtypes = [i64, P, P, P, P, P]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = None
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """Threads of the OpenMP loops (the host baseline's 1-core and all-core runs)."""
    lib().orc_set_threads(int(n))


# --------------------------------------------------------------------------
# value formats (§4.2.2)
# --------------------------------------------------------------------------
def f16_bits(v: float) -> int:
    """binary16 bits of v, round to nearest even (the FP16 cast of §4.2.2)."""
    out = ctypes.c_uint16()
    st = lib().orc_f16_bits(float(v), ctypes.byref(out))
    if st:
        raise OracleError(st, "f16_bits")
    return out.value


def f16_value(h: int) -> float:
    return float(lib().orc_f16_value(int(h)))


def e8my_bits(v: float, D: int) -> int:
    """E8MY bits of v (§4.2.2: round half away on 2^(e-24+D+1), clear D+1 bits)."""
    out = ctypes.c_uint32()
    st = lib().orc_e8my_bits(float(v), int(D), ctypes.byref(out))
    if st:
        raise OracleError(st, "e8my_bits")
    return out.value


def fixed_exponent(M: float, D: int) -> int:
    """The fixed-point exponent s for the largest magnitude M (V = 31 - D)."""
    return int(lib().orc_fixed_exponent(float(M), int(D)))


def fixed_bits(v: float, D: int, s: int) -> int:
    out = ctypes.c_uint32()
    st = lib().orc_fixed_bits(float(v), int(D), int(s), ctypes.byref(out))
    if st:
        raise OracleError(st, "fixed_bits")
    return out.value


def fixed_value(field: int, D: int, s: int) -> float:
    return float(lib().orc_fixed_value(int(field), int(D), int(s)))


def quantize(val: np.ndarray, fmt: int, D: int):
    """Value fields (uint32, the upper V bits of a word) and the values they
    stand for (float64) for an array of real values. Raises on overflow or a
    non-finite input, reporting the first offending index. Fixed point takes
    its exponent from the largest magnitude (see quantize_fixed)."""
    if fmt == FMT_FIXED:
        field, deq, _ = quantize_fixed(val, D)
        return field, deq
    v = _c(val, np.float64)
    field = np.empty(v.size, np.uint32)
    deq = np.empty(v.size, np.float64)
    bad = ctypes.c_int64()
    st = lib().orc_quantize(v.size, _p(v), fmt, D, _p(field), _p(deq), ctypes.byref(bad))
    if st:
        e = OracleError(st, f"quantize (index {bad.value})")
        e.index = bad.value
        raise e
    return field, deq


def quantize_fixed(val: np.ndarray, D: int):
    """Fixed-point fields, values and the matrix exponent s."""
    v = _c(val, np.float64)
    field = np.empty(v.size, np.uint32)
    deq = np.empty(v.size, np.float64)
    s = ctypes.c_int32()
    bad = ctypes.c_int64()
    st = lib().orc_quantize_fixed(v.size, _p(v), D, _p(field), _p(deq), ctypes.byref(s),
                                  ctypes.byref(bad))
    if st:
        e = OracleError(st, f"quantize_fixed (index {bad.value})")
        e.index = bad.value
        raise e
    return field, deq, s.value


# --------------------------------------------------------------------------
# words (§4.2.1)
# --------------------------------------------------------------------------
def word_value(field: int, delta: int) -> int:
    return int(lib().orc_word_value(field, delta))


def word_dummy(delta: int) -> int:
    return int(lib().orc_word_dummy(delta))


def unpack(w: int, D: int):
    """(flag, delta, value field) of a word."""
    f, d, v = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    lib().orc_unpack(w, D, ctypes.byref(f), ctypes.byref(d), ctypes.byref(v))
    return f.value, d.value, v.value


# --------------------------------------------------------------------------
# encoding (§4.1, §4.3) and decoding
# --------------------------------------------------------------------------
@dataclass
class Encoded:
    n: int
    m: int
    C: int
    sigma: int
    D: int
    fmt: int
    k_left: int
    words: np.ndarray  # int64 [n], stored words per original row
    perm: np.ndarray  # int32 [n], storage row -> offset inside its sigma block
    offset: np.ndarray  # int64 [S + 1]
    pack: np.ndarray  # uint32 [N_w]
    field: np.ndarray  # uint32 [nnz], value fields in CSR order
    deq: np.ndarray  # float64 [nnz], quantised values in CSR order
    n_words: int
    n_dummies: int
    n_pad: int
    value_exp: int = 0  # fixed point: the matrix exponent s (value = q * 2^s)

    @property
    def n_slices(self) -> int:
        return self.offset.size - 1


def lower_bandwidth(csr) -> int:
    return int(lib().orc_lower_bandwidth(csr.n, _p(_c(csr.rowptr, np.int64)),
                                         _p(_c(csr.col, np.int32))))


def left_offset(i: int, sigma: int, k_left: int) -> int:
    """Eq. 4."""
    return int(lib().orc_left_offset(i, sigma, k_left))


def encode(csr, C: int = 32, sigma: int = 256, D: int = 15, fmt: int = FMT_FP16,
           k_left: int = -1) -> Encoded:
    """The PackSELL encoding of a CSR matrix (§4.1-§4.3). Parity: bit-exact."""
    L = lib()
    rowptr, col = _c(csr.rowptr, np.int64), _c(csr.col, np.int32)
    vexp = 0
    if fmt == FMT_FIXED:
        field, deq, vexp = quantize_fixed(csr.val, D)
    else:
        field, deq = quantize(csr.val, fmt, D)
    n, m = csr.n, csr.m
    S = (n + C - 1) // C
    words = np.empty(n, np.int64)
    perm = np.empty(n, np.int32)
    offset = np.empty(S + 1, np.int64)
    stats = np.empty(4, np.int64)
    st = L.orc_encode_plan(n, m, _p(rowptr), _p(col), C, sigma, D, k_left, _p(words),
                           _p(perm), _p(offset), _p(stats))
    if st:
        raise OracleError(st, "encode_plan")
    pack = np.empty(int(stats[1]), np.uint32)
    st = L.orc_encode_fill(n, _p(rowptr), _p(col), _p(field), C, sigma, D, int(stats[0]),
                           _p(perm), _p(offset), _p(pack))
    if st:
        raise OracleError(st, "encode_fill")
    return Encoded(n=n, m=m, C=C, sigma=sigma, D=D, fmt=fmt, k_left=int(stats[0]),
                   words=words, perm=perm, offset=offset, pack=pack, field=field, deq=deq,
                   n_words=int(stats[1]), n_dummies=int(stats[2]), n_pad=int(stats[3]),
                   value_exp=vexp)


def e4m3_bits(v: float) -> int:
    """FP8 E4M3 code of v (round to nearest even); OracleError on NaN/inf or
    a value that rounds past 448."""
    out = ctypes.c_uint8()
    st = lib().orc_e4m3_bits(float(v), ctypes.byref(out))
    if st:
        raise OracleError(st, "e4m3_bits")
    return int(out.value)


def e4m3_value(code: int) -> float:
    return float(lib().orc_e4m3_value(code))


def quantize_e4m3(val: np.ndarray):
    """E4M3 codes (uint8) and their values (float64) of every entry."""
    v = np.asarray(val, np.float64).ravel()
    codes = np.array([e4m3_bits(t) for t in v], np.uint8) if v.size else np.zeros(0, np.uint8)
    table = np.array([e4m3_value(c) for c in range(256)], np.float64)
    return codes, table[codes]


@dataclass
class Encoded16:
    """16-bit PackSELL words (W = 16, D = 7, E4M3 values)."""
    n: int
    m: int
    C: int
    sigma: int
    k_left: int
    words: np.ndarray  # int64 [n]
    perm: np.ndarray  # int32 [n]
    offset: np.ndarray  # int64 [S + 1]
    pack: np.ndarray  # uint16 [N_w]
    codes: np.ndarray  # uint8 [nnz], E4M3 codes in CSR order
    deq: np.ndarray  # float64 [nnz]
    n_words: int
    n_dummies: int
    n_pad: int

    @property
    def D(self) -> int:
        return 7


def encode16(csr, C: int = 32, sigma: int = 256, k_left: int = -1) -> Encoded16:
    """PackSELL with 16-bit words: D = 7 delta bits, E4M3 values in the upper
    byte, 15-bit dummy deltas (several dummies for a gap of 2^15 or more)."""
    L = lib()
    rowptr, col = _c(csr.rowptr, np.int64), _c(csr.col, np.int32)
    codes, deq = quantize_e4m3(csr.val)
    n, m = csr.n, csr.m
    S = (n + C - 1) // C
    words = np.empty(n, np.int64)
    perm = np.empty(n, np.int32)
    offset = np.empty(S + 1, np.int64)
    stats = np.empty(4, np.int64)
    st = L.orc_encode_plan_w(n, m, _p(rowptr), _p(col), C, sigma, 7, 16, k_left, _p(words),
                             _p(perm), _p(offset), _p(stats))
    if st:
        raise OracleError(st, "encode_plan_w")
    pack = np.empty(int(stats[1]), np.uint16)
    codes_c = _c(codes, np.uint8)
    st = L.orc_encode16_fill(n, _p(rowptr), _p(col), _p(codes_c), C, sigma, int(stats[0]),
                             _p(perm), _p(offset), _p(pack))
    if st:
        raise OracleError(st, "encode16_fill")
    return Encoded16(n=n, m=m, C=C, sigma=sigma, k_left=int(stats[0]), words=words, perm=perm,
                     offset=offset, pack=pack, codes=codes, deq=deq, n_words=int(stats[1]),
                     n_dummies=int(stats[2]), n_pad=int(stats[3]))


def decode16(enc: Encoded16, rowptr: np.ndarray):
    """(col, codes, counts) of the 16-bit words, as decode()."""
    rowptr = _c(rowptr, np.int64)
    nnz = int(rowptr[-1])
    col = np.full(nnz, -1, np.int32)
    codes = np.zeros(nnz, np.uint8)
    counts = np.zeros(enc.n, np.int64)
    lib().orc_decode16(enc.n, enc.C, enc.sigma, enc.k_left, _p(enc.perm), _p(enc.offset),
                       _p(enc.pack), _p(rowptr), _p(col), _p(codes), _p(counts))
    return col, codes, counts


# --------------------------------------------------------------------------
# 64-bit words (§4.2.1 with W = 64): E11MY values, FP64 products
# --------------------------------------------------------------------------
def e11my_bits(v: float, D: int) -> int:
    """E11MY bits of v: E8MY's rule on binary64 (round half away from zero on
    2^(e-53+D+1), clear the low D + 1 bits); D in [1, 31]."""
    out = ctypes.c_uint64()
    st = lib().orc_e11my_bits(float(v), int(D), ctypes.byref(out))
    if st:
        raise OracleError(st, "e11my_bits")
    return out.value


def e11my_value(bits: int) -> float:
    return float(lib().orc_e11my_value(int(bits)))


def quantize_e11my(val: np.ndarray, D: int):
    """E11MY fields (uint64) and values (float64) of every entry."""
    v = _c(np.asarray(val, np.float64).ravel(), np.float64)
    field = np.empty(v.size, np.uint64)
    deq = np.empty(v.size, np.float64)
    bad = ctypes.c_int64(-1)
    st = lib().orc_quantize_e11my(v.size, _p(v), int(D), _p(field), _p(deq), ctypes.byref(bad))
    if st:
        raise OracleError(st, f"quantize_e11my (index {bad.value})")
    return field, deq


@dataclass
class Encoded64:
    """PackSELL with 64-bit words (W = 64, V = 63 - D, E11MY values)."""
    n: int
    m: int
    C: int
    sigma: int
    D: int
    k_left: int
    words: np.ndarray  # int64 [n]
    perm: np.ndarray  # int32 [n]
    offset: np.ndarray  # int64 [S + 1]
    pack: np.ndarray  # uint64 [N_w]
    field: np.ndarray  # uint64 [nnz], E11MY fields in CSR order
    deq: np.ndarray  # float64 [nnz]
    n_words: int
    n_dummies: int
    n_pad: int

    @property
    def n_slices(self) -> int:
        return self.offset.size - 1


def encode64(csr, C: int = 32, sigma: int = 256, D: int = 11, k_left: int = -1) -> Encoded64:
    """The PackSELL encoding with 64-bit words (§4.1-§4.3 with W = 64).
    Parity: bit-exact."""
    L = lib()
    rowptr, col = _c(csr.rowptr, np.int64), _c(csr.col, np.int32)
    field, deq = quantize_e11my(csr.val, D)
    n, m = csr.n, csr.m
    S = (n + C - 1) // C
    words = np.empty(n, np.int64)
    perm = np.empty(n, np.int32)
    offset = np.empty(S + 1, np.int64)
    stats = np.empty(4, np.int64)
    st = L.orc_encode_plan_w(n, m, _p(rowptr), _p(col), C, sigma, D, 64, k_left, _p(words),
                             _p(perm), _p(offset), _p(stats))
    if st:
        raise OracleError(st, "encode_plan_w")
    pack = np.empty(int(stats[1]), np.uint64)
    st = L.orc_encode64_fill(n, _p(rowptr), _p(col), _p(field), C, sigma, D, int(stats[0]),
                             _p(perm), _p(offset), _p(pack))
    if st:
        raise OracleError(st, "encode64_fill")
    return Encoded64(n=n, m=m, C=C, sigma=sigma, D=D, k_left=int(stats[0]), words=words,
                     perm=perm, offset=offset, pack=pack, field=field, deq=deq,
                     n_words=int(stats[1]), n_dummies=int(stats[2]), n_pad=int(stats[3]))


def decode64(enc: Encoded64, rowptr: np.ndarray):
    """(col, field, counts) of the 64-bit words, as decode()."""
    rowptr = _c(rowptr, np.int64)
    nnz = int(rowptr[-1])
    col = np.full(nnz, -1, np.int32)
    field = np.zeros(nnz, np.uint64)
    counts = np.zeros(enc.n, np.int64)
    lib().orc_decode64(enc.n, enc.C, enc.sigma, enc.D, enc.k_left, _p(enc.perm), _p(enc.offset),
                       _p(enc.pack), _p(rowptr), _p(col), _p(field), _p(counts))
    return col, field, counts


def packsell64_spmv_f64(enc: Encoded64, x: np.ndarray, explicit: bool = False) -> np.ndarray:
    """The §4.4 algorithm over 64-bit words: one double fused multiply-add
    per real word in stored order, from +0."""
    y = np.zeros(enc.n, np.float64)
    lib().orc_packsell64_spmv_f64(enc.n, enc.C, enc.sigma, enc.D, enc.k_left, _p(enc.perm),
                                  _p(enc.offset), _p(enc.pack), _p(_c(x, np.float64)), _p(y),
                                  int(explicit))
    return y


def csr_spmv_fma_f64(csr, val: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A x in double, one fused multiply-add per nonzero in column order
    from +0 (the result of one thread walking one row's words)."""
    y = np.empty(csr.n, np.float64)
    lib().orc_csr_spmv_fma_f64(csr.n, _p(_c(csr.rowptr, np.int64)), _p(_c(csr.col, np.int32)),
                               _p(_c(val, np.float64)), _p(_c(x, np.float64)), _p(y))
    return y


def check_csr(csr) -> int:
    return int(lib().orc_check_csr(csr.n, csr.m, _p(_c(csr.rowptr, np.int64)),
                                   _p(_c(csr.col, np.int32))))


def decode(enc: Encoded, rowptr: np.ndarray):
    """Walk the packed words back into (col, field) in CSR order of ``rowptr``;
    also returns the real-word count per original row."""
    rowptr = _c(rowptr, np.int64)
    nnz = int(rowptr[-1])
    col = np.full(nnz, -1, np.int32)
    field = np.zeros(nnz, np.uint32)
    counts = np.zeros(enc.n, np.int64)
    lib().orc_decode(enc.n, enc.C, enc.sigma, enc.D, enc.k_left, _p(enc.perm), _p(enc.offset),
                     _p(enc.pack), _p(rowptr), _p(col), _p(field), _p(counts))
    return col, field, counts


# --------------------------------------------------------------------------
# SpMV definitions
# --------------------------------------------------------------------------
def csr_spmv_f64(csr, val: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A x in double over CSR (Eq. 1), with values ``val``."""
    y = np.empty(csr.n, np.float64)
    v, xx = _c(val, np.float64), _c(x, np.float64)
    lib().orc_csr_spmv_f64(csr.n, _p(_c(csr.rowptr, np.int64)), _p(_c(csr.col, np.int32)),
                           _p(v), _p(xx), _p(y))
    return y


def csr_spmv_fma_f32(csr, val: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A x in FP32, one fused multiply-add per nonzero in column order,
    starting from +0: the result of one thread walking one row's words."""
    y = np.empty(csr.n, np.float32)
    v, xx = _c(val, np.float32), _c(x, np.float32)
    lib().orc_csr_spmv_fma_f32(csr.n, _p(_c(csr.rowptr, np.int64)), _p(_c(csr.col, np.int32)),
                               _p(v), _p(xx), _p(y))
    return y


def csr_spmv_t_f64(csr, val: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """dx = A^T dy in double."""
    dx = np.empty(csr.m, np.float64)
    lib().orc_csr_spmv_t_f64(csr.n, csr.m, _p(_c(csr.rowptr, np.int64)),
                             _p(_c(csr.col, np.int32)), _p(_c(val, np.float64)),
                             _p(_c(dy, np.float64)), _p(dx))
    return dx


def csr_spmm_f64(csr, val: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y = A X in double, X row-major [m, k]."""
    X = _c(X, np.float64)
    k = X.shape[1]
    Y = np.empty((csr.n, k), np.float64)
    lib().orc_csr_spmm_f64(csr.n, k, _p(_c(csr.rowptr, np.int64)), _p(_c(csr.col, np.int32)),
                           _p(_c(val, np.float64)), _p(X), k, _p(Y), k)
    return Y


def packsell_spmv_f64(enc: Encoded, x: np.ndarray, explicit: bool = False) -> np.ndarray:
    """The §4.4 PackSELL SpMV algorithm over packed words, in double."""
    y = np.zeros(enc.n, np.float64)
    lib().orc_packsell_spmv_f64(enc.n, enc.C, enc.sigma, enc.D, enc.fmt, enc.k_left,
                                _p(enc.perm), _p(enc.offset), _p(enc.pack),
                                _p(_c(x, np.float64)), _p(y), int(explicit), int(enc.value_exp))
    return y


def storage_rows(enc: Encoded) -> np.ndarray:
    """Original row index of every storage row (§3: block base + perm)."""
    i = np.arange(enc.n, dtype=np.int64)
    return (i // enc.sigma) * enc.sigma + enc.perm


def backward_error(y: np.ndarray, csr, val: np.ndarray, x: np.ndarray) -> float:
    """||y - A x||_inf / (||A||_inf ||x||_inf), the metric of §5.1.2."""
    ax = csr_spmv_f64(csr, val, x)
    row_of = np.repeat(np.arange(csr.n), np.diff(csr.rowptr))
    row_abs = np.bincount(row_of, weights=np.abs(np.asarray(val, np.float64)),
                          minlength=csr.n)
    norm_a = float(row_abs.max()) if csr.n else 0.0
    norm_x = float(np.max(np.abs(x))) if x.size else 0.0
    den = norm_a * norm_x
    return float(np.max(np.abs(np.asarray(y, np.float64) - ax)) / den) if den else 0.0


def spmv_error_bound(csr, deq: np.ndarray, x: np.ndarray, words: np.ndarray) -> np.ndarray:
    """Componentwise bound for an FP32 accumulation of row i over w_i words:
    |y_hat - y|_i <= gamma_{w_i} sum_j |q(a_ij) x_j|, gamma_w = w u / (1 - w u),
    u = 2^-24 (standard forward error bound of a recursive dot product)."""
    u = 2.0 ** -24
    absdot = csr_spmv_f64(csr, np.abs(deq), np.abs(np.asarray(x, np.float64)))
    w = np.maximum(np.asarray(words, np.float64), 1.0)
    return (w * u / (1.0 - w * u)) * absdot
