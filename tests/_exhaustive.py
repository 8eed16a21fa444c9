"""Loader of ``exhaustive.c`` (the sweeps of the exhaustive quantizer checks).

The C file is compiled once per process into a temporary directory with gcc
and OpenMP. The oracle's quantizer is handed to it as a function pointer, so
the arithmetic being checked stays in the oracle.
"""
import ctypes
import os
import subprocess
import tempfile

import oracle as O

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

ALL = 1 << 32


def lib():
    global _lib
    if _lib is None:
        out = os.path.join(tempfile.mkdtemp(prefix="ps_exh_"), "libexhaustive.so")
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                        "-ffp-contract=off", "-o", out, os.path.join(_HERE, "exhaustive.c")],
                       check=True)
        L = ctypes.CDLL(out)
        P, i64, u64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
        L.sweep_route.argtypes = [P, i32, i32, u64, u64, ctypes.POINTER(u64)]
        L.sweep_route.restype = i64
        L.compare_fields.argtypes = [P, i32, i32, u64, i64, P, ctypes.POINTER(u64)]
        L.compare_fields.restype = i64
        _lib = L
    return _lib


def oracle_field_fn():
    """Address of the oracle's orc_value_field(double, fmt, D, uint32_t *)."""
    return ctypes.cast(O.lib().orc_value_field, ctypes.c_void_p)


def sweep_route(fmt, D, lo=0, hi=ALL):
    first = ctypes.c_uint64()
    bad = lib().sweep_route(oracle_field_fn(), fmt, D, lo, hi, ctypes.byref(first))
    return int(bad), int(first.value)


def compare_fields(fmt, D, lo, fields_ptr, n):
    first = ctypes.c_uint64()
    bad = lib().compare_fields(oracle_field_fn(), fmt, D, lo, n, fields_ptr, ctypes.byref(first))
    return int(bad), int(first.value)
