"""The C-ABI library builds, loads and exports every function the public
header declares (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

from paper_2604_13433_gb300 import build, packsell

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(packsell_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert "packsell_encode" in names and "packsell_spmv" in names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_declared_symbols():
    assert declared_functions() <= set(packsell.SIGNATURES)


def test_struct_layouts():
    # packsell_params: 6 int32 + int64; packsell_info as declared
    assert ctypes.sizeof(packsell.Params) == 32
    assert ctypes.sizeof(packsell.Info) == 144


def test_version_and_defaults_without_gpu():
    lib = packsell.lib()
    assert b"packsell" in lib.packsell_version()
    p = packsell.Params()
    lib.packsell_params_default(ctypes.byref(p))
    assert (p.C, p.sigma, p.D, p.format, p.explicit_perm, p.k_left) == (32, 256, 15, 1, 0, -1)
