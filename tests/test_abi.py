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
    assert ctypes.sizeof(packsell.Info) == 152


def test_version_and_defaults_without_gpu():
    lib = packsell.lib()
    assert b"packsell" in lib.packsell_version()
    p = packsell.Params()
    lib.packsell_params_default(ctypes.byref(p))
    assert (p.C, p.sigma, p.D, p.format, p.explicit_perm, p.k_left) == (32, 256, 15, 1, 0, -1)


# ---- argument and blob checks that return before any CUDA call ----

_MAGIC = 0x324C4C4553434B50  # "PKCSELL2"


def _blob(n=64, m=64, C=32, sigma=1, D=15, fmt=1, widths=(3, 2), max_width=None,
          offsets=None, magic=_MAGIC, words_extra=0, value_exp=0):
    """A packsell_export blob built by hand: 112-byte header (magic; n, m,
    nnz; params; n_slices, n_words, n_dummies, n_pad; max_width, perm_bytes,
    value_exp, 0), slice offsets, then the words (no perm with sigma = 1)."""
    import struct
    S = (n + C - 1) // C
    if offsets is None:
        offsets = [0]
        for w in widths:
            offsets.append(offsets[-1] + C * w)
    nw = offsets[-1]
    mw = max(widths) if max_width is None else max_width
    hdr = struct.pack("<Q3q6iq4q2i", magic, n, m, nw, C, sigma, D, fmt, 0, 0, 0,
                      S, nw, 0, 0, mw, 0) + struct.pack("<2i", value_exp, 0)
    assert len(hdr) == 112
    return hdr + struct.pack(f"<{S + 1}q", *offsets) + b"\0" * (4 * (nw + words_extra))


def _patch(blob, offset, fmt, value):
    import struct
    return blob[:offset] + struct.pack(fmt, value) + blob[offset + struct.calcsize(fmt):]


def _import(blob):
    lib = packsell.lib()
    out = ctypes.c_void_p()
    code = lib.packsell_import(blob, len(blob), None, ctypes.byref(out))
    return code, lib.packsell_last_error().decode(), out.value


def test_import_rejects_bad_blobs_on_the_host():
    # each blob fails one host-side check, before the library touches the GPU
    cases = [
        (_blob(magic=0), "bad header"),
        (_patch(_blob(), 32, "<i", 0), "bad header"),  # C = 0
        (_blob(D=23), "bad header"),
        (_blob(fmt=7, D=5), "bad header"),  # fixed point needs D in [6, 22]
        (_blob(fmt=5, D=15), "bad header"),  # 16-bit words have D = 7
        (_blob(value_exp=3), "bad header"),  # an exponent only fixed point has
        (_blob(fmt=7, value_exp=5000), "bad header"),
        (_blob(fmt=9), "bad header"),  # no such format
        (_blob(fmt=8, D=32), "bad header"),  # 64-bit words have D in [1, 31]
        (_blob(sigma=300), "bad header"),  # perm_bytes 0 does not match sigma > 1
        (_blob()[:-4], "truncated"),
        (_blob(offsets=[32, 96, 160]), "offsets do not match"),
        (_blob(offsets=[0, 95, 160]), "not C-aligned"),
        (_blob(offsets=[0, 128, 96]), "not C-aligned"),  # decreasing
        (_blob(max_width=2), "widest slice"),
        (_blob(max_width=4), "widest slice"),
    ]
    for blob, why in cases:
        code, msg, out = _import(blob)
        assert code == 9 and why in msg and out is None, (why, code, msg)
    code, msg, _ = _import(b"\0" * 50)  # shorter than the header
    assert code == 1


def test_null_arguments_refused_without_gpu():
    lib = packsell.lib()
    assert lib.packsell_spmv(None, None, None, None) == 1
    assert lib.packsell_spmv_backward(None, None, None, None, None, None) == 1
    assert lib.packsell_set_spmv_variant(None, 5) == 1
    assert lib.packsell_storage_rows(None, None, None) == 1
    assert lib.packsell_spmv_host(None, None, None, None, None, None) == 1
    assert lib.packsell_validate(None, None) == 1
    assert lib.packsell_checks_build() == 0  # the regular build (the checks build is separate)
    assert b"NULL" in lib.packsell_last_error()
