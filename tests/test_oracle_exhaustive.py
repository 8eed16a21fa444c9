"""Exhaustive pins of the oracle's quantizers (§4.2.2) over every FP32 bit
pattern.

For each of the 2^32 patterns the oracle's field (orc_value_field, the
paper's steps in double precision) is compared with a route of the tests'
own that works on the FP32 bits with integer arithmetic (``exhaustive.c``):
- E8MY: add half a grid step (2^D units in the last place) to the magnitude
  bits and clear the low D + 1 bits; the result overflows once it reaches the
  Inf pattern. This is round half away from zero on the E8MY grid, subnormals
  included, which is the reading the oracle takes below FP32's normal range.
- binary16: shift the FP32 significand to binary16's step for the binade
  (2^-24 below 2^-14) and round the dropped bits to nearest, ties to even.
Non-finite inputs must be refused by both (NONFINITE) and overflow reported
by both (RANGE). Any difference in any pattern fails.
"""
import pytest

import _exhaustive as X
import oracle as O


@pytest.mark.parametrize("D", [1, 7, 11, 15, 22])
def test_e8my_every_pattern_equals_integer_rounding(D):
    bad, first = X.sweep_route(O.FMT_E8MY, D)
    assert bad == 0, f"D = {D}: {bad} patterns differ, first 0x{first:08x}"


def test_f16_every_pattern_equals_integer_rounding():
    bad, first = X.sweep_route(O.FMT_FP16, 15)
    assert bad == 0, f"{bad} patterns differ, first 0x{first:08x}"


def test_routes_catch_a_planted_rounding_mistake():
    """The sweep must notice a quantizer that rounds ties the other way: an
    E8MY with ties to even (bfloat16's rule for D = 15) differs from the
    oracle's ties-away on exactly the tie patterns."""
    import ctypes

    import numpy as np

    FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                          ctypes.POINTER(ctypes.c_uint32))

    def ties_even(v, fmt, D, out):
        b = int(np.array(v, np.float32).view(np.uint32))
        mag, half = b & 0x7FFFFFFF, 1 << D
        keep = mag >> (D + 1)
        rest = mag & ((2 << D) - 1)
        if rest > half or (rest == half and keep & 1):
            keep += 1
        out[0] = (b & 0x80000000) | ((keep << (D + 1)) & 0xFFFFFFFF)
        return 0

    cb = FN(ties_even)
    first = ctypes.c_uint64()
    lo, hi = 0x3F800000, 0x3F800000 + (1 << 18)  # [1, 1 + 2^-5): four ties of D = 15
    bad = X.lib().sweep_route(ctypes.cast(cb, ctypes.c_void_p), O.FMT_E8MY, 15, lo, hi,
                              ctypes.byref(first))
    # the ties are 0x3F808000 + k * 0x10000; with k even the kept part is even,
    # ties-to-even rounds down there and the oracle rounds away (up)
    assert bad == (hi - lo) >> 17
    assert first.value == 0x3F808000
