"""The GPU value quantiser (packsell_quantize, §4.2.2) against the oracle on
every FP32 bit pattern the format can hold, both signs: binary16 (round to
nearest even, |v| < 65520) and E8MY for D = 1, 7, 11, 15, 22 (round half away
from zero, every finite pattern below the largest one that rounds to Inf,
FP32 subnormals and exponents up to 2^127 included). The oracle computes the
expected fields (orc_value_field, called from the C loop in exhaustive.c);
the patterns just past each format's range must be refused with RANGE."""
import ctypes

import numpy as np
import pytest

import _exhaustive as X
import oracle as O

from _gpu import P, need_gpu, torch

pytestmark = pytest.mark.gpu

CHUNK = 1 << 26


def _limits(fmt, D):
    """Magnitude patterns [0, lim) the format holds."""
    if fmt == O.FMT_FP16:
        return 0x477FF000  # 65520: the midpoint to 65536, rounds up (ties to even)
    return 0x7F800000 - (1 << D)  # adding half a step would reach the Inf pattern


def _sweep(ps, fmt, D):
    lim = _limits(fmt, D)
    fmtname = "fp16" if fmt == O.FMT_FP16 else "e8my"
    field = torch.empty(CHUNK, dtype=torch.int32, device="cuda")
    host = torch.empty(CHUNK, dtype=torch.int32).pin_memory()
    checked = 0
    for sign in (0, 0x80000000):
        for lo in range(0, lim, CHUNK):
            cnt = min(CHUNK, lim - lo)
            first = sign + lo
            # the patterns first .. first + cnt - 1 as float32 values, made on the device
            pat = torch.arange(first, first + cnt, dtype=torch.int64, device="cuda")
            vals = (pat - (1 << 32) * (pat >= 2 ** 31)).to(torch.int32).view(torch.float32)
            ps.packsell_quantize(vals, fmtname, D, out=field[:cnt])
            host[:cnt].copy_(field[:cnt])
            bad, firstbad = X.compare_fields(fmt, D, first, ctypes.c_void_p(host.data_ptr()), cnt)
            assert bad == 0, f"{bad} fields differ from the oracle, first pattern 0x{firstbad:08x}"
            checked += cnt
            del pat, vals
    return checked


@pytest.mark.parametrize("fmt,D", [(O.FMT_FP16, 15), (O.FMT_E8MY, 1), (O.FMT_E8MY, 7),
                                   (O.FMT_E8MY, 11), (O.FMT_E8MY, 15), (O.FMT_E8MY, 22)])
def test_quantizer_every_pattern_matches_oracle(fmt, D):
    need_gpu()
    ps = P()
    n = _sweep(ps, fmt, D)
    assert n == 2 * _limits(fmt, D)


@pytest.mark.parametrize("fmt,D", [(O.FMT_FP16, 15), (O.FMT_E8MY, 1), (O.FMT_E8MY, 22)])
def test_quantizer_refuses_patterns_past_the_range(fmt, D):
    need_gpu()
    ps = P()
    lim = _limits(fmt, D)
    fmtname = "fp16" if fmt == O.FMT_FP16 else "e8my"
    for pat in (lim, lim + 1, 0x7F7FFFFF, 0x80000000 + lim):
        v = torch.tensor([1.0, float(np.array(pat, np.uint32).view(np.float32))], device="cuda")
        with pytest.raises(ps.PackSELLError) as e:
            ps.packsell_quantize(v, fmtname, D)
        assert e.value.code == 4  # RANGE
    for bad in (float("inf"), float("nan")):
        with pytest.raises(ps.PackSELLError) as e:
            ps.packsell_quantize(torch.tensor([bad], device="cuda"), fmtname, D)
        assert e.value.code == 3  # NONFINITE
    # the last pattern inside the range is held
    v = torch.tensor([float(np.array(lim - 1, np.uint32).view(np.float32))], device="cuda")
    f = ps.packsell_quantize(v, fmtname, D).cpu().numpy().view(np.uint32)[0]
    assert f == O.quantize(np.array([v.item()]), fmt, D)[0][0]
