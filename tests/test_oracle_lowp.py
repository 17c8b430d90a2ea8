"""Pins of the bf16 / binary16 forms: exhaustive over all 65536 inputs, the
error against __float128 in the 16-bit format's own ULPs, and the
conversions against numpy's binary16 and an independent bf16 rounding."""
import ctypes

import numpy as np
import pytest

import oracle
import quadref
from paper_2001_09258_gb300 import inputs as I

needs_quad = pytest.mark.skipif(not quadref.available(), reason="__float128 needs x86-64")
ALL = np.arange(65536, dtype=np.uint16)
FNS = ["erf", "tanh", "exp", "log1p"]
# the FP32 result is within 1 (u10) or 3.5 (u35) float ULP before the final
# rounding to 8 or 11 bits, so the 16-bit result is within half a 16-bit ULP
# plus that fraction (double rounding)
BOUND = {("u10", "bf16"): 0.5 + 2 ** -15, ("u35", "bf16"): 0.5 + 3.5 * 2 ** -16,
         ("u10", "f16"): 0.5 + 2 ** -12, ("u35", "f16"): 0.5 + 3.5 * 2 ** -13}


@needs_quad
@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("acc", ["u10", "u35"])
@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_exhaustive_ulp(fn, acc, fmt):
    y = oracle.apply(f"{fn}_{acc}_{fmt}", ALL)
    x = I.bits16_to_f64(ALL, fmt)
    out = I.bits16_to_f64(y, fmt)
    err = quadref.ulp_err_fmt(fn, x, out, fmt)
    i = int(np.argmax(err))
    assert err.max() <= BOUND[(acc, fmt)], (fn, acc, fmt, x[i], out[i], err.max())
    nan = np.isnan(out)
    canon = 0x7FC0 if fmt == "bf16" else 0x7E00
    assert np.all(y[nan] == canon)


def test_conversions():
    L = oracle.lib()
    L.oracle_f32_to_bf16.restype = ctypes.c_uint16
    L.oracle_f32_to_bf16.argtypes = [ctypes.c_float]
    L.oracle_f32_to_f16.restype = ctypes.c_uint16
    L.oracle_f32_to_f16.argtypes = [ctypes.c_float]
    with np.errstate(over="ignore"):
        r = np.concatenate([I.loguniform("cv1", 20000, 1e-45, 3.4e38), I.uniform("cv2", 20000, -7e4, 7e4),
                            I.loguniform("cv3", 20000, 1e-9, 1e-4)]).astype(np.float32)
    mine16 = np.array([L.oracle_f32_to_f16(float(v)) for v in r], dtype=np.uint16)
    with np.errstate(over="ignore"):
        assert np.array_equal(mine16, r.astype(np.float16).view(np.uint16))
    mineb = np.array([L.oracle_f32_to_bf16(float(v)) for v in r], dtype=np.uint16)
    assert np.array_equal(mineb, I.to_bf16_bits(r))
