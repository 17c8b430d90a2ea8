"""GPU parity of the rest of the FP32 family (tan, sincos, asin, acos, atan,
atan2, exp2, exp10, expm1, log2, log10, pow, cbrt, sinh, cosh, asinh, acosh,
atanh, erfc, tgamma, lgamma, fmod, remainder): bit-exact against the oracle
through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2001_09258_gb300 as sleefcu
from gpu_util import assert_bitexact, gpu_call
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
F = np.float32
FNS = ("tan", "sincos", "asin", "acos", "atan", "atan2", "exp2", "exp10", "expm1", "log2", "log10", "pow",
       "cbrt", "sinh", "cosh", "asinh", "acosh", "atanh", "erfc", "tgamma", "lgamma", "fmod", "remainder")
NAMES = [f"{fn}_{a}_f32" for fn in FNS for a in ("u10", "u35")]


def mixed(fn, n, operand=0):
    lo, hi = I.DOMAINS_F32[fn]
    k = f"g32b/{fn}/{operand}"
    with np.errstate(over="ignore", under="ignore"):
        return np.concatenate([I.uniform(k + "/a", n, lo, hi), I.loguniform(k + "/b", n, 1e-45, 3.4e38),
                               I.uniform(k + "/c", n, -2, 2), I.uniform(k + "/d", n, -130, 130),
                               I.loguniform(k + "/e", n, 1e5, 3.4e38),
                               I.specials_f32().astype(np.float64)]).astype(F)


def check(name, x, y=None, **kw):
    got = gpu_call(name, x, y, **kw)
    want = oracle.apply(name, x, y)
    if isinstance(want, tuple):
        assert_bitexact(got[0], want[0], x, name + "/sin")
        assert_bitexact(got[1], want[1], x, name + "/cos")
    else:
        assert_bitexact(got, want, x, name)


def binary(fn):
    return sleefcu.FUNCS[fn] == "b"


@pytest.mark.parametrize("name", NAMES)
def test_mixed_bitexact(name):
    fn = name.split("_")[0]
    x = mixed(fn, 30000)
    y = mixed(fn, 30000, operand=1)[::-1].copy() if binary(fn) else None
    check(name, x, y)


@pytest.mark.parametrize("name", ["tan_u10_f32", "sincos_u10_f32", "pow_u10_f32", "fmod_u10_f32",
                                  "lgamma_u10_f32"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 1023, 1025, 4099])
def test_ragged(name, n):
    fn = name.split("_")[0]
    x = I.workload(fn, n, key=f"r32b{n}", dtype=F)
    y = I.workload(fn, n, key=f"r32b{n}", operand=1, dtype=F) if binary(fn) else None
    check(name, x, y)


@pytest.mark.parametrize("name", ["sincos_u35_f32", "atan2_u10_f32", "erfc_u10_f32"])
def test_misaligned(name):
    fn = name.split("_")[0]
    x = I.workload(fn, 9999, key="m32b", dtype=F)
    y = I.workload(fn, 9999, key="m32b", operand=1, dtype=F) if binary(fn) else None
    check(name, x, y, offset=1)


@pytest.mark.parametrize("name", NAMES)
def test_c3_workload_2p22(name):
    fn = name.split("_")[0]
    x = I.workload(fn, 1 << 22, dtype=F)
    y = I.workload(fn, 1 << 22, operand=1, dtype=F) if binary(fn) else None
    check(name, x, y)


@pytest.mark.parametrize("name", ["tan_u10_f32", "pow_u10_f32", "tgamma_u10_f32", "remainder_u10_f32"])
def test_c3_full_size_2p28(name):
    """2^28 floats of the FP32 bench workload, every output compared."""
    fn = name.split("_")[0]
    x = I.workload(fn, 1 << 28, dtype=F)
    y = I.workload(fn, 1 << 28, operand=1, dtype=F) if binary(fn) else None
    check(name, x, y)
