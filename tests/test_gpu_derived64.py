"""GPU parity of the FP64 functions built on the exp/log cores (exp2, exp10,
expm1, log2, log10, log1p, cbrt, sinh, cosh, tanh, asinh, acosh, atanh):
bit-exact against the oracle through the C ABI."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_bitexact, gpu_call
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
FNS = ("exp2", "exp10", "expm1", "log2", "log10", "log1p", "cbrt", "sinh", "cosh", "tanh",
       "asinh", "acosh", "atanh", "erf", "erfc", "tgamma", "lgamma")
NAMES = [f"{fn}_{a}_f64" for fn in FNS for a in ("u10", "u35")]
EDGE = [0.0, -0.0, math.inf, -math.inf, math.nan, 1.0, -1.0, 2.0, -2.0, 5e-324, -5e-324,
        2.2250738585072014e-308, 1.7976931348623157e308, -1.7976931348623157e308, 1024.0, -1075.0,
        -1074.5, 308.25, 308.26, -323.6, -324.0, 709.78, 709.79, 710.47, 710.48, 711.0, -40.0, -39.9,
        19.0, 20.0, 20.5, 22.0, 22.1, 1e-30, -1e-30, 2.0 ** -28, 2.0 ** 500, 0.999999, 1.000001, 8.0, 27.0,
        4.0, -4.0, 6.0, -6.0, 5.99999, 7.99999, -8.0, 27.3, 27.5, 27.50001, -27.5,
        -0.5, -1.5, -2.457, -2.747, -7.0, -7.5, -190.5, -200.5, 0.5, 0.75, 1.25, 1.75, 2.5, 171.62, 171.63,
        2.5e305, 2.6e305, 1e-310, -1e-310]


def check(name, x, **kw):
    assert_bitexact(gpu_call(name, x, **kw), oracle.apply(name, x), x, name)


@pytest.mark.parametrize("name", NAMES)
def test_bitexact_mixed(name):
    fn = name.split("_")[0]
    lo, hi = I.DOMAINS_F64[fn]
    x = np.concatenate([I.uniform(f"gd/{fn}/a", 40000, lo, hi), I.loguniform(f"gd/{fn}/b", 40000, 5e-324, 1.7e308),
                        I.uniform(f"gd/{fn}/c", 40000, -2, 2), I.uniform(f"gd/{fn}/d", 20000, -30, 30),
                        I.SPECIALS_F64, np.array(EDGE)])
    check(name, x)


@pytest.mark.parametrize("name", ["expm1_u10_f64", "cbrt_u10_f64", "sinh_u35_f64", "acosh_u10_f64",
                                  "erfc_u10_f64", "tgamma_u10_f64", "lgamma_u10_f64"])
@pytest.mark.parametrize("n", [1, 3, 33, 1023, 1025, 4097])
def test_ragged(name, n):
    check(name, I.workload(name.split("_")[0], n, key=f"rgd{n}"))


@pytest.mark.parametrize("name", ["log1p_u10_f64", "tanh_u35_f64"])
def test_misaligned(name):
    check(name, I.workload(name.split("_")[0], 9999, key="misd"), offset=1)


@pytest.mark.parametrize("name", NAMES)
def test_full_size_c2_workload(name):
    """2^26 elements of the bench workload, every output compared."""
    x = I.workload(name.split("_")[0], 1 << 26)
    check(name, x)
