"""GPU parity of the FP64 exp/log/pow/asin/acos/atan/atan2 kernels: bit-exact
against the oracle through the C ABI (Section 4, bit-wise consistency)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_bitexact, gpu_call
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
UNARY = [f"{fn}_{a}_f64" for fn in ("exp", "log", "asin", "acos", "atan") for a in ("u10", "u35")]
BINARY = [f"{fn}_{a}_f64" for fn in ("pow", "atan2") for a in ("u10", "u35")]
SPEC = [0.0, -0.0, 1.0, -1.0, 0.5, -0.5, 2.0, -2.0, 3.0, -3.0, math.inf, -math.inf, math.nan,
        1e-310, -1e-310, 1e300, -1e300, 7.5, 2.0 ** 53, 0.999, 1.001, 709.8, -745.5]


def unary_set(fn, n):
    lo, hi = I.DOMAINS_F64[fn]
    return np.concatenate([I.uniform(f"g/{fn}/a", n, lo, hi), I.loguniform(f"g/{fn}/b", n, 5e-324, 1.7e308),
                           I.uniform(f"g/{fn}/c", n, -2, 2), I.SPECIALS_F64, np.array(SPEC)])


def check(name, x, y=None, **kw):
    got = gpu_call(name, x, y, **kw)
    want = oracle.apply(name, x, y)
    assert_bitexact(got, want, x, name)


@pytest.mark.parametrize("name", UNARY)
def test_unary_bitexact(name):
    check(name, unary_set(name.split("_")[0], 40000))


@pytest.mark.parametrize("name", BINARY)
def test_binary_bitexact(name):
    pairs = list(itertools.product(SPEC, SPEC))
    a = np.concatenate([I.uniform("g/b1", 50000, -30, 30), I.loguniform("g/b2", 50000, 1e-300, 1e300),
                        np.array([p[0] for p in pairs])])
    b = np.concatenate([I.uniform("g/b3", 50000, -30, 30), I.uniform("g/b4", 50000, -3, 3),
                        np.array([p[1] for p in pairs])])
    check(name, a, b)


@pytest.mark.parametrize("name", ["exp_u10_f64", "asin_u10_f64", "pow_u10_f64", "atan2_u35_f64"])
@pytest.mark.parametrize("n", [1, 3, 33, 1023, 1025, 4097])
def test_ragged(name, n):
    fn = name.split("_")[0]
    x = I.workload(fn, n, key=f"rg{n}")
    y = I.workload(fn, n, key=f"rg{n}", operand=1) if fn in ("pow", "atan2") else None
    check(name, x, y)


@pytest.mark.parametrize("name", ["log_u10_f64", "acos_u35_f64", "pow_u10_f64"])
def test_misaligned(name):
    fn = name.split("_")[0]
    x = I.workload(fn, 9999, key="mis")
    y = I.workload(fn, 9999, key="mis", operand=1) if fn in ("pow", "atan2") else None
    check(name, x, y, offset=1)


@pytest.mark.parametrize("name", UNARY + BINARY)
def test_full_size_c2_workload(name):
    """2^26 elements of the bench workload (89% main domain, 10% log-uniform
    tail, 1% specials), every output compared."""
    fn = name.split("_")[0]
    x = I.workload(fn, 1 << 26)
    y = I.workload(fn, 1 << 26, operand=1) if fn in ("pow", "atan2") else None
    check(name, x, y)
