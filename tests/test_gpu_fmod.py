"""GPU parity of the FP64 fmod/remainder kernels: bit-exact against the
oracle (the results are exact, so this is also exactness)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_bitexact, gpu_call
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
NAMES = ["fmod_u10_f64", "fmod_u35_f64", "remainder_u10_f64", "remainder_u35_f64"]
SPEC = [0.0, -0.0, 1.0, -1.0, 0.75, 3.0, 2.5, math.inf, -math.inf, math.nan, 5e-324, -5e-324,
        2.2250738585072014e-308, 1.7976931348623157e308, 1e40, 1e-300]


def check(name, x, y, **kw):
    assert_bitexact(gpu_call(name, x, y, **kw), oracle.apply(name, x, y), x, name)


@pytest.mark.parametrize("name", NAMES)
def test_mixed_pairs(name):
    pairs = list(itertools.product(SPEC, SPEC))
    x = np.concatenate([I.loguniform("gf1", 30000, 1e-300, 1.79e308), I.loguniform("gf3", 30000, 5e-324, 1.79e308),
                        I.uniform("gf5", 30000, -1e25, 1e25), np.array([p[0] for p in pairs])])
    y = np.concatenate([I.loguniform("gf2", 30000, 1e-300, 1e300), I.loguniform("gf4", 30000, 5e-324, 1e-300),
                        I.uniform("gf6", 30000, 1, 100), np.array([p[1] for p in pairs])])
    check(name, x, y)


@pytest.mark.parametrize("name", ["fmod_u10_f64", "remainder_u10_f64"])
@pytest.mark.parametrize("n", [1, 5, 1023, 1025, 3001])
def test_ragged(name, n):
    check(name, I.workload("fmod", n, key=f"fr{n}"), I.workload("fmod", n, key=f"fr{n}", operand=1))


def test_misaligned():
    check("fmod_u10_f64", I.workload("fmod", 7777, key="fm"), I.workload("fmod", 7777, key="fm", operand=1),
          offset=1)


@pytest.mark.parametrize("name", ["fmod_u10_f64", "remainder_u10_f64"])
def test_full_size_c2_workload(name):
    fn = name.split("_")[0]
    check(name, I.workload(fn, 1 << 26), I.workload(fn, 1 << 26, operand=1))


def test_large_argument_stress_sample():
    """|x| log-uniform in [1e5, 1.79e308], y log-uniform in [1e-300, 1e300]."""
    x = I.loguniform("c5/fx", 1 << 21, 1e5, 1.79e308)
    y = I.loguniform("c5/fy", 1 << 21, 1e-300, 1e300)
    for name in ("fmod_u10_f64", "remainder_u10_f64"):
        check(name, x, y)


@pytest.mark.parametrize("name", ["fmod_u10_f64", "remainder_u10_f64"])
@pytest.mark.parametrize("r", [1.0, 1e8, 1e16, 1e25])
def test_section71_sweep_workload(name, r):
    """The remainder workload of Section 7.1 (d in [1, 100], dividend in
    [0.95 r d, 1.05 r d]) at several quotient sizes: bit-exact."""
    x, y = I.fmod_sweep(r, 20001)
    assert_bitexact(gpu_call(name, x, y), oracle.apply(name, x, y), x, f"{name}/r={r:g}")
