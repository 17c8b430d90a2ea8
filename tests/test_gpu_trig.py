"""GPU parity of the FP64 trigonometric kernels: bit-exact against the oracle
through the C ABI (the paper's bit-consistent property, Section 4)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitexact, gpu_call
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NAMES = [f"{fn}_{a}_f64" for fn in ("sin", "cos", "tan") for a in ("u10", "u35")]
SC = ["sincos_u10_f64", "sincos_u35_f64"]


def c1_input():
    """1,048,576 doubles uniform in [-100, 100] plus the 64 special values."""
    return np.concatenate([I.uniform("c1/sin", 1 << 20, -100.0, 100.0), I.SPECIALS_F64])


def mixed(n, key):
    return np.concatenate([
        I.uniform(key + "/a", n, -15, 15), I.loguniform(key + "/b", n, 15, 1e14),
        I.loguniform(key + "/c", n, 1e14, 1.79e308), I.loguniform(key + "/d", n // 4, 5e-324, 1e-3),
        I.near_pi_half(range(1, 300)), I.SPECIALS_F64])


def check(name, x, **kw):
    got = gpu_call(name, x, **kw)
    want = oracle.apply(name, x)
    if isinstance(got, tuple):
        assert_bitexact(got[0], want[0], x, name + "[sin]")
        assert_bitexact(got[1], want[1], x, name + "[cos]")
    else:
        assert_bitexact(got, want, x, name)


@pytest.mark.parametrize("name", NAMES + SC)
def test_c1_workload_bitexact(name):
    check(name, c1_input())


@pytest.mark.parametrize("name", NAMES + SC)
def test_all_reduction_paths_bitexact(name):
    check(name, mixed(30000, "gpu/mixed"))


@pytest.mark.parametrize("name", ["sin_u10_f64", "cos_u35_f64", "tan_u10_f64", "sincos_u10_f64"])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 255, 257, 1023, 4097, 65537])
def test_ragged_sizes(name, n):
    check(name, I.workload("sin", n, key=f"rag{n}"))


@pytest.mark.parametrize("name", ["sin_u10_f64", "tan_u35_f64", "sincos_u35_f64"])
def test_misaligned_pointers(name):
    check(name, I.workload("sin", 10001, key="mis"), offset=1)


def test_in_place():
    import torch
    import paper_2001_09258_gb300 as sleefcu
    x = I.workload("sin", 100003, key="inplace")
    t = torch.from_numpy(x).cuda()
    sleefcu.call("sin_u10_f64", t, out=t)
    assert_bitexact(t.cpu().numpy(), oracle.apply("sin_u10_f64", x), x, "in-place")


@pytest.mark.parametrize("name", NAMES + SC)
def test_full_size_c2_workload(name):
    """The 2^26-element mixed workload of the bench (89% [-100, 100], 10%
    Payne-Hanek arguments, 1% specials), every output compared."""
    x = I.workload(name.split("_")[0], 1 << 26)
    check(name, x)


def test_large_argument_stress_sample():
    """Payne-Hanek stress: |x| log-uniform in [1e5, 1.79e308], random sign."""
    x = I.loguniform("c5/trig", 1 << 22, 1e5, 1.79e308)
    for name in ("sin_u10_f64", "cos_u10_f64", "tan_u10_f64", "sincos_u10_f64"):
        check(name, x)
