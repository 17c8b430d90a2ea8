"""GPU parity of the FP32 (float-float) kernels: bit-exact against the
oracle through the C ABI."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitexact, gpu_call
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
F = np.float32
NAMES = [f"{fn}_{a}_f32" for fn in ("sin", "cos", "exp", "log", "log1p", "tanh", "erf") for a in ("u10", "u35")]


def mixed(fn, n):
    lo, hi = I.DOMAINS_F32[fn]
    with np.errstate(over="ignore", under="ignore"):
        return np.concatenate([I.uniform(f"g32/{fn}/a", n, lo, hi), I.loguniform(f"g32/{fn}/b", n, 1e-45, 3.4e38),
                               I.uniform(f"g32/{fn}/c", n, -2, 2), I.uniform(f"g32/{fn}/d", n, -130, 130),
                               I.specials_f32().astype(np.float64)]).astype(F)


def check(name, x, **kw):
    assert_bitexact(gpu_call(name, x, **kw), oracle.apply(name, x), x, name)


@pytest.mark.parametrize("name", NAMES)
def test_mixed_bitexact(name):
    check(name, mixed(name.split("_")[0], 50000))


@pytest.mark.parametrize("name", ["sin_u10_f32", "exp_u10_f32", "erf_u10_f32", "log1p_u35_f32"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 1023, 1025, 4099])
def test_ragged(name, n):
    check(name, I.workload(name.split("_")[0], n, key=f"r32{n}", dtype=F))


@pytest.mark.parametrize("name", ["cos_u10_f32", "tanh_u10_f32", "log_u35_f32"])
def test_misaligned(name):
    check(name, I.workload(name.split("_")[0], 9999, key="m32", dtype=F), offset=1)


@pytest.mark.parametrize("name", NAMES)
def test_c3_workload_2p24(name):
    check(name, I.workload(name.split("_")[0], 1 << 24, dtype=F))


@pytest.mark.parametrize("name", ["sin_u10_f32", "erf_u10_f32"])
def test_c3_full_size_2p28(name):
    """2^28 floats of the FP32 bench workload, every output compared."""
    check(name, I.workload(name.split("_")[0], 1 << 28, dtype=F))
