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


DEFERRED = ["sin_u10_f32", "sin_u35_f32", "cos_u10_f32", "cos_u35_f32", "tan_u10_f32", "tan_u35_f32",
            "sincos_u10_f32", "sincos_u35_f32", "asinh_u10_f32", "asinh_u35_f32", "acosh_u10_f32"]
# (arguments of the main path, arguments of the deferred path) per function
DEFER_SETS = {
    "trig": (lambda n: I.uniform("dq/cw", n, -100, 100), lambda n: I.loguniform("dq/ph", n, 1.1e6, 3.4e38)),
    "ainv": (lambda n: I.loguniform("dq/ab", n, 2.4e18, 3.3e38, signed=False),
             lambda n: I.loguniform("dq/as", n, 1.0, 1e18, signed=False)),
}


def _deferral_cases(fn):
    """Arrays for the deferred queue of the binary32 kernels: no deferred
    lane, every lane deferred, a scattered tenth, whole 2048-element chunks of
    each kind back to back, and deferred lanes on chunk edges; sizes around
    the chunk and the 16-byte vector."""
    kind = "trig" if fn in ("sin", "cos", "tan", "sincos") else "ainv"
    main, rare = DEFER_SETS[kind]
    cw = main(20000).astype(F)
    ph = rare(20000).astype(F)
    pick = (I.raw("dq/pick", 20000) % np.uint64(10)) == 0
    mix = np.where(pick, ph, cw)
    blocks = np.concatenate([cw[:2048], ph[:2048], cw[2048:4096], ph[2048:4096], cw[4096:4100]])
    edges = cw[:6151].copy()
    for i in (0, 3, 2047, 2048, 4095, 4096, 6143, 6150):
        edges[i] = ph[i]
    spec = I.specials_f32()
    return {"none": cw[:8195], "all": ph[:8195], "tenth": mix, "blocks": blocks, "edges": edges,
            "specials": np.concatenate([spec, cw[:61]]), "n1": ph[:1], "n5": mix[:5], "n2049": mix[:2049]}


@pytest.mark.parametrize("name", DEFERRED)
@pytest.mark.parametrize("case", ["none", "all", "tenth", "blocks", "edges", "specials", "n1", "n5", "n2049"])
def test_deferred_queue(name, case):
    x = _deferral_cases(name.split("_")[0])[case]
    got, want = gpu_call(name, x), oracle.apply(name, x)
    if isinstance(want, tuple):
        assert_bitexact(got[0], want[0], x, name + "/sin")
        assert_bitexact(got[1], want[1], x, name + "/cos")
    else:
        assert_bitexact(got, want, x, name)
