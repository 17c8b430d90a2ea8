"""Dense accuracy pin of the 3.5-ULP inverse hyperbolic functions (reading
R28): their logarithm runs in double (binary32) with z corrected once, and
the ranges where that logarithm is small against the rounding of its
argument (asinh and atanh near 0, acosh near 1) are sampled with 2^21
arguments each, in both formats, against the __float128 value: <= 3.5 ULP.
The plain 3.5-ULP log core (z rounded three times) reaches 4.04 ULP on asinh
in [0.02, 0.6] on such a sample, which is why the corrected core is used."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
from paper_2001_09258_gb300 import inputs as I

quadref = pytest.importorskip("quadref")
pytestmark = pytest.mark.skipif(not quadref.available(), reason="needs __float128")
N = 1 << 21
RANGES = {"asinh": [(0.0, 0.6), (0.6, 10.0)], "acosh": [(1.0, 1.2), (1.2, 10.0)],
          "atanh": [(0.0, 0.5), (0.5, 1.0)]}


def maxerr(fn, x, y):
    k = max(1, x.size // 8)
    parts = [slice(i, min(i + k, x.size)) for i in range(0, x.size, k)]
    with cf.ThreadPoolExecutor(min(8, os.cpu_count() or 1)) as ex:
        return max(float(e.max()) for e in ex.map(lambda s: quadref.ulp_err(fn, x[s], y[s]), parts))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("fn", list(RANGES))
def test_dense_u35(fn, prec):
    dt = np.float64 if prec == "f64" else np.float32
    for lo, hi in RANGES[fn]:
        x = I.uniform(f"u35dense/{fn}/{lo}", N, lo, hi).astype(dt)
        y = oracle.apply(f"{fn}_u35_{prec}", x)
        e = maxerr(fn, x, y)
        print(f"{fn}_u35_{prec} [{lo}, {hi}]: max {e:.4f} ulp")
        assert e <= 3.5, (fn, prec, lo, hi, e)
