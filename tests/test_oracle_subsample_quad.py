"""The accuracy bound on the benchmark's own inputs (P1 of the accuracy
plan): for every FP64 and FP32 entry point, a 2^20-element sample drawn with
the full-FP64-set recipe (89 % main domain, 10 % log-uniform tail, 1 %
specials; second operands independent) or its binary32 counterpart, the
oracle's result against the __float128 value: <= 1.0 ULP (u10) and <= 3.5
ULP (u35) with the ULP of reading R5, NaN against NaN and correctly signed
infinities counting 0.  lgamma on the negative axis near its zeros carries the
absolute bound 2^-51 max(1, |lgamma x|) instead (reading A16), the 1-ULP bound
where |lgamma x| >= 1.  SUBSAMPLE_N changes the sample size."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import paper_2001_09258_gb300 as sleefcu
from paper_2001_09258_gb300 import inputs as I

quadref = pytest.importorskip("quadref")
pytestmark = pytest.mark.skipif(not quadref.available(), reason="needs __float128")

N = int(os.environ.get("SUBSAMPLE_N", 1 << 20))
NAMES = [e for e in sleefcu.entry_points() if e.endswith(("_f64", "_f32"))]
THREADS = min(16, os.cpu_count() or 1)


def chunked(fn, x, out, y=None):
    """quadref.ulp_err over host threads (the C loop releases the GIL)"""
    k = max(1, x.size // THREADS)
    parts = [slice(i, min(i + k, x.size)) for i in range(0, x.size, k)]
    with cf.ThreadPoolExecutor(THREADS) as ex:
        errs = list(ex.map(lambda s: quadref.ulp_err(fn, x[s], out[s], None if y is None else y[s]), parts))
    return np.concatenate(errs)


@pytest.mark.parametrize("name", NAMES)
def test_bound_on_the_workload_sample(name):
    fn, acc, prec = name.split("_")
    dt = np.float64 if prec == "f64" else np.float32
    key = "c2/rank0" if prec == "f64" else "c3"
    kind = sleefcu.FUNCS[fn]
    x = I.workload(fn, N, key=key, operand=0, dtype=dt)
    y = I.workload(fn, N, key=key, operand=1, dtype=dt) if kind == "b" else None
    out = oracle.apply(name, x, y)
    bound = 1.0 if acc == "u10" else 3.5
    outs = [("sin", out[0]), ("cos", out[1])] if kind == "sc" else [(fn, out)]
    for qfn, o in outs:
        keep = np.ones(x.size, dtype=bool)
        if fn == "lgamma":
            ref = quadref.ref("lgamma", x.astype(np.float64))
            near = (x < 0) & (np.abs(ref) < 1)
            absdev = np.abs(o.astype(np.float64) - ref) / np.maximum(1, np.abs(ref))
            lim = 2.0 ** -51 if prec == "f64" else 2.0 ** -22
            assert np.nanmax(np.where(near, absdev, 0)) <= lim, name
            keep = ~near
        err = chunked(qfn, x[keep], o[keep], None if y is None else y[keep])
        worst = int(np.argmax(err))
        print(f"{name} {qfn}: max {err.max():.4f} ulp over {int(keep.sum())} elements")
        assert err.max() <= bound, (name, qfn, float(x[keep][worst]), float(err.max()))
