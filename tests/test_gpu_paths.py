"""GPU parity per reduction path.

Each binary64 entry point runs on arrays whose elements all take one path
class (the classes of the operation-count table: Cody-Waite levels and
Payne-Hanek for the trigonometric functions, the intervals of erf/erfc, the
eight gamma paths, ...), drawn from the function's own workload, so that
every warp of the launch runs that path alone.  Outputs are compared with
the oracle bit for bit.  One launch per (entry point, class), in a fixed
order, which also makes this file the workload for per-path hardware
counters.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitexact, gpu_call
from oracle.counting import gen_opcounts as G
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
N = 1 << 16
NAMES = [n for n in oracle.names() if n.endswith("_f64")]


def path_arrays(name):
    """[(class, x, y)] with N elements each, in the table's class order."""
    fn = name.split("_")[0]
    binary = oracle.kind(name) == oracle.K_B64
    xs = [I.workload(fn, 1 << 18, key="paths")]
    ys = [I.workload(fn, 1 << 18, key="paths", operand=1)] if binary else None
    if fn in I.STRESS_FNS:
        xs.append(I.stress(fn, 1 << 18, key="paths"))
        if binary:
            ys.append(I.stress(fn, 1 << 18, key="paths", operand=1))
    x = np.concatenate(xs)
    y = np.concatenate(ys) if binary else None
    out = []
    for cls, mask in G.classes(fn, x, y).items():
        idx = np.flatnonzero(mask)
        if idx.size == 0:
            continue
        idx = np.resize(idx, N)
        out.append((cls, x[idx], None if y is None else y[idx]))
    return out


@pytest.mark.parametrize("name", NAMES)
def test_path_pure_arrays(name):
    for cls, x, y in path_arrays(name):
        got = gpu_call(name, x, y)
        want = oracle.apply(name, x, y)
        if isinstance(want, tuple):
            assert_bitexact(got[0], want[0], x, f"{name}/{cls}/sin")
            assert_bitexact(got[1], want[1], x, f"{name}/{cls}/cos")
        else:
            assert_bitexact(got, want, x, f"{name}/{cls}")
