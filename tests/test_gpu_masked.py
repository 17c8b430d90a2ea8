"""GPU parity of the masked FP64 entry points (the paper's whole-function
opmask): the selected elements equal the oracle bit for bit, the others keep
what the output held before the call."""
import numpy as np
import pytest

import oracle
import paper_2001_09258_gb300 as sleefcu
from gpu_util import torch_cuda
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
SENTINEL = 1234.5


def operands(name, n, key):
    fn = name.split("_")[0]
    x = np.concatenate([I.workload(fn, n, key=key), I.SPECIALS_F64])
    y = None
    if sleefcu.FUNCS[fn] == "b":
        y = np.concatenate([I.workload(fn, n, key=key, operand=1), I.SPECIALS_F64[::-1]])
    return x, y


def masks(n):
    r = I.raw("mask/r", n)
    alt = np.zeros(n, dtype=np.uint8)
    alt[::2] = 1
    ends = np.zeros(n, dtype=np.uint8)
    ends[[0, n - 1]] = 1
    return {"tenth": ((r % np.uint64(10)) == 0).astype(np.uint8),
            "third": ((r % np.uint64(3)) == 0).astype(np.uint8) * 7,       # any non-zero byte selects
            "none": np.zeros(n, dtype=np.uint8), "all": np.ones(n, dtype=np.uint8), "alternate": alt, "ends": ends}


def run(name, x, y, mask):
    torch = torch_cuda()
    fn = name.split("_")[0]
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda() if y is not None else None
    md = torch.from_numpy(mask).cuda()
    out = torch.full_like(xd, SENTINEL)
    out2 = torch.full_like(xd, SENTINEL) if sleefcu.FUNCS[fn] == "sc" else None
    sleefcu.call_masked(name, xd, md, y=yd, out=out, out2=out2)
    torch.cuda.synchronize()
    return out.cpu().numpy(), None if out2 is None else out2.cpu().numpy()


def check(name, x, y, mask):
    got, got2 = run(name, x, y, mask)
    want = oracle.apply(name, x, y)
    sel = mask != 0
    for g, w in ([(got, want[0]), (got2, want[1])] if got2 is not None else [(got, want)]):
        assert np.array_equal(g[sel].view(np.uint64), w[sel].view(np.uint64)), name
        assert np.all(g[~sel] == SENTINEL), name


@pytest.mark.parametrize("name", sleefcu.masked_entry_points())
def test_masked_matches_oracle(name):
    x, y = operands(name, 5000, "msk")
    for kind, m in masks(x.size).items():
        check(name, x, y, m)


@pytest.mark.parametrize("name", ["sin_u10_f64", "tgamma_u10_f64", "pow_u10_f64", "sincos_u35_f64", "exp_u10_f64"])
def test_masked_large_sparse(name):
    """2^20 + 3 elements, a tenth selected, over several grid waves."""
    x, y = operands(name, (1 << 20) + 3 - I.SPECIALS_F64.size, "msk2")
    check(name, x, y, masks(x.size)["tenth"])
