"""GPU parity on random bit patterns: every entry point (binary64, binary32
and 16-bit) on arguments whose bits are drawn uniformly, so that every
exponent, both signs, subnormals, infinities and NaNs with arbitrary
payloads occur; the second operand of the binary functions likewise.
Results must equal the oracle's bit for bit (NaN results are the canonical
NaN on both sides)."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitexact, gpu_call, torch_cuda
import paper_2001_09258_gb300 as sleefcu
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
N = 1 << 18
NAMES = [n for n in oracle.names()]


def bits_array(key, prec, n):
    r = I.raw(key, n)
    if prec == "f64":
        return r.view(np.float64)
    if prec == "f32":
        return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return (r & np.uint64(0xFFFF)).astype(np.uint16)


@pytest.mark.parametrize("name", NAMES)
def test_random_bits(name):
    prec = name.split("_")[-1]
    x = bits_array(f"fuzz/{name}/x", prec, N)
    kind = oracle.kind(name)
    y = bits_array(f"fuzz/{name}/y", prec, N) if kind in (oracle.K_B64, oracle.K_B32) else None
    want = oracle.apply(name, x, y)
    if prec in ("bf16", "f16"):
        torch = torch_cuda()
        xd = torch.from_numpy(x.view(np.int16)).cuda()
        od = torch.empty_like(xd)
        import ctypes
        rc = sleefcu.raw(name)(xd.data_ptr(), od.data_ptr(), N, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        got = od.cpu().numpy().view(np.uint16)
        assert np.array_equal(got, want), name
        return
    got = gpu_call(name, x, y)
    if isinstance(want, tuple):
        assert_bitexact(got[0], want[0], x, name + "/sin")
        assert_bitexact(got[1], want[1], x, name + "/cos")
    else:
        assert_bitexact(got, want, x, name)
