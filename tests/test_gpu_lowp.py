"""GPU parity of the bf16 / binary16 forms: all 65536 inputs bit-exact
against the oracle, and the [8192, 28672] N(0, 3) activation tensor."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2001_09258_gb300 as sleefcu
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
NAMES = [f"{fn}_{a}_{t}" for fn in ("erf", "tanh", "exp", "log1p") for a in ("u10", "u35") for t in ("bf16", "f16")]


def run(name, h, offset=0):
    import torch
    n = h.size
    buf = torch.empty(n + offset, dtype=torch.int16, device="cuda")
    buf[offset:].copy_(torch.from_numpy(h.view(np.int16)))
    out = torch.zeros(n + offset, dtype=torch.int16, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = sleefcu.raw(name)(buf.data_ptr() + 2 * offset, out.data_ptr() + 2 * offset, n, st)
    assert rc == 0, sleefcu.last_error()
    torch.cuda.synchronize()
    return out[offset:].cpu().numpy().view(np.uint16)


@pytest.mark.parametrize("name", NAMES)
def test_exhaustive_bitexact(name):
    h = np.arange(65536, dtype=np.uint16)
    got, want = run(name, h), oracle.apply(name, h)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (name, bad.size, hex(h[bad[0]]), hex(got[bad[0]]), hex(want[bad[0]]))


@pytest.mark.parametrize("name", ["erf_u10_bf16", "tanh_u35_f16"])
@pytest.mark.parametrize("n", [1, 7, 9, 1001])
def test_ragged_and_misaligned(name, n):
    h = np.arange(n, dtype=np.uint16) * np.uint16(37)
    assert np.array_equal(run(name, h), oracle.apply(name, h))
    assert np.array_equal(run(name, h, offset=1), oracle.apply(name, h))


@pytest.mark.parametrize("name", ["erf_u10_bf16", "tanh_u10_bf16", "exp_u35_bf16", "log1p_u10_f16"])
def test_activation_tensor_8192x28672(name):
    """The bench's activation workload: N(0, 3) of shape [8192, 28672]."""
    fmt = name.split("_")[-1]
    h = I.activations("c3/act", (8192, 28672), fmt).reshape(-1)
    got, want = run(name, h), oracle.apply(name, h)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("name", NAMES)
def test_table_form_every_input(name):
    """Arrays of 2^24 elements and more take the shared-memory table form:
    every 16-bit pattern, in a scrambled order and with a ragged tail, gives
    the oracle's bits."""
    n = (1 << 24) + 11
    perm = (I.raw(f"tab/{name}", n) & np.uint64(0xFFFF)).astype(np.uint16)
    perm[:65536] = np.arange(65536, dtype=np.uint16)
    table = oracle.apply(name, np.arange(65536, dtype=np.uint16))
    got = run(name, perm)
    bad = np.nonzero(got != table[perm])[0]
    assert bad.size == 0, (name, bad.size, hex(perm[bad[0]]), hex(got[bad[0]]), hex(table[perm[bad[0]]]))
