"""Every binary32 input (all 2^32 bit patterns) through sin, exp and log u10
on the GPU, bit-exact against the oracle on the host cores, in chunks of
2^28 so that host and device memory stay small."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_bitexact

pytestmark = pytest.mark.gpu
CHUNK = 1 << 28


@pytest.mark.parametrize("name", ["sin_u10_f32", "exp_u10_f32", "log_u10_f32"])
def test_all_binary32_inputs(name):
    import ctypes
    import torch
    import paper_2001_09258_gb300 as sleefcu
    f = sleefcu.raw(name)
    st = torch.cuda.current_stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    dx = torch.empty(CHUNK, dtype=torch.float32, device="cuda")
    do = torch.empty_like(dx)
    for c in range((1 << 32) // CHUNK):
        bits = np.arange(c * CHUNK, (c + 1) * CHUNK, dtype=np.uint64).astype(np.uint32)
        x = bits.view(np.float32)
        dx.copy_(torch.from_numpy(x))
        assert f(dx.data_ptr(), do.data_ptr(), CHUNK, sp) == 0
        got = do.cpu().numpy()
        assert_bitexact(got, oracle.apply(name, x), x, f"{name} chunk {c}")
