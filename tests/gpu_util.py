"""Helpers of the GPU parity tests: run a C-ABI entry point on device copies
of numpy inputs and compare bit patterns with the oracle."""
import ctypes

import numpy as np

import paper_2001_09258_gb300 as sleefcu


def torch_cuda():
    import torch
    return torch


def gpu_call(name, x, y=None, offset=0):
    """Run sleefcu_<name> through the C ABI.  `offset` shifts every device
    buffer by that many elements (misaligned pointers)."""
    torch = torch_cuda()
    fn = name.split("_")[0]
    kind = sleefcu.FUNCS[fn]
    n = x.size
    dt = torch.float64 if x.dtype == np.float64 else torch.float32

    def dev(a):
        buf = torch.empty(n + offset, dtype=dt, device="cuda")
        if n:
            buf[offset:].copy_(torch.from_numpy(np.ascontiguousarray(a)))
        return buf

    xb = dev(x)
    ob = torch.full((n + offset,), float("nan"), dtype=dt, device="cuda")
    o2 = torch.full((n + offset,), float("nan"), dtype=dt, device="cuda") if kind == "sc" else None
    es = xb.element_size()
    p = lambda t: t.data_ptr() + offset * es
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    f = sleefcu.raw(name)
    if kind == "u":
        rc = f(p(xb), p(ob), n, st)
    elif kind == "b":
        yb = dev(y)
        rc = f(p(xb), p(yb), p(ob), n, st)
    else:
        rc = f(p(xb), p(ob), p(o2), n, st)
    assert rc == 0, (name, rc, sleefcu.last_error())
    torch.cuda.synchronize()
    r = ob[offset:].cpu().numpy()
    if kind == "sc":
        return r, o2[offset:].cpu().numpy()
    return r


def ubits(a):
    a = np.asarray(a)
    return a.view(np.uint64 if a.dtype == np.float64 else np.uint32)


def assert_bitexact(got, want, x, name):
    g, w = ubits(got), ubits(want)
    bad = np.nonzero(g != w)[0]
    if bad.size:
        i = bad[0]
        raise AssertionError(f"{name}: {bad.size} of {g.size} differ; first at {i}: "
                             f"x={x[i]!r} gpu={got[i]!r} ({g[i]:#x}) oracle={want[i]!r} ({w[i]:#x})")
