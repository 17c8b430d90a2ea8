"""The checked build (libsleefcu_checked.so): device-pointer checks before
every launch (host memory, pinned host memory and arrays running past their
allocation are refused with SLEEFCU_EINVAL before anything is enqueued), the
same results as the normal build bit for bit, and a device error word that
stays zero on workloads that reach the Payne-Hanek table gathers with every
kind of argument.  All failures here are host-side returns: no kernel is
launched on a bad pointer."""
import ctypes

import numpy as np
import pytest

import paper_2001_09258_gb300 as sleefcu
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def err_count(L, reset=1):
    c = ctypes.c_ulonglong(0)
    assert L.sleefcu_checked_error_count(ctypes.byref(c), reset) == 0, sleefcu.lib_checked().sleefcu_last_error()
    return c.value


def test_host_pointers_refused():
    import torch
    L = sleefcu.lib_checked()
    h = np.linspace(-3, 3, 1000)
    o = torch.empty(1000, dtype=torch.float64, device="cuda")
    f = L.sleefcu_sin_u10_f64
    assert f(h.ctypes.data, o.data_ptr(), 1000, stream()) == -1
    assert b"not device memory" in L.sleefcu_last_error()
    pinned = torch.from_numpy(h).pin_memory()
    assert f(pinned.data_ptr(), o.data_ptr(), 1000, stream()) == -1
    x = torch.from_numpy(h).cuda()
    assert f(x.data_ptr(), h.ctypes.data, 1000, stream()) == -1          # the output too
    assert L.sleefcu_pow_u10_f64(x.data_ptr(), h.ctypes.data, o.data_ptr(), 1000, stream()) == -1
    m = np.ones(1000, dtype=np.uint8)
    assert L.sleefcu_sin_u10_f64_masked(x.data_ptr(), m.ctypes.data, o.data_ptr(), 1000, stream()) == -1
    assert L.sleefcu_exp_u10_bf16(h.ctypes.data, o.data_ptr(), 1000, stream()) == -1
    assert L.sleefcu_ldexp_f64(x.data_ptr(), h.ctypes.data, o.data_ptr(), 1000, stream()) == -1
    torch.cuda.synchronize()


def test_overrun_refused():
    import torch
    L = sleefcu.lib_checked()
    x = torch.zeros(100, dtype=torch.float64, device="cuda")
    o = torch.empty_like(x)
    n = 1 << 31                          # far beyond the allocation that holds x
    assert L.sleefcu_sin_u10_f64(x.data_ptr(), o.data_ptr(), n, stream()) == -1
    assert b"past the end" in L.sleefcu_last_error()
    assert L.sleefcu_sin_u10_f32(x.data_ptr(), o.data_ptr(), n, stream()) == -1
    torch.cuda.synchronize()


def test_batch_items_checked():
    import torch
    L = sleefcu.lib_checked()
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    h = np.zeros(64)
    bad = sleefcu.BatchItem(sleefcu.FN_IDS["sin"], 0, 10, 0, h.ctypes.data, None, x.data_ptr(), None, 64)
    arr = (sleefcu.BatchItem * 1)(bad)
    plan = ctypes.c_void_p()
    assert L.sleefcu_batch_create(arr, 1, None, ctypes.byref(plan)) == -1
    assert L.sleefcu_batch_launch_static(arr, 1, stream()) == -1
    good = sleefcu.BatchItem(sleefcu.FN_IDS["sin"], 0, 10, 0, x.data_ptr(), None, x.data_ptr(), None, 64)
    arr = (sleefcu.BatchItem * 1)(good)
    assert L.sleefcu_batch_launch_static(arr, 1, stream()) == 0
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["sin_u10_f64", "cos_u35_f64", "tan_u10_f64", "sincos_u10_f64",
                                  "sin_u10_f32", "tan_u35_f32", "sincos_u10_f32", "sin_u10_f64_masked"])
def test_same_bits_and_zero_error_word(name):
    """Payne-Hanek arguments of every binade, specials and small arguments:
    the checked build equals the normal one bit for bit and counts no
    clamped table index."""
    import torch
    L, N = sleefcu.lib_checked(), sleefcu.lib()
    err_count(L)
    f32 = "_f32" in name
    x = np.concatenate([I.uniform("chk/a", 5000, -100, 100), I.loguniform("chk/b", 20000, 1e14, 1.7e308),
                        -I.loguniform("chk/c", 3000, 1e5, 1e14), I.SPECIALS_F64])
    if f32:
        x = x.astype(np.float32)
    dx = torch.from_numpy(x).cuda()
    outs = []
    for lib_ in (N, L):
        o = torch.full_like(dx, 0.25)
        o2 = torch.full_like(dx, 0.25)
        f = getattr(lib_, "sleefcu_" + name)
        if name.endswith("_masked"):
            m = torch.from_numpy((np.arange(x.size) % 3 != 0).astype(np.uint8)).cuda()
            rc = f(dx.data_ptr(), m.data_ptr(), o.data_ptr(), x.size, stream())
        elif name.startswith("sincos"):
            rc = f(dx.data_ptr(), o.data_ptr(), o2.data_ptr(), x.size, stream())
        else:
            rc = f(dx.data_ptr(), o.data_ptr(), x.size, stream())
        assert rc == 0, lib_.sleefcu_last_error()
        torch.cuda.synchronize()
        outs.append((o.cpu().numpy(), o2.cpu().numpy()))
    (a, a2), (b, b2) = outs
    assert a.view(np.uint8).tobytes() == b.view(np.uint8).tobytes()
    assert a2.view(np.uint8).tobytes() == b2.view(np.uint8).tobytes()
    assert err_count(L) == 0
