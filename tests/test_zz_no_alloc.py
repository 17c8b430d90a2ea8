"""The allocation-free batched launch (sleefcu_batch_launch_static): two
calls in a row on the same arrays give the same bits as a plan's launch,
repeated calls allocate no device memory and return without waiting for the
stream, and oversize or malformed requests are refused with an error.
Collected last so that it also runs after every other GPU test in one
session."""
import ctypes

import numpy as np
import pytest

import paper_2001_09258_gb300 as sleefcu
from test_gpu_batch import F32, F64, LOWP, lengths, make_items

pytestmark = pytest.mark.gpu


def snapshot(items):
    import torch
    torch.cuda.synchronize()
    return [(out.cpu().numpy().copy(), None if out2 is None else out2.cpu().numpy().copy())
            for _, _, _, out, out2 in items]


def poison(items):
    for _, _, _, out, out2 in items:
        out.view(dtype=out.dtype).fill_(float("nan") if out.is_floating_point() else -1)
        if out2 is not None:
            out2.fill_(float("nan"))


def same(a, b):
    return a.view(np.uint8).tobytes() == b.view(np.uint8).tobytes()


def test_static_launch_matches_plan_twice():
    names = (F64 + F32 + LOWP) * 2
    items, _ = make_items(names, lengths(len(names), "za"), "z1")
    plan = sleefcu.Batch(items)
    plan.launch()
    want = snapshot(items)
    plan.close()
    for call in range(2):
        poison(items)
        sleefcu.batch_launch_static(items)
        got = snapshot(items)
        for (name, *_), (g, g2), (w, w2) in zip(items, got, want):
            assert same(g, w), (call, name)
            if w2 is not None:
                assert same(g2, w2), (call, name)


def test_static_launch_limits():
    import torch
    L = sleefcu.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    arr = (sleefcu.BatchItem * 4097)()
    sleefcu.batch_launch_static([])                                     # nothing to do
    assert L.sleefcu_batch_launch_static(arr, 4097, st) == -1           # beyond the fixed scratch
    assert "4096" in sleefcu.last_error()
    assert L.sleefcu_batch_launch_static(None, 3, st) == -1             # null item array
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    bad = sleefcu.BatchItem(999, 0, 10, 0, x.data_ptr(), None, x.data_ptr(), None, 8)
    one = (sleefcu.BatchItem * 1)(bad)
    assert L.sleefcu_batch_launch_static(one, 1, st) == -3              # unsupported function
    nul = sleefcu.BatchItem(0, 0, 10, 0, x.data_ptr(), None, None, None, 8)
    one = (sleefcu.BatchItem * 1)(nul)
    assert L.sleefcu_batch_launch_static(one, 1, st) == -1              # null output with n > 0


def test_static_launch_allocates_nothing():
    """After the first call (which looks up the fixed array's address), more
    calls leave the device's free memory and the caching allocator's
    counters unchanged."""
    import torch
    names = F64[:4] + F32[:4] + LOWP[:2]
    items, _ = make_items(names, lengths(len(names), "zb"), "z2")
    sleefcu.batch_launch_static(items)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = torch.cuda.memory_stats()
    for _ in range(3):
        sleefcu.batch_launch_static(items)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    stats1 = torch.cuda.memory_stats()
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key


def test_static_launch_does_not_wait_for_the_stream():
    """The descriptors travel as kernel arguments: the call returns while an
    earlier busy kernel on the same stream is still running."""
    import torch
    names = F64[:4] + F32[:2]
    items, _ = make_items(names, lengths(len(names), "zc"), "z3")
    sleefcu.batch_launch_static(items)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    torch.cuda._sleep(200_000_000)                 # about 0.1 s of GPU time
    busy = torch.cuda.Event()
    busy.record(st)
    sleefcu.batch_launch_static(items, stream=st)
    assert not busy.query()
    torch.cuda.synchronize()
