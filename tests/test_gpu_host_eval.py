"""Evaluation from host memory (sleefcu_eval_host): chunked, overlapped
copies around the same kernels, so every result equals the oracle's bit for
bit; ragged chunk counts, every signature, pinned and pageable arrays."""
import numpy as np
import pytest

import oracle
import paper_2001_09258_gb300 as sleefcu
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
NAMES = ["sin_u10_f64", "pow_u10_f64", "sincos_u35_f64", "erfc_u10_f64", "fmod_u10_f64", "exp_u10_f32",
         "erf_u35_f32", "tanh_u10_bf16", "log1p_u35_f16"]


def operands(name, n, key):
    fn, acc, prec = name.split("_")
    if prec in ("bf16", "f16"):
        return (I.raw(key, n) & np.uint64(0xFFFF)).astype(np.uint16), None
    dt = np.float64 if prec == "f64" else np.float32
    x = I.workload(fn, n, key=key, dtype=dt)
    y = I.workload(fn, n, key=key, operand=1, dtype=dt) if sleefcu.FUNCS[fn] == "b" else None
    return x, y


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("n,chunk", [(1, 0), (100003, 4096), (1 << 20, 0), (37, 8)])
def test_eval_host_matches_oracle(name, n, chunk):
    x, y = operands(name, n, f"he/{n}")
    out = np.empty_like(x)
    out2 = np.empty_like(x) if sleefcu.FUNCS[name.split("_")[0]] == "sc" else None
    sleefcu.eval_host(name, x, y, out, out2, chunk=chunk)
    want = oracle.apply(name, x, y)
    if out2 is not None:
        assert np.array_equal(out.view(np.uint64), want[0].view(np.uint64))
        assert np.array_equal(out2.view(np.uint64), want[1].view(np.uint64))
    else:
        w = want.view(out.dtype) if want.dtype.itemsize == out.dtype.itemsize else want
        assert out.view(np.uint8).tobytes() == w.view(np.uint8).tobytes()


def test_eval_host_pinned_and_errors():
    import torch
    x = torch.from_numpy(I.workload("exp", 1 << 21, key="hp")).pin_memory()
    o = torch.empty_like(x).pin_memory()
    sleefcu.eval_host("exp_u35_f64", x.numpy(), None, o.numpy())
    assert np.array_equal(o.numpy().view(np.uint64), oracle.apply("exp_u35_f64", x.numpy()).view(np.uint64))
    with pytest.raises(sleefcu.SleefcuError):
        sleefcu.eval_host("pow_u10_f64", x.numpy(), None, o.numpy())          # missing y


def test_eval_host_many_one_pipeline():
    """sleefcu_eval_host_many over items of every signature and precision,
    ragged sizes and chunk counts, an empty item: each result equals the
    oracle's bit for bit."""
    names = NAMES + ["atan2_u35_f64", "sincos_u10_f32"]
    sizes = [100003, 1, 0, 70001, 4096, 33, 250000, 5, 8193, 777, 12345]
    items, wants = [], []
    for i, name in enumerate(names):
        n = sizes[i % len(sizes)]
        x, y = operands(name, n, f"hm/{i}")
        out = np.empty_like(x)
        out2 = np.empty_like(x) if sleefcu.FUNCS[name.split("_")[0]] == "sc" else None
        items.append((name, x, y, out, out2))
        wants.append(oracle.apply(name, x, y) if n else None)
    sleefcu.eval_host_many(items, chunk=8192)
    for (name, x, y, out, out2), want in zip(items, wants):
        if x.size == 0:
            continue
        if out2 is not None:
            assert out.tobytes() == want[0].tobytes() and out2.tobytes() == want[1].tobytes(), name
        else:
            w = want.view(out.dtype) if want.dtype.itemsize == out.dtype.itemsize else want
            assert out.view(np.uint8).tobytes() == w.view(np.uint8).tobytes(), name


def test_eval_host_many_checks_every_item_first():
    x = I.workload("exp", 1000, key="hm/e")
    o = np.full_like(x, 7.0)
    bad = [("exp_u10_f64", x, None, o, None), ("pow_u10_f64", x, None, np.empty_like(x), None)]
    with pytest.raises(sleefcu.SleefcuError):
        sleefcu.eval_host_many(bad)
    assert np.all(o == 7.0)                       # nothing ran
    sleefcu.eval_host_many([])
