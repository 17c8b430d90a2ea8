"""The batched mixed launch: every output equals the single-array entry
point's (and so the oracle's) bit for bit, for plain launches, graph replays
and every tuning configuration."""
import math

import numpy as np
import pytest

import oracle
import paper_2001_09258_gb300 as sleefcu
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
F64 = [e for e in sleefcu.entry_points() if e.endswith("_f64")]
F32 = [e for e in sleefcu.entry_points() if e.endswith("_f32")]
LOWP = [e for e in sleefcu.entry_points() if e.endswith(("_bf16", "_f16"))]


def make_items(names, lengths, key):
    import torch
    items, host = [], []
    for k, (name, n) in enumerate(zip(names, lengths)):
        fn, acc, prec = name.split("_")
        if prec in ("f64", "f32"):
            dt = np.float64 if prec == "f64" else np.float32
            x = I.workload(fn, n, key=f"{key}/{k}", dtype=dt)
            y = I.workload(fn, n, key=f"{key}/{k}", operand=1, dtype=dt) if sleefcu.FUNCS[fn] == "b" else None
            tx = torch.from_numpy(x).cuda()
            ty = torch.from_numpy(y).cuda() if y is not None else None
        else:
            x = (I.raw(f"{key}/{k}", n) & np.uint64(0xFFFF)).astype(np.uint16)
            y = None
            tx = torch.from_numpy(x.view(np.int16)).cuda()
            ty = None
        out = torch.empty_like(tx)
        out2 = torch.empty_like(tx) if sleefcu.FUNCS[fn] == "sc" else None
        items.append((name, tx, ty, out, out2))
        host.append((x, y))
    return items, host


def check(items, host):
    import torch
    torch.cuda.synchronize()
    for (name, tx, ty, out, out2), (x, y) in zip(items, host):
        want = oracle.apply(name, x, y)
        got = out.cpu().numpy()
        if out2 is not None:
            assert got.view(np.uint8).tobytes() == want[0].view(np.uint8).tobytes(), name
            assert out2.cpu().numpy().view(np.uint8).tobytes() == want[1].view(np.uint8).tobytes(), name
        else:
            w = want.view(got.dtype) if want.dtype.itemsize == got.dtype.itemsize else want
            assert np.array_equal(got.view(np.uint8), w.view(np.uint8)), name


def lengths(n, key):
    u = (I.raw(key, n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.clip(np.floor(np.exp(u * math.log(2 ** 16))), 1, 2 ** 16).astype(np.int64)


def test_mixed_batch_bitexact():
    names = (F64 + F32 + LOWP) * 3
    items, host = make_items(names, lengths(len(names), "bl"), "b1")
    b = sleefcu.Batch(items)
    b.launch()
    check(items, host)


@pytest.mark.parametrize("cfg", [(128, 512, 1, 1), (256, 4096, 2, 2), (512, 32768, 4, 2), (64, 64, 1, 1),
                                 (96, 960, 1, 2), (128, 1000, 3, 1)])
def test_configs_and_graph(cfg):
    names = F64[::3] + F32[::2] + LOWP[::4]
    items, host = make_items(names, [1, 7, 1000, 4099, 65536, 3] * 10, "b2")
    b = sleefcu.Batch(items[:len(names)])
    b.set_config(*cfg)
    b.launch(graph=True)
    b.launch(graph=True)
    check(items[:len(names)], host[:len(names)])


def test_autotune_and_cache(tmp_path):
    names = F64[:6] + F32[:4]
    items, host = make_items(names, [20000] * len(names), "b3")
    b = sleefcu.Batch(items)
    cache = str(tmp_path / "tune.jsonl")
    b.autotune(cache)
    cfg = b.config()
    b2 = sleefcu.Batch(items)
    b2.autotune(cache)                   # reused from the cache
    assert b2.config() == cfg
    b2.launch()
    check(items, host)
    b3 = sleefcu.Batch(items, tune_file=cache)      # tuned inside sleefcu_batch_create
    assert b3.config() == cfg
    b3.launch()
    check(items, host)
    b4 = sleefcu.Batch(items, tune_file="")         # tuned, no cache file
    b4.launch(graph=True)
    check(items, host)
    for b_ in (b, b2, b3, b4):
        b_.close()


def test_empty_and_bad_items():
    import torch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    b = sleefcu.Batch([("sin_u10_f64", x[:0], None, x[:0], None)])
    b.launch()
    b.launch(graph=True)
    with pytest.raises(sleefcu.SleefcuError):
        sleefcu.Batch([("sin_u10_f16", x, None, x, None)])
