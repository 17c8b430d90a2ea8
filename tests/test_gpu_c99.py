"""GPU parity of the remaining C99 functions through the C ABI: every entry
point, bit for bit against the oracle, on uniformly random bit patterns
(every exponent, subnormals, infinities, NaN payloads), the functions' own
domains and hand-set cases, with ragged lengths, misaligned buffers (the
scalar path) and a 2^24 + 5 element launch."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2001_09258_gb300 as sleefcu
from gpu_util import torch_cuda
from paper_2001_09258_gb300 import inputs as I

pytestmark = pytest.mark.gpu
NAMES = sleefcu.c99_entry_points()
FT = {"f64": np.float64, "f32": np.float32}
UT = {"f64": np.uint64, "f32": np.uint32}


def kind(name):
    return sleefcu.C99_FUNCS[name.split("_")[0]]


def rand_bits(key, prec, n):
    r = I.raw(key, n)
    if prec == "f64":
        return r.view(np.float64)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)


def domain(name, prec, n, key):
    """values in the function's working range: uniform [-8, 8], log-uniform
    magnitudes over the whole format, integers and half-integers with their
    neighbours"""
    t = FT[prec]
    u = I.raw(key + "/u", n).astype(np.float64) / 2.0 ** 64
    a = (u * 16 - 8).astype(t)
    big = 300 if prec == "f64" else 37
    b = (np.exp((I.raw(key + "/l", n).astype(np.float64) / 2.0 ** 64 * 2 - 1) * big * np.log(10)) *
         np.where(I.raw(key + "/s", n) & np.uint64(1), 1.0, -1.0)).astype(t)
    k = (np.round(u * 2000 - 1000) / 2).astype(t)
    c = np.concatenate([k, np.nextafter(k, t(np.inf)), np.nextafter(k, t(-np.inf))])
    return np.concatenate([a, b, c[: n]])


def hand(prec):
    t = FT[prec]
    fi = np.finfo(t)
    v = [0.0, -0.0, 0.5, -0.5, 1.5, -2.5, 0.25, -0.75, 1.0, 3.0, 2.0 ** 52 + 1, 2.0 ** 23 + 0.5,
         float(fi.max), -float(fi.max), float(fi.tiny), float(fi.smallest_subnormal),
         -float(fi.smallest_subnormal), np.inf, -np.inf, np.nan]
    return np.array(v, dtype=t)


def inputs(name, n, key):
    prec = name.split("_")[-1]
    x = np.concatenate([rand_bits(key + "/x", prec, n), domain(name, prec, n, key + "/d"), hand(prec)])
    y = None
    kd = kind(name)
    if kd == "b":
        y = np.concatenate([rand_bits(key + "/y", prec, n), domain(name, prec, n, key + "/e"), hand(prec)[::-1]])
    elif kd == "bi":
        r = I.raw(key + "/n", x.size)
        y = ((r % np.uint64(4601)).astype(np.int64) - 2300).astype(np.int32)
        y[:8] = [-(1 << 31), (1 << 31) - 1, 0, 1, -1, 1074, -1074, -1075]
    return x, y


def run(name, x, y=None, offset=0):
    torch = torch_cuda()
    kd = kind(name)
    n = x.size
    dt = torch.float64 if x.dtype == np.float64 else torch.float32

    def dev(a, d):
        buf = torch.zeros(n + offset, dtype=d, device="cuda")
        if n:
            buf[offset:].copy_(torch.from_numpy(np.ascontiguousarray(a)))
        return buf

    xb = dev(x, dt)
    od = torch.int32 if kd == "ui" else dt
    ob = torch.full((n + offset,), 7, dtype=od, device="cuda")
    o2 = None
    if kd in ("sc", "si"):
        o2 = torch.full((n + offset,), 7, dtype=torch.int32 if kd == "si" else dt, device="cuda")
    p = lambda t: t.data_ptr() + offset * t.element_size()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    f = sleefcu.raw(name)
    if kd in ("u", "ui"):
        rc = f(p(xb), p(ob), n, st)
    elif kd in ("b", "bi"):
        yb = dev(y, torch.int32 if kd == "bi" else dt)
        rc = f(p(xb), p(yb), p(ob), n, st)
    else:
        rc = f(p(xb), p(ob), p(o2), n, st)
    assert rc == 0, (name, rc, sleefcu.last_error())
    torch.cuda.synchronize()
    r = ob[offset:].cpu().numpy()
    return (r, o2[offset:].cpu().numpy()) if o2 is not None else r


def bits_of(a):
    a = np.asarray(a)
    if a.dtype == np.float64:
        return a.view(np.uint64)
    if a.dtype == np.float32:
        return a.view(np.uint32)
    return a


def check(name, x, y=None, offset=0):
    got = run(name, x, y, offset)
    want = oracle.apply(name, x, y)
    pairs = list(zip(got, want)) if isinstance(got, tuple) else [(got, want)]
    for g, w in pairs:
        gb, wb = bits_of(g), bits_of(w)
        bad = np.nonzero(gb != wb)[0]
        assert bad.size == 0, (f"{name}: {bad.size} of {gb.size} differ; first x={x[bad[0]]!r} "
                               f"y={None if y is None else y[bad[0]]!r} gpu={g[bad[0]]!r} oracle={w[bad[0]]!r}")


@pytest.mark.parametrize("name", NAMES)
def test_c99_matches_oracle(name):
    x, y = inputs(name, (1 << 16) + 3, f"c99gpu/{name}")
    check(name, x, y)


@pytest.mark.parametrize("name", NAMES)
def test_c99_misaligned_and_ragged(name):
    """offset 1: the scalar path; lengths 1 to 9 around the vector width"""
    x, y = inputs(name, 4099, f"c99gpu/mis/{name}")
    check(name, x, y, offset=1)
    for n in (1, 2, 3, 4, 5, 7, 9):
        check(name, x[:n], None if y is None else y[:n])


@pytest.mark.parametrize("name", ["hypot_u05_f64", "sinpi_u05_f64", "cospi_u05_f32", "ldexp_f64",
                                  "frexp_f32", "round_f64", "nextafter_f32", "modf_f64"])
def test_c99_large(name):
    """2^24 + 5 elements: many grid-stride rounds and a ragged tail"""
    x, y = inputs(name, ((1 << 24) + 5) // 2, f"c99gpu/big/{name}")
    check(name, x, y)


def test_c99_python_wrappers():
    torch = torch_cuda()
    x = torch.tensor([0.25, -1.5, 3.0], dtype=torch.float64, device="cuda")
    y = torch.tensor([4.0, 2.0, 4.0], dtype=torch.float64, device="cuda")
    assert sleefcu.hypot(torch.tensor([3.0], dtype=torch.float64, device="cuda"),
                         torch.tensor([4.0], dtype=torch.float64, device="cuda")).item() == 5.0
    assert sleefcu.sinpi(x[:1]).item() == oracle.apply("sinpi_u05_f64", np.array([0.25]))[0]
    assert sleefcu.floor(x).tolist() == [0.0, -2.0, 3.0]
    m, e = sleefcu.frexp(x)
    assert e.dtype == torch.int32 and e.tolist() == [-1, 1, 2]
    assert sleefcu.ldexp(x, e).tolist() == [0.125, -3.0, 12.0]
    assert sleefcu.ilogb(y).tolist() == [2, 1, 2]
