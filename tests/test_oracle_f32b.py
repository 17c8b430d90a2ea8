"""Pins of the FP32 functions beyond the first seven: tan, sincos, asin,
acos, atan, atan2, exp2, exp10, expm1, log2, log10, pow, cbrt, sinh, cosh,
asinh, acosh, atanh, erfc, tgamma, lgamma (ULP bounds against __float128),
fmod/remainder (exact, against the C library), and C99 Annex F special
values against the host libm's binary32 functions."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import quadref
from paper_2001_09258_gb300 import inputs as I

needs_quad = pytest.mark.skipif(not quadref.available(), reason="__float128 needs x86-64")
BOUND = {"u10": 1.0, "u35": 3.5}
N = 30000
U, L = I.uniform, I.loguniform
F = np.float32

SETS = {
    "tan": lambda: [U("a", N, -100, 100), L("b", N, 1e5, 3.4e38), U("c", N, -1, 1), U("d", N, 120, 130),
                    L("e", N, 1e-30, 1), U("f", N, 5e5, 1048575)],
    "asin": lambda: [U("a", N, -1, 1), U("b", N, 0.49, 0.51), U("c", N, 0.99, 1), L("d", N, 1e-30, 1e-3)],
    "acos": lambda: [U("a", N, -1, 1), U("b", N, -0.51, -0.49), U("c", N, 0.99, 1), U("d", N, -1, -0.99)],
    "atan": lambda: [U("a", N, -700, 700), U("b", N, -2, 2), L("c", N, 1e-30, 3e38)],
    "exp2": lambda: [U("a", N, -150, 128), U("b", N, -1, 1)],
    "exp10": lambda: [U("a", N, -45, 38.6), U("b", N, -1, 1)],
    "expm1": lambda: [U("a", N, -18, 88.7), U("b", N, -1, 1), L("c", N, 1e-30, 1e-3)],
    "log2": lambda: [L("a", N, 1e-45, 3e38, signed=False), U("b", N, 0.5, 2)],
    "log10": lambda: [L("a", N, 1e-45, 3e38, signed=False), U("b", N, 0.5, 2)],
    "cbrt": lambda: [L("a", N, 1e-45, 3e38), U("b", N, -10, 10)],
    "sinh": lambda: [U("a", N, -89.4, 89.4), U("b", N, -2, 2), L("c", N, 1e-30, 1e-3), U("d", N, 11, 13)],
    "cosh": lambda: [U("a", N, -89.4, 89.4), U("b", N, -2, 2), U("d", N, 11, 13)],
    "asinh": lambda: [L("a", N, 1e-30, 3e38), U("b", N, -2, 2)],
    "acosh": lambda: [L("a", N, 1, 3e38, signed=False), U("b", N, 1, 1.01)],
    "atanh": lambda: [U("a", N, -1, 1), U("b", N, 0.99, 1), L("c", N, 1e-30, 1e-3)],
    "erfc": lambda: [U("a", N, -5, 10.1), U("b", N, -1, 1), U("c", N, 9, 10.1), U("d", N, 0.9, 1.1),
                     U("e", N, 3.8, 4.1)],
    "tgamma": lambda: [U("a", N, -40, 35.9), U("b", N, 0, 3), L("c", N, 1e-30, 1e-3), U("d", N, -5, 0),
                       L("s", N, 1.4e-45, 1e-30)],
    "lgamma": lambda: [U("a", N, 0, 1000), U("b", N, 0, 3), L("c", N, 1e-30, 4e36, signed=False),
                       U("d", N, 0.99, 1.01), U("e", N, 1.99, 2.01)],
}


@needs_quad
@pytest.mark.parametrize("fn", list(SETS))
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_f32_ulp_bound(fn, acc):
    x = np.concatenate([a.astype(F) for a in SETS[fn]()] + [I.specials_f32()])
    if fn == "lgamma":
        x = x[~(x < 0)]
    y = oracle.apply(f"{fn}_{acc}_f32", x)
    err = quadref.ulp_err(fn, x, y)
    i = int(np.argmax(err))
    assert err.max() <= BOUND[acc], (fn, acc, x[i], y[i], err.max())


@needs_quad
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_f32_sincos_and_binary(acc):
    x = np.concatenate([a.astype(F) for a in SETS["tan"]()] + [I.specials_f32()])
    s, c = oracle.apply(f"sincos_{acc}_f32", x)
    assert max(quadref.ulp_err("sin", x, s).max(), quadref.ulp_err("cos", x, c).max()) <= BOUND[acc]
    for fn, a, b in [("atan2", U("q1", N, -100, 100), U("q2", N, -100, 100)),
                     ("atan2", L("q3", N, 1e-40, 3e38), L("q4", N, 1e-40, 3e38)),
                     ("pow", U("p1", N, 0, 30), U("p2", N, -30, 30)),
                     ("pow", L("p3", N, 1e-30, 1e30, signed=False), U("p4", N, -2, 2)),
                     ("pow", U("p5", N, 0.99, 1.01), L("p6", N, 1e2, 1e4))]:
        a, b = a.astype(F), b.astype(F)
        r = oracle.apply(f"{fn}_{acc}_f32", a, b)
        err = quadref.ulp_err(fn, a, r, b)
        assert err.max() <= BOUND[acc], (fn, acc, err.max())


_libm = ctypes.CDLL("libm.so.6")


def _cf(name, nargs=1):
    f = getattr(_libm, name)
    f.restype = ctypes.c_float
    f.argtypes = [ctypes.c_float] * nargs
    return f


def _same(a, b):
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return a == b and math.copysign(1, a) == math.copysign(1, b)


EDGE = np.array([0.0, -0.0, math.inf, -math.inf, math.nan, 1.0, -1.0, 2.0, -2.0, 1e-45, -1e-45, 1.1754944e-38,
                 3.4028235e38, -3.4028235e38, 128.0, -150.0, 88.72, 89.5, -18.0, 38.6, -45.0, 10.1, 0.5,
                 -0.5, 36.0, -42.5], dtype=F)


@pytest.mark.parametrize("fn", ["tan", "asin", "acos", "atan", "exp2", "exp10", "expm1", "log2", "log10",
                                "cbrt", "sinh", "cosh", "asinh", "acosh", "atanh", "erfc", "tgamma", "lgamma"])
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_f32_special_values(fn, acc):
    f = _cf(fn + "f")
    y = oracle.apply(f"{fn}_{acc}_f32", EDGE)
    for xi, yi in zip(EDGE, y):
        want = f(float(xi))
        if math.isnan(want) or math.isinf(want) or want == 0 or math.isnan(xi) or math.isinf(xi):
            assert _same(float(yi), want), (fn, acc, xi, yi, want)
    nans = y[np.isnan(y)].view(np.uint32)
    assert np.all(nans == np.uint32(0x7FC00000))


@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_f32_binary_special_pairs(acc):
    vals = [0.0, -0.0, 1.0, -1.0, 0.5, -2.5, 3.0, math.inf, -math.inf, math.nan, 1e-45, 3.4e38]
    for fn in ("atan2", "pow"):
        f = _cf(fn + "f", 2)
        a = np.array([p for p in vals for _ in vals], dtype=F)
        b = np.array([q for _ in vals for q in vals], dtype=F)
        r = oracle.apply(f"{fn}_{acc}_f32", a, b)
        for ai, bi, ri in zip(a, b, r):
            want = f(float(ai), float(bi))
            if math.isnan(want) or math.isinf(want) or want == 0 or abs(want) == 1 or \
                    math.isinf(ai) or math.isinf(bi) or ai == 0 or bi == 0:
                if fn == "atan2" and not (math.isnan(want) or want == 0):
                    assert abs(float(ri) - want) <= abs(want) * 2.0 ** -23, (fn, ai, bi, ri, want)
                else:
                    assert _same(float(ri), want), (fn, acc, ai, bi, ri, want)


def test_f32_fmod_remainder_exact():
    rem = _cf("remainderf", 2)
    for a, b in [(U("r1", N, -1e5, 1e5), U("r2", N, 1, 100)), (L("r3", N, 1e-40, 3e38), L("r4", N, 1e-40, 3e38)),
                 (L("r5", N, 1e30, 3e38), L("r6", N, 1e-45, 1e-38))]:
        a, b = a.astype(F), b.astype(F)
        got = oracle.apply("fmod_u10_f32", a, b)
        assert np.array_equal(got.view(np.uint32), np.fmod(a, b).view(np.uint32))
        got = oracle.apply("remainder_u10_f32", a, b)
        want = np.array([rem(float(p), float(q)) for p, q in zip(a[:3000], b[:3000])], dtype=F)
        ok = (got[:3000] == want) | (np.isnan(got[:3000]) & np.isnan(want))
        assert ok.all()


def test_f32_identities():
    k = np.arange(-149, 128).astype(F)
    for acc in ("u10", "u35"):
        assert np.array_equal(oracle.apply(f"exp2_{acc}_f32", k), np.ldexp(F(1), k.astype(int)).astype(F))
        assert np.array_equal(oracle.apply(f"log2_{acc}_f32", np.ldexp(F(1), k.astype(int)).astype(F)), k)
        c = np.arange(-100, 101).astype(F)
        assert np.array_equal(oracle.apply(f"cbrt_{acc}_f32", c ** 3), c)
    x = U("s1", N, -20, 20).astype(F)
    for fn in ("tan", "sinh", "asinh", "atan", "cbrt", "erfc"):
        a, b = oracle.apply(f"{fn}_u10_f32", x), oracle.apply(f"{fn}_u10_f32", -x)
        if fn == "erfc":
            assert np.max(np.abs(a + b - 2)) <= 2.0 ** -22
        else:
            assert np.array_equal(a, -b), fn


@needs_quad
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_f32_lgamma_negative_axis(acc):
    """x < 0 in binary32, tiny negative subnormals included (pi x formed
    from x 2^64 there): near the zeros of lgamma the absolute bound
    2^-22 max(1, |lgamma x|) (reading A16), the ULP bound where |lgamma x| >= 1."""
    x = np.concatenate([U("n1", N, -40, 0), U("n2", N, -5, 0), U("n3", N, -2.5, -2.4),
                        -L("n4", N, 1e-30, 1e-3, signed=False), -L("n5", N, 1.4e-45, 1e-30, signed=False),
                        -np.array([1.4e-45, 1e-40, 2.0 ** -126, 2.0 ** -100, 2.0 ** -101])]).astype(F)
    x = x[x != np.rint(x)]
    y = oracle.apply(f"lgamma_{acc}_f32", x)
    ref = quadref.ref("lgamma", x.astype(np.float64))
    assert np.max(np.abs(y - ref) / np.maximum(1, np.abs(ref))) <= 2.0 ** -22
    far = np.abs(ref) >= 1
    err = quadref.ulp_err("lgamma", x[far], y[far])
    assert err.max() <= BOUND[acc], (x[far][np.argmax(err)], err.max())
