"""Pins of the FP64 functions built on the exp/log cores (exp2, exp10,
expm1, log2, log10, log1p, cbrt, sinh, cosh, tanh, asinh, acosh, atanh):
ULP bounds against __float128, C99 Annex F special values against the host
C library, and exact identities."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import quadref
from paper_2001_09258_gb300 import inputs as I

needs_quad = pytest.mark.skipif(not quadref.available(), reason="__float128 needs x86-64")
BOUND = {"u10": 1.0, "u35": 3.5}
N = 40000
U, L = I.uniform, I.loguniform

SETS = {
    "exp2": lambda: [U("x1", N, -1075, 1024), U("x2", N, -1, 1), L("x3", N, 1e-300, 1e-3),
                     U("x4", N, -1075, -1020), U("x5", N, 1020, 1024)],
    "exp10": lambda: [U("t1", N, -324, 308.3), U("t2", N, -1, 1), L("t3", N, 1e-300, 1e-3),
                      U("t4", N, -324, -307), U("t5", N, 300, 308.3)],
    "expm1": lambda: [U("m1", N, -40, 709.8), U("m2", N, -1, 1), L("m3", N, 1e-300, 1e-3),
                      U("m4", N, -0.7, 0.7), U("m5", N, 700, 709.8), U("m6", N, -45, -30)],
    "log2": lambda: [L("l1", N, 5e-324, 1.7e308, signed=False), U("l2", N, 0.5, 2), U("l3", N, 0.999, 1.001)],
    "log10": lambda: [L("g1", N, 5e-324, 1.7e308, signed=False), U("g2", N, 0.5, 2), U("g3", N, 0.999, 1.001)],
    "log1p": lambda: [L("p1", N, 1e-300, 1e300, signed=False), U("p2", N, -1, 1), L("p3", N, 1e-300, 1e-3),
                      U("p4", N, -1, -0.99), U("p5", N, -0.3, -0.2), U("p6", N, 0.4, 0.6)],
    "cbrt": lambda: [L("c1", N, 5e-324, 1.7e308), U("c2", N, -10, 10), U("c3", N, 0.99, 8.01)],
    "sinh": lambda: [U("s1", N, -710.4, 710.4), U("s2", N, -1, 1), L("s3", N, 1e-300, 1e-3),
                     U("s4", N, 15, 30), U("s5", N, 700, 710.47)],
    "cosh": lambda: [U("h1", N, -710.4, 710.4), U("h2", N, -1, 1), L("h3", N, 1e-300, 1e-3),
                     U("h4", N, 15, 30), U("h5", N, 700, 710.47)],
    "tanh": lambda: [U("n1", N, -20, 20), U("n2", N, -1, 1), L("n3", N, 1e-300, 1e-3), U("n4", N, 17, 22)],
    "asinh": lambda: [L("a1", N, 1e-300, 1.7e308), U("a2", N, -2, 2), L("a3", N, 1e-300, 1e-3)],
    "acosh": lambda: [L("b1", N, 1, 1.7e308, signed=False), U("b2", N, 1, 2), U("b3", N, 1, 1 + 1e-6)],
    "atanh": lambda: [U("d1", N, -1, 1), L("d2", N, 1e-300, 1e-3), U("d3", N, 0.99, 1), U("d4", N, 0.4, 0.6)],
}


@needs_quad
@pytest.mark.parametrize("fn", list(SETS))
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_ulp_bound(fn, acc):
    x = np.concatenate(SETS[fn]() + [I.SPECIALS_F64])
    y = oracle.apply(f"{fn}_{acc}_f64", x)
    err = quadref.ulp_err(fn, x, y)
    i = int(np.argmax(err))
    assert err.max() <= BOUND[acc], (fn, acc, x[i], y[i], err.max())


_libm = ctypes.CDLL("libm.so.6")
for _f in SETS:
    getattr(_libm, _f).restype = ctypes.c_double
    getattr(_libm, _f).argtypes = [ctypes.c_double]


def _same(a, b):
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    return a == b and math.copysign(1, a) == math.copysign(1, b)


EDGE = [0.0, -0.0, math.inf, -math.inf, math.nan, 1.0, -1.0, 2.0, -2.0, 5e-324, -5e-324,
        2.2250738585072014e-308, 1.7976931348623157e308, -1.7976931348623157e308,
        1024.0, -1075.0, -1074.5, 308.25, 308.26, -323.6, -324.0, 709.78, 709.79, 710.47, 710.48,
        711.0, -40.0, -39.9, 19.0, 20.0, 20.5, 22.0, 22.1, 1e-30, -1e-30]


@pytest.mark.parametrize("fn", list(SETS))
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_special_values(fn, acc):
    x = np.array(EDGE)
    y = oracle.apply(f"{fn}_{acc}_f64", x)
    for xi, yi in zip(x, y):
        want = getattr(_libm, fn)(float(xi))
        if math.isnan(want) or math.isinf(want) or want == 0 or abs(want) == 1 or math.isnan(xi):
            assert _same(yi, want), (fn, acc, xi, yi, want)
        assert math.isnan(yi) == math.isnan(want), (fn, acc, xi, yi, want)
    nans = y[np.isnan(y)].view(np.uint64)
    assert np.all(nans == np.uint64(0x7FF8000000000000))


@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_exact_identities(acc):
    k = np.arange(-1074, 1024, dtype=np.float64)
    assert np.array_equal(oracle.apply(f"exp2_{acc}_f64", k), np.ldexp(1.0, k.astype(int)))
    assert np.array_equal(oracle.apply(f"log2_{acc}_f64", np.ldexp(1.0, k.astype(int))), k)
    p = np.arange(0, 23, dtype=np.float64)
    if acc == "u10":                       # the 3.5-ULP form only stays within its bound
        assert np.array_equal(oracle.apply(f"exp10_{acc}_f64", p), 10.0 ** p)
    assert np.array_equal(oracle.apply(f"log10_{acc}_f64", 10.0 ** p), p)
    c = np.arange(-200, 201, dtype=np.float64)
    assert np.array_equal(oracle.apply(f"cbrt_{acc}_f64", c ** 3), c)
    assert np.array_equal(oracle.apply(f"cbrt_{acc}_f64", np.ldexp(1.0, 3 * np.arange(-358, 341))),
                          np.ldexp(1.0, np.arange(-358, 341)))


def test_symmetries():
    x = np.concatenate([U("y1", 20000, 0, 30), L("y2", 20000, 1e-300, 1e300, signed=False)])
    for fn in ("sinh", "tanh", "asinh", "atanh", "cbrt"):
        for acc in ("u10", "u35"):
            a = oracle.apply(f"{fn}_{acc}_f64", x)
            b = oracle.apply(f"{fn}_{acc}_f64", -x)
            ok = np.isnan(a) & np.isnan(b) | (a == -b)
            assert ok.all(), fn
    for acc in ("u10", "u35"):
        assert np.array_equal(oracle.apply(f"cosh_{acc}_f64", x), oracle.apply(f"cosh_{acc}_f64", -x))


@needs_quad
def test_composite_identities():
    """log1p(expm1 x) ~ x and exp2(log2 x) ~ x within the combined bounds;
    cosh^2 - sinh^2 = 1 on |x| <= 1 to a few ulp."""
    x = U("z1", 50000, -1, 30)           # below -1, log1p near -1 amplifies by e^|x|
    r = oracle.apply("log1p_u10_f64", oracle.apply("expm1_u10_f64", x))
    assert np.max(np.abs(r - x) / np.maximum(np.abs(x), 1e-300)) < 2.0 ** -49
    x = L("z2", 50000, 1e-300, 1e300, signed=False)
    r = oracle.apply("exp2_u10_f64", oracle.apply("log2_u10_f64", x))
    assert np.max(np.abs(r - x) / x) < 2.0 ** -41      # |log2 x| up to 997 amplifies 1 ulp
    x = U("z3", 50000, -1, 1)
    c, s = oracle.apply("cosh_u10_f64", x), oracle.apply("sinh_u10_f64", x)
    assert np.max(np.abs((c - s) * (c + s) - 1)) < 2.0 ** -50


ERF_SETS = {
    "erf": lambda: [U("e1", N, -6, 6), U("e2", N, -1, 1), L("e3", N, 1e-300, 1e-3), U("e4", N, 0.9, 1.1),
                    U("e5", N, 1.9, 2.1), U("e6", N, 3.9, 4.1), U("e7", N, 5.5, 6.5), L("e8", N, 5e-324, 1e-300)],
    "erfc": lambda: [U("f1", N, -6, 27.3), U("f2", N, -1, 1), L("f3", N, 1e-300, 1e-3), U("f4", N, 0.9, 1.1),
                     U("f5", N, 1.9, 2.1), U("f6", N, 3.9, 4.1), U("f7", N, 7.9, 8.1), U("f8", N, 26, 27.5),
                     U("f9", N, -27, -0.9)],
}


@needs_quad
@pytest.mark.parametrize("fn", list(ERF_SETS))
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_erf_ulp_bound(fn, acc):
    x = np.concatenate(ERF_SETS[fn]() + [I.SPECIALS_F64])
    y = oracle.apply(f"{fn}_{acc}_f64", x)
    err = quadref.ulp_err(fn, x, y)
    i = int(np.argmax(err))
    assert err.max() <= BOUND[acc], (fn, acc, x[i], y[i], err.max())


@pytest.mark.parametrize("fn", ["erf", "erfc"])
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_erf_special_values(fn, acc):
    f = getattr(_libm, fn)
    f.restype, f.argtypes = ctypes.c_double, [ctypes.c_double]
    x = np.array(EDGE + [6.0, -6.0, 27.2, 27.3, 27.5, 28.0, -28.0, 8.0, -8.0, 4.0, 1.0, -1.0])
    y = oracle.apply(f"{fn}_{acc}_f64", x)
    for xi, yi in zip(x, y):
        want = f(float(xi))
        if math.isnan(want) or math.isinf(xi) or want == 0 or abs(want) in (1.0, 2.0) or xi == 0:
            assert _same(yi, want), (fn, acc, xi, yi, want)


def test_erf_identities():
    x = np.concatenate([U("g1", 50000, -6, 6), L("g2", 20000, 1e-300, 1)])
    e, c = oracle.apply("erf_u10_f64", x), oracle.apply("erfc_u10_f64", x)
    assert np.max(np.abs(e + c - 1)) <= 2.0 ** -52
    assert np.array_equal(oracle.apply("erf_u10_f64", -x), -e)
    c2 = oracle.apply("erfc_u10_f64", -x)
    assert np.max(np.abs(c + c2 - 2)) <= 2.0 ** -51


GAMMA_SETS = {
    "tgamma": lambda: [U("t1", N, -170, 171.6), U("t2", N, 0, 3), L("t3", N, 1e-300, 1e-3), U("t4", N, -5, 0),
                       U("t5", N, 160, 171.62), U("t6", N, -190, -170), L("t7", N, 5e-324, 1e-300, signed=False),
                       U("t8", N, 0.99, 2.01), -L("t9", N, 5e-324, 1e-290, signed=False),
                       U("t10", N, -1.0001, -0.9999)],
    "lgamma": lambda: [U("l1", N, 0, 1000), U("l2", N, 0, 3), L("l3", N, 1e-300, 2.5e305, signed=False),
                       U("l4", N, 0.99, 1.01), U("l5", N, 1.99, 2.01), U("l6", N, 1.2, 1.8), U("l7", N, 2.4, 8.5),
                       U("l9", N, 0.5, 0.8), L("l10", N, 5e-324, 1e-300, signed=False)],
}


@needs_quad
@pytest.mark.parametrize("fn", list(GAMMA_SETS))
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_gamma_ulp_bound(fn, acc):
    """tgamma everywhere, lgamma on x > 0 (relative accuracy across its zeros
    at 1 and 2): within the 1-ULP bound (u35 runs the same algorithm)."""
    x = np.concatenate(GAMMA_SETS[fn]() + [I.SPECIALS_F64[I.SPECIALS_F64 > 0] if fn == "lgamma" else I.SPECIALS_F64])
    y = oracle.apply(f"{fn}_{acc}_f64", x)
    err = quadref.ulp_err(fn, x, y)
    i = int(np.argmax(err))
    assert err.max() <= 1.0, (fn, acc, x[i], y[i], err.max())


@needs_quad
def test_lgamma_negative_axis():
    """x < 0: the reflection cancels near the zeros of lgamma (x = -2.457...,
    -2.747..., ...), as in every libm, so the bound there is absolute:
    |error| <= 2^-51 max(1, |lgamma x|); away from them (|lgamma x| >= 1) it
    is the 1-ULP bound."""
    x = np.concatenate([U("n1", N, -1000, 0), U("n2", N, -5, 0), U("n3", N, -2.5, -2.4),
                        L("n4", N, 1e-300, 1e-3, signed=False) * -1,
                        L("n5", N, 5e-324, 1e-260, signed=False) * -1,      # pi x subnormal: the 2^200 path
                        -np.array([5e-324, 1e-320, 2.0 ** -1022, 2.0 ** -900, 2.0 ** -901])])
    x = x[x != np.rint(x)]
    y = oracle.apply("lgamma_u10_f64", x)
    ref = quadref.ref("lgamma", x)
    assert np.max(np.abs(y - ref) / np.maximum(1, np.abs(ref))) <= 2.0 ** -51
    far = np.abs(ref) >= 1
    err = quadref.ulp_err("lgamma", x[far], y[far])
    assert err.max() <= 1.0, (x[far][np.argmax(err)], err.max())


@pytest.mark.parametrize("fn", ["tgamma", "lgamma"])
def test_gamma_special_values(fn):
    f = getattr(_libm, fn)
    f.restype, f.argtypes = ctypes.c_double, [ctypes.c_double]
    x = np.array([0.0, -0.0, 1.0, 2.0, -1.0, -2.0, -1e300, math.inf, -math.inf, math.nan, 172.0, 171.7,
                  -200.5, -201.5, 2.6e305, 5e-324, -0.5, 0.5, 3.0])
    y = oracle.apply(f"{fn}_u10_f64", x)
    for xi, yi in zip(x, y):
        want = f(float(xi))
        if math.isnan(want) or math.isinf(want) or want == 0 or xi in (1.0, 2.0):
            assert _same(yi, want), (fn, xi, yi, want)


@needs_quad
def test_gamma_identities():
    n = np.arange(1, 24, dtype=np.float64)
    fact = np.array([float(math.factorial(int(k) - 1)) for k in n])
    assert np.all(quadref.ulp_err("tgamma", n, oracle.apply("tgamma_u10_f64", n)) <= 1.0)
    assert np.max(np.abs(oracle.apply("tgamma_u10_f64", n) / fact - 1)) <= 2.0 ** -52
    x = np.round(U("gi", 20000, 0.1, 100) * 2.0 ** 40) * 2.0 ** -40      # x + 1 exact
    t, t1 = oracle.apply("tgamma_u10_f64", x), oracle.apply("tgamma_u10_f64", x + 1)
    ok = np.abs(t1 / (x * t) - 1) <= 2.0 ** -50
    assert ok.all()
    lg = oracle.apply("lgamma_u10_f64", x)
    assert np.max(np.abs(lg - np.log(t)) / np.maximum(1, np.abs(lg))) <= 2.0 ** -50
