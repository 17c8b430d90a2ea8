"""Pins of the oracle's remaining C99 functions (both formats).

The exact functions are written out on the IEEE fields in the oracle; here
they are checked against the platform's C library through numpy (trunc,
floor, ceil, rint, fabs, copysign, fmax, fmin, nextafter, ldexp, frexp,
modf, sqrt), against exact rational arithmetic (round, fdim) and against
Python's frexp (logb, ilogb), on uniformly random bit patterns (every
exponent, subnormals, infinities, NaNs) plus hand-set cases.  hypot, sinpi and
cospi are checked against binary128 within their bounds, and on the closed
forms and Annex F special values.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2001_09258_gb300 import inputs as I

N = 1 << 16
INT_MIN, INT_MAX = -(1 << 31), (1 << 31) - 1
FT = {"f64": np.float64, "f32": np.float32}
UT = {"f64": np.uint64, "f32": np.uint32}


def bits(key, prec, n=N):
    r = I.raw(key, n)
    if prec == "f64":
        return r.view(np.float64)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)


def hand(prec):
    t = FT[prec]
    fi = np.finfo(t)
    v = [0.0, -0.0, 0.5, -0.5, 1.5, -1.5, 2.5, -2.5, 0.49999999999999994, 1.0, -1.0, 3.0, 7.5,
         2.0 ** 52 + 1, 2.0 ** 52 - 0.5, 2.0 ** 23 + 0.5, -(2.0 ** 23) - 0.5, 2.0 ** 24 - 1,
         float(fi.max), -float(fi.max), float(fi.tiny), -float(fi.tiny), float(fi.smallest_subnormal),
         -float(fi.smallest_subnormal), np.inf, -np.inf, np.nan]
    return np.array(v, dtype=t)


def samples(prec, key):
    return np.concatenate([bits(key, prec), hand(prec)])


def same(a, b):
    """bit equality with every NaN equal to the canonical NaN on the oracle side"""
    a, b = np.asarray(a), np.asarray(b)
    u = UT[a.dtype.name.replace("float64", "f64").replace("float32", "f32")] if a.dtype.kind == "f" else None
    if u is None:
        return np.array_equal(a, b)
    nan = np.isnan(b)
    return np.array_equal(a[~nan].view(u), b[~nan].view(u)) and bool(np.all(np.isnan(a[nan])))


def canonical_nans(out, prec):
    o = np.asarray(out)
    want = 0x7FF8000000000000 if prec == "f64" else 0x7FC00000
    return bool(np.all(o[np.isnan(o)].view(UT[prec]) == want))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("fn,ref", [("trunc", np.trunc), ("floor", np.floor), ("ceil", np.ceil),
                                    ("rint", np.rint), ("sqrt_u05", np.sqrt), ("sqrt_u35", np.sqrt)])
def test_unary_against_libm(fn, ref, prec):
    x = samples(prec, f"c99/{fn}")
    with np.errstate(invalid="ignore"):
        want = ref(x)
    got = oracle.apply(f"{fn}_{prec}", x)
    assert same(got, want), fn
    assert canonical_nans(got, prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fabs_copysign_bits(prec):
    """sign-bit operations, bit for bit; a NaN result is the canonical NaN"""
    x, y = samples(prec, "c99/fa"), samples(prec, "c99/fb")
    for got, want in ((oracle.apply(f"fabs_{prec}", x), np.fabs(x)),
                      (oracle.apply(f"copysign_{prec}", x, y), np.copysign(x, y))):
        assert same(got, want)
        assert canonical_nans(got, prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_round_half_away_exact(prec):
    x = samples(prec, "c99/round")
    got = oracle.apply(f"round_{prec}", x)
    for xi, gi in zip(x.tolist(), got.tolist()):
        if not math.isfinite(xi):
            assert (math.isnan(xi) and math.isnan(gi)) or gi == xi
            continue
        f = Fraction(abs(xi))
        r = math.floor(f + Fraction(1, 2))
        want = math.copysign(float(r), xi)
        assert gi == want and math.copysign(1, gi) == math.copysign(1, want), xi


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_minmax_dim_nextafter(prec):
    x, y = samples(prec, "c99/mx"), samples(prec, "c99/my")
    x = np.concatenate([x, x[:5000]])
    y = np.concatenate([y, x[:5000]])                  # equal pairs too
    zeros = (x == 0) & (y == 0)
    for fn, ref in (("fmax", np.fmax), ("fmin", np.fmin)):
        got = oracle.apply(f"{fn}_{prec}", x, y)
        assert same(got[~zeros], ref(x, y)[~zeros]), fn
        assert canonical_nans(got, prec)
    with np.errstate(invalid="ignore", over="ignore"):
        assert same(oracle.apply(f"nextafter_{prec}", x, y), np.nextafter(x, y))
    got = oracle.apply(f"fdim_{prec}", x, y)
    for xi, yi, gi in zip(x.tolist(), y.tolist(), got.tolist()):
        if math.isnan(xi) or math.isnan(yi):
            assert math.isnan(gi)
        elif xi > yi:
            t = FT[prec]
            if math.isinf(xi) or math.isinf(yi):
                assert gi == xi - yi
            else:
                want = float(t(float(Fraction(xi) - Fraction(yi)))) if prec == "f64" else \
                    float(np.float32(Fraction(xi) - Fraction(yi)))
                assert gi == want or (math.isinf(gi) and abs(float(Fraction(xi) - Fraction(yi))) > 3e38)
        else:
            assert gi == 0 and math.copysign(1, gi) == 1


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_signed_zero_choices(prec):
    t = FT[prec]
    p, m = t(0.0), t(-0.0)
    a = np.array([p, m], dtype=t)
    b = np.array([m, p], dtype=t)
    assert list(np.signbit(oracle.apply(f"fmax_{prec}", a, b))) == [False, False]
    assert list(np.signbit(oracle.apply(f"fmin_{prec}", a, b))) == [True, True]
    assert list(np.signbit(oracle.apply(f"fdim_{prec}", a, b))) == [False, False]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ldexp_frexp_ilogb_logb_modf(prec):
    x = samples(prec, "c99/ld")
    r = I.raw("c99/ldn", x.size)
    n = ((r % np.uint64(4401)).astype(np.int64) - 2200).astype(np.int32)
    n[:64] = [INT_MIN, INT_MAX, 0, 1, -1, 1100, -1100, 2100, -2100, 160, -160, 300, -300] + [0] * 51
    with np.errstate(over="ignore", invalid="ignore"):
        assert same(oracle.apply(f"ldexp_{prec}", x, n), np.ldexp(x, n.clip(-100000, 100000)))
        m, e = oracle.apply(f"frexp_{prec}", x)
        wm, we = np.frexp(x)
    fin = np.isfinite(x)
    assert same(m, wm)
    assert np.array_equal(e[fin], we[fin]) and np.all(e[~fin] == 0)
    il = oracle.apply(f"ilogb_{prec}", x)
    lb = oracle.apply(f"logb_{prec}", x)
    for xi, a, b in zip(x.tolist(), il.tolist(), lb.tolist()):
        if math.isnan(xi):
            assert a == INT_MAX and math.isnan(b)
        elif math.isinf(xi):
            assert a == INT_MAX and b == math.inf
        elif xi == 0:
            assert a == INT_MIN and b == -math.inf
        else:
            k = math.frexp(xi)[1] - 1
            assert a == k and b == k
    with np.errstate(invalid="ignore"):
        fr, ip = oracle.apply(f"modf_{prec}", x)
        wfr, wip = np.modf(x)
    assert same(fr, wfr) and same(ip, wip)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_ldexp_rounding_cases(prec):
    """one rounding into the subnormal range, ties to even, and the carry
    into the least normal number"""
    t = FT[prec]
    emin, p = (-1022, 53) if prec == "f64" else (-126, 24)
    tiny = 2.0 ** (emin - p + 1)
    x = np.array([1.5, 2.5, 1.25, 1.75, 0.75, 1.0, 1.0 - 2.0 ** -p, 3.0], dtype=t)
    n = np.array([emin - p, emin - p, emin - p + 1, emin - p + 1, emin - p + 1, emin - p, emin, emin - p],
                 dtype=np.int32)
    got = oracle.apply(f"ldexp_{prec}", x, n).astype(np.float64)
    # 0.75, 1.25, 1.25, 1.75, 0.75 least subnormals round to the nearest; 0.5 and 1.5 are ties (to even);
    # 2^p - 1/2 least subnormals is a tie that carries into the least normal number
    want = [tiny, tiny, tiny, 2 * tiny, tiny, 0.0, 2.0 ** emin, 2 * tiny]
    assert got.tolist() == want


def _ulp_split(fn, x, out, prec, y=None):
    import quadref
    e = quadref.ulp_err(fn, x, out, y)
    tiny = 2.0 ** (-1022 if prec == "f64" else -126)
    sub = np.abs(out.astype(np.float64)) < tiny
    return e[~sub], e[sub]


def _lu(key, lo, hi, n, t):
    u = I.raw(key, n).astype(np.float64) / 2.0 ** 64
    s = np.where(I.raw(key + "/s", n) & np.uint64(1), 1.0, -1.0)
    return (np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo))) * s).astype(t)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_hypot_against_binary128(prec):
    import quadref
    if not quadref.available():
        pytest.skip("binary128 reference needs x86-64")
    t = FT[prec]
    lo, hi = (1e-320, 1e307) if prec == "f64" else (1e-44, 1e37)
    x = _lu("c99/hx", lo, hi, 40000, t)
    ratio = _lu("c99/hr", 1e-20, 1.0, 40000, np.float64)
    y = (x.astype(np.float64) * ratio).astype(t)
    x2 = _lu("c99/hx2", lo, hi, 20000, t)
    y2 = (x2 * t(0.75)).astype(t)
    x, y = np.concatenate([x, x2]), np.concatenate([y, y2])
    for acc, bound in (("u05", 0.5 + 2.0 ** -20), ("u35", 1.0)):
        out = oracle.apply(f"hypot_{acc}_{prec}", x, y)
        norm, sub = _ulp_split("hypot", x, out, prec, y)
        assert norm.max() <= bound, (acc, norm.max())
        assert sub.size == 0 or sub.max() <= 1.0, (acc, sub.max())


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("acc", ["u05", "u35"])
def test_hypot_special_values(prec, acc):
    t = FT[prec]
    big = float(np.finfo(t).max)
    x = np.array([np.inf, np.nan, -np.inf, np.nan, 3.0, -3.0, 0.0, -0.0, 5.0, big, 1.0, np.nan], dtype=t)
    y = np.array([np.nan, -np.inf, 1.0, 1.0, 4.0, -4.0, -0.0, -0.0, 0.0, big, -0.0, 0.0], dtype=t)
    got = oracle.apply(f"hypot_{acc}_{prec}", x, y).astype(np.float64)
    assert got[:3].tolist() == [np.inf] * 3                 # an infinity wins over a NaN
    assert np.isnan(got[3]) and np.isnan(got[11])
    assert got[4] == 5.0 and got[5] == 5.0
    assert got[6] == 0 and not np.signbit(got[6]) and not np.signbit(got[7])
    assert got[8] == 5.0 and got[10] == 1.0
    assert got[9] == np.inf


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("fn", ["sinpi", "cospi"])
def test_sincospi_against_binary128(fn, prec):
    import quadref
    if not quadref.available():
        pytest.skip("binary128 reference needs x86-64")
    t = FT[prec]
    big = 2.0 ** 53 if prec == "f64" else 2.0 ** 24
    u = (I.raw(f"c99/{fn}/u", 60000).astype(np.float64) / 2.0 ** 64 * 8 - 4).astype(t)
    lu = _lu(f"c99/{fn}/lu", 1e-320 if prec == "f64" else 1e-45, big, 60000, t)
    k = np.round((I.raw(f"c99/{fn}/k", 20000).astype(np.float64) / 2.0 ** 64 - 0.5) * 2e6) / 2
    near = np.concatenate([np.nextafter(k.astype(t), t(np.inf)), np.nextafter(k.astype(t), t(-np.inf))])
    x = np.concatenate([u, lu, near]).astype(t)
    for acc, bound in (("u05", 0.501), ("u35", 2.0)):
        out = oracle.apply(f"{fn}_{acc}_{prec}", x)
        norm, sub = _ulp_split(fn, x, out, prec)
        assert norm.max() <= bound, (acc, norm.max())
        assert sub.size == 0 or sub.max() <= 1.0, (acc, sub.max())


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("acc", ["u05", "u35"])
def test_sincospi_closed_forms(prec, acc):
    t = FT[prec]
    big = 2.0 ** 60
    x = np.array([0.0, -0.0, 0.5, -0.5, 1.0, -1.0, 3.0, -3.0, 1.5, -2.5, 0.25, -0.75, big, -big,
                  np.inf, np.nan, 1e6 + 0.5, -1e6], dtype=t)
    s = oracle.apply(f"sinpi_{acc}_{prec}", x).astype(np.float64)
    c = oracle.apply(f"cospi_{acc}_{prec}", x).astype(np.float64)
    r2 = float(t(math.sqrt(0.5)))
    assert s[:10].tolist() == [0, 0, 1, -1, 0, 0, 0, 0, -1, -1]
    assert list(np.signbit(s[[0, 1, 4, 5, 6, 7]])) == [False, True, False, True, False, True]
    assert c[:10].tolist() == [1, 1, 0, 0, -1, -1, -1, -1, 0, 0]
    assert not np.any(np.signbit(c[[2, 3, 8, 9, 16]]))          # cospi(n + 1/2) = +0
    if acc == "u05":
        assert s[10] == r2 and s[11] == -r2 and c[10] == r2 and c[11] == -r2
    assert s[12] == 0 and not np.signbit(s[12]) and np.signbit(s[13]) and c[12] == 1 and c[13] == 1
    assert np.isnan(s[14]) and np.isnan(c[14]) and np.isnan(s[15]) and np.isnan(c[15])
    assert s[16] == 1 and c[16] == 0 and c[17] == 1


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("acc", ["u05", "u35"])
def test_sincospi_symmetries(prec, acc):
    """sinpi odd, cospi even, both of period 2 (exact shifts), and
    sinpi(x + 1/2) = cospi(x) where x + 1/2 is exact"""
    t = FT[prec]
    x = (I.raw("c99/sym", 20000).astype(np.float64) / 2.0 ** 64 * 64 - 32)
    g = 2.0 ** (16 if prec == "f32" else 40)          # x, x +- 2 and x + 1/2 exactly representable
    x = (np.round(x * g) / g).astype(t)
    sp, cp = f"sinpi_{acc}_{prec}", f"cospi_{acc}_{prec}"
    s, c = oracle.apply(sp, x), oracle.apply(cp, x)
    assert same(oracle.apply(sp, -x), -s) and same(oracle.apply(cp, -x), c)
    assert same(oracle.apply(sp, x + t(2)), s) and same(oracle.apply(cp, x - t(2)), c)
    sh = oracle.apply(sp, x + t(0.5))
    nz = (c != 0) & (np.round(x * 4) != x * 4)        # quarter points reduce to s = +-1/4 either way
    assert same(sh[nz], c[nz])
