"""Pins of the FP64 trigonometric oracle against things other than itself:
__float128 values (ULP bounds), exact integer reduction, the paper's printed
constants, C99 Annex F special values and closed forms."""
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import oracle
import quadref
from paper_2001_09258_gb300 import inputs as I

needs_quad = pytest.mark.skipif(not quadref.available(), reason="__float128 needs x86-64")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sets():
    s = {
        "u15": I.uniform("t/u15", 20000, -15, 15),
        "u100": I.uniform("t/u100", 20000, -100, 100),
        "cw2": I.loguniform("t/cw2", 20000, 15, 1e14),
        "ph": I.loguniform("t/ph", 20000, 1e14, 1.7e308),
        "tiny": I.loguniform("t/tiny", 5000, 5e-324, 1e-3),
        "near": I.near_pi_half(list(range(1, 400)) + list(range(10**6, 10**6 + 200))
                               + [int(1e13) + i for i in range(200)]),
        "special": I.SPECIALS_F64,
        "edges": np.array([np.nextafter(15.0, 0), 15.0, np.nextafter(1e14, 0), 1e14,
                           -np.nextafter(15.0, 0), -15.0, 6381956970095103 * 2.0 ** 797]),
    }
    return s


SETS = _sets()
BOUND = {"u10": 1.0, "u35": 3.5}


@needs_quad
@pytest.mark.parametrize("fn", ["sin", "cos", "tan"])
@pytest.mark.parametrize("acc", ["u10", "u35"])
@pytest.mark.parametrize("which", list(SETS))
def test_trig_ulp_bound(fn, acc, which):
    """Section 2 / Section 6: 1-ULP and 3.5-ULP bounds against a high-precision
    reference (MPFR in the paper, __float128 here)."""
    x = SETS[which]
    y = oracle.apply(f"{fn}_{acc}_f64", x)
    err = quadref.ulp_err(fn, x, y)
    worst = int(np.argmax(err))
    assert err.max() <= BOUND[acc], (fn, acc, which, x[worst], y[worst], err.max())


@needs_quad
@pytest.mark.parametrize("acc", ["u10", "u35"])
@pytest.mark.parametrize("which", list(SETS))
def test_sincos_ulp_bound(acc, which):
    x = SETS[which]
    s, c = oracle.apply(f"sincos_{acc}_f64", x)
    for fn, y in (("sin", s), ("cos", c)):
        err = quadref.ulp_err(fn, x, y)
        assert err.max() <= BOUND[acc], (fn, acc, which, x[int(np.argmax(err))], err.max())


def _bits(a):
    return np.asarray(a, dtype=np.float64).view(np.uint64)


CANON = np.uint64(0x7FF8000000000000)


@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_trig_special_values(acc):
    """C99 Annex F: sin/tan(+-0) = +-0, cos(+-0) = 1, non-finite -> NaN
    (Section 5.10: libm values, no errno, no flags); NaN results are the
    canonical quiet NaN."""
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan])
    for fn in ("sin", "tan"):
        y = oracle.apply(f"{fn}_{acc}_f64", x)
        assert list(_bits(y[:2])) == list(_bits(x[:2]))
        assert all(_bits(y[2:]) == CANON)
    y = oracle.apply(f"cos_{acc}_f64", x)
    assert list(y[:2]) == [1.0, 1.0] and all(_bits(y[2:]) == CANON)
    s, c = oracle.apply(f"sincos_{acc}_f64", x)
    assert list(_bits(s[:2])) == list(_bits(x[:2])) and list(c[:2]) == [1.0, 1.0]
    assert all(_bits(s[2:]) == CANON) and all(_bits(c[2:]) == CANON)


@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_trig_odd_symmetry_bitwise(acc):
    """rint is symmetric, so the reductions and odd polynomials give
    sin(-x) = -sin(x) and tan(-x) = -tan(x) bit for bit."""
    x = np.concatenate([SETS["u100"], SETS["cw2"][:5000], SETS["ph"][:5000]])
    for fn in ("sin", "tan"):
        a = oracle.apply(f"{fn}_{acc}_f64", x)
        b = oracle.apply(f"{fn}_{acc}_f64", -x)
        assert np.array_equal(_bits(a), _bits(-b)), fn


def test_sin2_cos2_closed_forms():
    x = SETS["u100"]
    s, c = oracle.apply("sincos_u10_f64", x)
    assert np.max(np.abs(s * s + c * c - 1)) < 4 * 2.0 ** -53
    assert abs(oracle.apply("sin_u10_f64", np.array([math.pi / 6]))[0] - 0.5) <= 2.0 ** -53
    assert oracle.apply("cos_u10_f64", np.array([0.0]))[0] == 1.0


def test_tan_uses_printed_constants():
    """Appendix A's tan listing fixes every coefficient and the Cody-Waite
    constants; the oracle source must carry exactly those values."""
    gold = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "tan_listing.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            gold[k] = float.fromhex(v) if "0x" in v else float(v)
    src = open(os.path.join(ROOT, "oracle", "src", "trig64.c")).read()
    body = re.search(r"TAN_C\[8\] = \{(.*?)\};", src, re.S).group(1)
    coeffs = [float(t) for t in re.findall(r"[-+]?[0-9.]+e[-+]?[0-9]+", body)]
    printed = [gold[f"estrin{i}"] for i in range(8)][::-1]      # constant term first
    assert coeffs == printed
    c3 = re.search(r"TAN_C3 = ([-+0-9.e]+);", src).group(1)
    assert float(c3) == gold["horner"]
    for name, key in (("PIO2_A", "pio2_hi"), ("PIO2_B", "pio2_lo"), ("TWOPI_H", "twopi_hi"),
                      ("TWOPI_L", "twopi_lo")):
        v = re.search(rf"#define {name} \(?([-0-9a-fx.p+]+)\)?", src).group(1)
        assert float.fromhex(v) == gold[key], name
    assert re.search(r"ax < 15 \?", src) and gold["threshold_cw"] == 15


# ---------------- Payne-Hanek (Section 5.8) ----------------

def _exact_reduce(x, P, B):
    """k = round(x / (pi/2)), r = x - k pi/2 with pi/2 to B bits (integers)."""
    m, e = math.frexp(abs(x))
    m = int(m * 2 ** 53)
    e -= 53
    X = m << (e + B)
    k = (2 * X + P) // (2 * P)
    r = Fraction(X - k * P, 2 ** B)
    return (-k, -r) if x < 0 else (k, r)


def test_payne_hanek_bruteforce():
    """The vectorized Payne-Hanek reduction against an exact reduction with
    pi/2 to 1500 bits: same quadrant mod 4, and the DD remainder agrees to
    2^-95 relative, including the hardest known case (|x mod pi/2| ~ 2^-61)."""
    B = 1500
    P = I._pi_half_int(B)
    Pf = Fraction(P, 2 ** B)
    xs = list(I.loguniform("ph/bf", 4000, 1e14, 1.79e308)) + \
        [6381956970095103 * 2.0 ** 797, 1e22, 2.0 ** 1023, 1e14] + list(I.SPECIALS_F64[-14:])
    for x in xs:
        x = float(x)
        q, hi, lo = oracle.ph_reduce(x)
        k, r = _exact_reduce(x, P, B)
        d = (q - k) % 4
        if d:          # a neighbouring quadrant is only allowed at |r| ~ pi/4
            assert d in (1, 3) and abs(float(r)) > 0.78, x
            kk = k + (1 if d == 1 else -1)
            r = r - (kk - k) * Pf
        err = abs(Fraction(hi) + Fraction(lo) - r) / abs(r)
        assert err < 2.0 ** -95, (x, float(err))
        assert abs(hi) <= math.pi / 4 + 1e-9


def test_payne_hanek_bruteforce_million():
    """The same exact check on 10^6 log-uniform huge arguments (1e14 to
    DBL_MAX), in integers scaled by 2^1500: the reduction x - k pi/2 with
    pi/2 to 1500 bits, the oracle's DD remainder hi + lo (every double down
    to 2^-1074 is an integer multiple of 2^-1500), same quadrant mod 4 (a
    neighbouring one only where |r| is near pi/4), relative error < 2^-95."""
    import ctypes
    B = 1500
    P = I._pi_half_int(B)
    near_quarter = 780 * (1 << B)          # 0.780 in units of 2^-1500, times 1000

    def scaled(v):                          # v * 2^B as an exact integer
        if v == 0.0:
            return 0
        m, e = math.frexp(v)
        return int(m * 2 ** 53) << (e - 53 + B)

    f = oracle.lib().oracle_ph_reduce
    q, hi, lo = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    xs = I.loguniform("ph/bf1m", 10 ** 6, 1e14, 1.79e308)
    for x in xs.tolist():
        f(x, ctypes.byref(q), ctypes.byref(hi), ctypes.byref(lo))
        m, e = math.frexp(abs(x))
        X = int(m * 2 ** 53) << (e - 53 + B)
        k = (2 * X + P) // (2 * P)
        r = X - k * P
        if x < 0:
            k, r = -k, -r
        d = (q.value - k) % 4
        if d:
            assert d in (1, 3) and abs(r) * 1000 > near_quarter, x
            r -= (1 if d == 1 else -1) * P
        assert abs(scaled(hi.value) + scaled(lo.value) - r) << 95 < abs(r), x


def test_payne_hanek_table_definition():
    """the Payne-Hanek table-generation figure: 1024 x 4 doubles (32 KB), each the
    RN double of the remaining fraction with its lowest bit cleared, E > 700
    scaled by 2^128; recomputed here independently with mpmath at 2000 bits."""
    mp = pytest.importorskip("mpmath")
    tab, ib = oracle.ph_table()
    assert tab.nbytes == 32768
    assert np.all((tab.view(np.uint64) & np.uint64(1)) == 0)
    with mp.workprec(2000):
        twoopi = 2 / mp.pi
        for E in list(range(0, 1024, 7)) + [700, 701, 1023]:
            M = -128 if E > 700 else 0
            v = twoopi * mp.mpf(2) ** (E - 53)
            ipart = mp.floor(v)
            m = (v - ipart) * mp.mpf(2) ** (-(E - 53 + M))
            for i in range(4):
                with mp.workprec(53):
                    t = float(+m)
                b = np.array([t]).view(np.uint64)[0] & ~np.uint64(1)
                t = np.array([b], dtype=np.uint64).view(np.float64)[0]
                assert tab[4 * E + i] == t, (E, i)
                m = m - t
            assert ib[E] == int(ipart) % 2, E
