"""Pins of the FP64 fmod/remainder oracle (Section 5.9): the results are
exact, so they must equal the host C library bit for bit; the worked
example of Section 5.9; the iteration count of Appendix C."""
import ctypes
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2001_09258_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_libm = ctypes.CDLL("libm.so.6")
for _f in ("fmod", "remainder"):
    getattr(_libm, _f).restype = ctypes.c_double
    getattr(_libm, _f).argtypes = [ctypes.c_double, ctypes.c_double]
N = 40000


def pair_sets():
    return [
        (I.loguniform("m1", N, 1e-300, 1.79e308), I.loguniform("m2", N, 1e-300, 1e300)),
        (I.loguniform("m3", N, 5e-324, 1.79e308), I.loguniform("m4", N, 5e-324, 1e-300)),
        (I.uniform("m5", N, -1e25, 1e25), I.uniform("m6", N, 1, 100)),
        (I.loguniform("m7", N, 1, 1e30), I.loguniform("m8", N, 1, 1e30)),
        (I.loguniform("m9", N, 1e300, 1.79e308), I.loguniform("m10", N, 5e-324, 1e-320)),
    ]


SPEC = [0.0, -0.0, 1.0, -1.0, 0.75, 3.0, -3.0, 2.5, math.inf, -math.inf, math.nan, 5e-324, -5e-324,
        2.2250738585072014e-308, 1.7976931348623157e308, -1.7976931348623157e308, 1e40, 1e-300]


def _ieee_zero_sign(x, y, ref):
    """IEEE 754 (5.3.1): a zero remainder has the sign of x."""
    return math.copysign(0.0, x) if ref == 0 else ref


@pytest.mark.parametrize("fn", ["fmod", "remainder"])
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_exact_against_libm(fn, acc):
    pairs = pair_sets() + [(np.array([p[0] for p in itertools.product(SPEC, SPEC)]),
                            np.array([p[1] for p in itertools.product(SPEC, SPEC)]))]
    for k, (x, y) in enumerate(pairs):
        r = oracle.apply(f"{fn}_{acc}_f64", x, y)
        ref = np.array([getattr(_libm, fn)(float(a), float(b)) for a, b in zip(x, y)])
        if fn == "remainder":
            ref = np.array([_ieee_zero_sign(a, b, v) for a, b, v in zip(x, y, ref)])
        nan = np.isnan(ref)
        assert np.all(np.isnan(r[nan])) and np.all(r[nan].view(np.uint64) == 0x7FF8000000000000)
        bad = np.nonzero(r[~nan].view(np.uint64) != ref[~nan].view(np.uint64))[0]
        assert bad.size == 0, (k, x[~nan][bad[0]], y[~nan][bad[0]], r[~nan][bad[0]], ref[~nan][bad[0]])


def test_worked_example():
    """Section 5.9, the worked-example figure: 1e40 / 0.75;
    first integer quotient about 1.333e40, second dividend about 4.836e24.
    The printed dividend is n - q d for q = RD53(n/d) - 2 ulp, which is what
    the oracle's reciprocal (reading R33) gives; the listing's formula with a
    correctly rounded 1/d would give RD53(n/d) - 1 ulp and 3.022e24.  Pinned:
    the quotient and the second dividend of the oracle's trace to the printed
    digits, both within Algorithm 1's allowed range."""
    from fractions import Fraction
    gold = dict(l.split() for l in open(os.path.join(ROOT, "tests", "golden", "fmod_example.txt"))
                if l.strip() and not l.startswith("#"))
    n, d = float(gold["n"]), float(gold["d"])
    qs, rs = oracle.fmod_trace(n, d)
    assert float(f"{qs[0]:.3e}") == float(gold["q0_approx"])
    s = Fraction(n) / Fraction(d)
    ulp = Fraction(2) ** (math.floor(math.log2(s)) - 52)
    rd = (s // ulp) * ulp
    q_paper = rd - int(gold["q0_ulps_below_rd_paper"]) * ulp
    r_paper = Fraction(n) - q_paper * Fraction(d)
    assert float(f"{float(r_paper):.3e}") == float(gold["r1_approx_paper"])
    assert s / 2 <= Fraction(qs[0]) <= s and Fraction(qs[0]) == q_paper
    assert Fraction(rs[0]) == Fraction(n) - Fraction(qs[0]) * Fraction(d)
    assert float(f"{rs[0]:.3e}") == float(gold["r1_approx_paper"])
    assert oracle.apply("fmod_u10_f64", np.array([n]), np.array([d]))[0] == math.fmod(n, d)


def test_iteration_count():
    """Appendix C: the loop needs ceil(log2(n/d) / (p-1)) steps (plus the
    fix-up steps for 1 < r/d < 3), p = 53."""
    x = I.loguniform("it1", 4000, 1, 1e300, signed=False)
    y = I.loguniform("it2", 4000, 1e-300, 1, signed=False)
    for a, b in zip(x, y):
        k = oracle.fmod_iters(a, b)
        bound = math.ceil((math.log2(a) - math.log2(b)) / 52)
        assert bound <= k + 1 and k <= bound + 3, (a, b, k, bound)
    assert max(oracle.fmod_iters(a, b) for a, b in [(1.79e308, 5e-324), (1.79e308, 1e-320)]) <= 44


def test_partial_remainders_stay_exact():
    """Appendix C: r_k is exactly representable in 2p bits, so every step's
    remainder r_k equals n - (sum of q_i) d computed in exact arithmetic."""
    from fractions import Fraction
    for n, d in [(1e40, 0.75), (123456789.123, 0.001), (1e300, 3.3), (7.5e22, 1.25e-3)]:
        qs, rs = oracle.fmod_trace(n, d)
        acc = Fraction(0)
        for q, r in zip(qs, rs):
            acc += Fraction(q)
            exact = Fraction(n) - acc * Fraction(d)
            assert abs(Fraction(r) - exact) <= abs(exact) * Fraction(1, 2 ** 52), (n, d)


def test_reciprocal_bound():
    """Reading R33: the reciprocal of the long division never exceeds 1/d and
    is within 2^-50 of it for d < 2^1021 (exact rationals; from 2^1021 on it
    is the listing's nextafter(1/d, 0)), so the quotient stays in
    Algorithm 1's range [(r/d)/2, r/d] (the proof's factor u =
    (1 - 2^-51)(1 - 2^-50)(1 - 2^-52) is far above the 5/6 it needs)."""
    from fractions import Fraction
    mant = (I.raw("recip", 100000) >> np.uint64(12)).astype(np.uint64)
    ex = (I.raw("recip/e", 100000) % np.uint64(2045)).astype(np.int64) - 1022
    ds = [math.ldexp(1.0 + int(m) * 2.0 ** -52, int(e)) for m, e in zip(mant, ex)]
    ds += [1.0, 2.0 - 2.0 ** -52, math.sqrt(2.0), 0.75, 3.0, 2.0 ** -1022, math.ldexp(2.0 - 2.0 ** -52, 1020),
           2.0 ** 1021, math.ldexp(2.0 - 2.0 ** -52, 1023), 1.5 - 2.0 ** -52, 1e-300, 1e300]
    worst = Fraction(0)
    for d in ds:
        r = Fraction(oracle.fmod_recip(d))
        e = 1 / Fraction(d)
        assert r <= e, d
        if d < 2.0 ** 1021:           # above, 1/d nears the subnormal range: the listing's own form
            worst = max(worst, (e - r) / e)
    assert worst < Fraction(1, 2 ** 50), float(worst)
