"""Coefficient design for the FP64 functions the paper does not describe
(cbrt, erf/erfc, tgamma/lgamma); the exponentials, logarithms and
hyperbolics reuse the exp/log/pow polynomials of fit_f64b.py.

Run:  python oracle/coeffs/fit_derived64.py [name ...]

  expm1_u35  e^r - 1 = r + r^2 u(r) with the error weighted relative to
         e^r - 1 (not e^r as for exp), |r| <= ln2/2, 12 terms
  cbrt   start value of the inverse cube root, m^(-1/3) on [1, 2] to about
         2^-26 relative, refined by Newton steps that need no division
"""
import os
import sys

sys.path.insert(0, os.path.dirname(__file__))
import mpmath as mp
from remez import fit_rounded, hexf

mp.mp.dps = 60


def show(name, stored, err):
    print(f"{name}: max weighted error 2^{float(mp.log(err, 2)):.2f}", flush=True)
    for e, v in stored:
        print(f"   x^{e}: {hexf(v)}", flush=True)


def icbrt(m):
    return m ** (-mp.mpf(1) / 3)


def icbrt_w(m):
    return 1 / icbrt(m)


LN2H = mp.log(2) / 2 * mp.mpf("1.0005")


def exp_u(r):
    if abs(r) < mp.mpf("1e-12"):
        return mp.mpf(1) / 2 + r / 6 + r * r / 24
    return (mp.exp(r) - 1 - r) / (r * r)


def expm1_w(r):
    if abs(r) < mp.mpf("1e-12"):
        return abs(r)
    return r * r / abs(mp.expm1(r))


JOBS = {
    "expm1_u35": lambda: fit_rounded(exp_u, expm1_w, range(10), ["d"] * 10, -LN2H, LN2H, n_grid=4000),
    "cbrt": lambda: fit_rounded(lambda t: icbrt(t + mp.mpf(1.5)), lambda t: icbrt_w(t + mp.mpf(1.5)),
                                range(8), ["d"] * 8, -mp.mpf(0.5), mp.mpf(0.5)),
}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(JOBS):
        show(name, *JOBS[name]())
