"""Coefficient design for the FP64 functions the paper does not describe
(cbrt, erf/erfc, tgamma/lgamma); the exponentials, logarithms and
hyperbolics reuse the exp/log/pow polynomials of fit_f64b.py.

Run:  python oracle/coeffs/fit_derived64.py [name ...]

  expm1_u35  e^r - 1 = r + r^2 u(r) with the error weighted relative to
         e^r - 1 (not e^r as for exp), |r| <= ln2/2, 12 terms
  erf_a  erf(x)/x = C0 + t (C1 + t P(t)), t = x^2 in [0, 1], C0 and C1 as DD
         pairs, error relative to erf(x)/x
  erfc_F<i>  F(x) = erfc(x) e^(x^2) on [1,2), [2,4), [4,8) as
         c0 + u (c1 + u P(u)), u = x - (interval midpoint), 24 terms, c0 and c1
         as DD pairs, relative error
  erfc_G G(w) = sqrt(pi) x erfc(x) e^(x^2), w = 1/x^2 in [0, 1/64] (x >= 8),
         where the asymptotic series converges fast enough; 16 terms
  lgamma_r2  R(e) = lgamma(2 + e) / e on [-0.25, 0.5] (x in [1.75, 2.5)) as
         c1 + e (c2 + e Q(e)), c1 and c2 DD pairs, relative error; 18 terms
  lgamma_m   lgamma(1.5 + u) on [-0.25, 0.25] (x in [1.25, 1.75), around the
         minimum) as c0 + u (c1 + u (c2 + u Q(u))), c0, c1, c2 DD pairs; 18 terms
  lgamma_st  the Stirling correction x (lgamma(x) - (x - 1/2) log x + x -
         log(2 pi)/2) as a polynomial in w = 1/x^2 on [0, 1/64] (x >= 8)
  sinpi  sin(pi s) = s (pi + t (c1 + t Q(t))), t = s^2 in [0, 1/4], pi and c1
         DD pairs
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


ERFC_IV = [(1, 2), (2, 4), (4, 8)]


def erf_over_x(t):
    if t < mp.mpf("1e-30"):
        return 2 / mp.sqrt(mp.pi) * (1 - t / 3)
    x = mp.sqrt(t)
    return mp.erf(x) / x


def F(x):
    return mp.erfc(x) * mp.exp(x * x)


def G(w):
    if w < mp.mpf("1e-12"):
        return 1 - w / 2 + 3 * w * w / 4
    x = 1 / mp.sqrt(w)
    return mp.sqrt(mp.pi) * x * F(x)


def erfc_job(i, n):
    a, b = ERFC_IV[i]
    m = (mp.mpf(a) + mp.mpf(b)) / 2
    return lambda: fit_rounded(lambda u: F(m + u), lambda u: 1 / F(m + u), range(n), ["dd", "dd"] + ["d"] * (n - 2),
                               mp.mpf(a) - m, mp.mpf(b) - m, n_grid=3000)


def lg_r2(e):
    if abs(e) < mp.mpf("1e-25"):
        return 1 - mp.euler + (mp.zeta(2) - 1) / 2 * e
    return mp.loggamma(2 + e) / e


def lg_st(w):
    if w < mp.mpf("1e-30"):
        return mp.mpf(1) / 12 - w / 360
    x = 1 / mp.sqrt(w)
    return x * (mp.loggamma(x) - ((x - mp.mpf(0.5)) * mp.log(x) - x + mp.log(2 * mp.pi) / 2))


def sinpi_q(t):
    if t < mp.mpf("1e-30"):
        return -mp.pi ** 3 / 6 + mp.pi ** 5 / 120 * t
    s = mp.sqrt(t)
    return (mp.sin(mp.pi * s) / s - mp.pi) / t


def sinpi_w(t):
    s = mp.sqrt(t)
    return t * s / mp.sin(mp.pi * s) if t != 0 else mp.mpf(0)


JOBS = {
    "lgamma_r2": lambda: fit_rounded(lg_r2, lambda e: 1 / abs(lg_r2(e)), range(18), ["dd", "dd"] + ["d"] * 16,
                                     -mp.mpf("0.25"), mp.mpf("0.5"), n_grid=3000),
    "lgamma_m": lambda: fit_rounded(lambda u: mp.loggamma(mp.mpf("1.5") + u),
                                    lambda u: 1 / abs(mp.loggamma(mp.mpf("1.5") + u)), range(18),
                                    ["dd", "dd", "dd"] + ["d"] * 15, -mp.mpf("0.25"), mp.mpf("0.25"), n_grid=3000),
    "lgamma_st": lambda: fit_rounded(lg_st, lambda w: 1 / lg_st(w), range(10), ["d"] * 10, 0, mp.mpf(1) / 64,
                                     n_grid=3000),
    "sinpi": lambda: fit_rounded(sinpi_q, sinpi_w, range(12), ["dd"] + ["d"] * 11, 0, mp.mpf("0.25"), n_grid=3000),
    "erf_a": lambda: fit_rounded(erf_over_x, lambda t: 1 / erf_over_x(t), range(18), ["dd", "dd"] + ["d"] * 16,
                                 0, 1, n_grid=3000),
    "erfc_F0": erfc_job(0, 24),
    "erfc_F1": erfc_job(1, 24),
    "erfc_F2": erfc_job(2, 24),
    "erfc_G": lambda: fit_rounded(G, lambda w: 1 / G(w), range(16), ["dd", "dd"] + ["d"] * 14, 0,
                                  mp.mpf(1) / 64, n_grid=3000),
    "expm1_u35": lambda: fit_rounded(exp_u, expm1_w, range(10), ["d"] * 10, -LN2H, LN2H, n_grid=4000),
    "cbrt": lambda: fit_rounded(lambda t: icbrt(t + mp.mpf(1.5)), lambda t: icbrt_w(t + mp.mpf(1.5)),
                                range(8), ["d"] * 8, -mp.mpf(0.5), mp.mpf(0.5)),
}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(JOBS):
        show(name, *JOBS[name]())
