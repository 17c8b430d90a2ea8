"""Coefficient design for exp, log, pow, asin/acos and atan (FP64).

Run:  python oracle/coeffs/fit_f64b.py [name ...]
Prints the hex-float literals used in the oracle and the CUDA sources.

Shapes (the term counts are the paper's where it gives them):
  exp_u10   Section 5.6: e^r = 1 + r + r^2 (c2 + c3 r + ... + c12 r^10), 13 terms,
            |r| <= ln2/2 (+slack), no DD
  exp_u35   the same with 11 terms
  log_u10   Section 5.5: log m = z + z^3 P(z^2), z = 2(m-1)/(m+1)
            (log m = 2 atanh(z/2) is odd in z), |z| <= 0.4; 9 terms: the
            paper's 7 terms reach only 2^-49 relative error on this domain
  log_u35   8 terms
  powlog    Section 5.7: the internal log of pow, 11 terms, first correction
            coefficient as a DD pair
  powexp    Section 5.7: the internal exp of pow, e^r = 1 + r + r^2/2 +
            r^3 (c3 + ... + c12 r^9), 13 terms
  asin_u10  Section 5.3: asin u = u + u^3 P(u^2) on [0, 0.5]; 14 terms: the
            paper's 12 terms reach 2^-52 relative error, too much for 1 ULP
  asin_u35  12 terms
  atan_u10  Section 5.4: atan s = s + s^3 P(s^2) on [0, 1], the first
            correction coefficient as a DD pair; 22 terms: the paper's 20
            terms reach 2^-55 relative error, which with the final rounding
            leaves no margin under 1 ULP
  atan_u35  20 terms, all in double
"""
import os
import sys

sys.path.insert(0, os.path.dirname(__file__))
import mpmath as mp
from remez import fit_rounded, hexf

mp.mp.dps = 60
LN2H = mp.log(2) / 2 * mp.mpf("1.0005")


def show(name, stored, err):
    print(f"{name}: max weighted error 2^{float(mp.log(err, 2)):.2f}", flush=True)
    for e, v in stored:
        print(f"   x^{e}: {hexf(v)}", flush=True)


# e^r = 1 + r + r^2 u(r)
def exp_u(r):
    if abs(r) < mp.mpf("1e-12"):
        return mp.mpf(1) / 2 + r / 6 + r * r / 24
    return (mp.exp(r) - 1 - r) / (r * r)


def exp_w(r):
    return r * r / mp.exp(r)


# e^r = 1 + r + r^2/2 + r^3 v(r)
def exp_v(r):
    if abs(r) < mp.mpf("1e-10"):
        return mp.mpf(1) / 6 + r / 24 + r * r / 120
    return (mp.exp(r) - 1 - r - r * r / 2) / (r ** 3)


def exp_wv(r):
    return abs(r) ** 3 / mp.exp(r)


# log m = z + z^3 P(t), t = z^2, log m = 2 atanh(z/2)
def log_g(t):
    if t < mp.mpf("1e-12"):
        return mp.mpf(1) / 12 + t / 80
    z = mp.sqrt(t)
    return (2 * mp.atanh(z / 2) - z) / (z * t)


def log_w(t):
    z = mp.sqrt(t)
    return z * t / (2 * mp.atanh(z / 2)) if t != 0 else mp.mpf(0)


def asin_g(t):
    if t < mp.mpf("1e-12"):
        return mp.mpf(1) / 6 + 3 * t / 40
    u = mp.sqrt(t)
    return (mp.asin(u) - u) / (u * t)


def asin_w(t):
    u = mp.sqrt(t)
    return u * t / mp.asin(u) if t != 0 else mp.mpf(0)


def atan_g(t):
    if t < mp.mpf("1e-12"):
        return -mp.mpf(1) / 3 + t / 5
    s = mp.sqrt(t)
    return (mp.atan(s) - s) / (s * t)


def atan_w(t):
    s = mp.sqrt(t)
    return s * t / mp.atan(s) if t != 0 else mp.mpf(0)


JOBS = {
    "exp_u10": lambda: fit_rounded(exp_u, exp_w, range(11), ["d"] * 11, -LN2H, LN2H, n_grid=4000),
    "exp_u35": lambda: fit_rounded(exp_u, exp_w, range(9), ["d"] * 9, -LN2H, LN2H, n_grid=4000),
    "log_u10": lambda: fit_rounded(log_g, log_w, range(8), ["d"] * 8, 0, mp.mpf("0.4001") ** 2),
    "log_u35": lambda: fit_rounded(log_g, log_w, range(7), ["d"] * 7, 0, mp.mpf("0.4001") ** 2),
    "powlog": lambda: fit_rounded(log_g, log_w, range(10), ["dd"] + ["d"] * 9, 0, mp.mpf("0.4001") ** 2),
    "powexp": lambda: fit_rounded(exp_v, exp_wv, range(10), ["d"] * 10, -LN2H, LN2H),
    "asin_u10": lambda: fit_rounded(asin_g, asin_w, range(13), ["d"] * 13, 0, mp.mpf("0.25"), n_grid=4000),
    "asin_u35": lambda: fit_rounded(asin_g, asin_w, range(11), ["d"] * 11, 0, mp.mpf("0.25"), n_grid=4000),
    "atan_u10": lambda: fit_rounded(atan_g, atan_w, range(21), ["dd"] + ["d"] * 20, 0, 1, n_grid=4000),
    "atan_u35": lambda: fit_rounded(atan_g, atan_w, range(19), ["d"] * 19, 0, 1, n_grid=4000),
}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(JOBS):
        show(name, *JOBS[name]())
