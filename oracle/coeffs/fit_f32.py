"""Coefficient design for the FP32 (float-float) family.

Run:  python oracle/coeffs/fit_f32.py [name ...]
Prints hex-float literals (binary32 values) for the oracle and CUDA sources.

The paper describes only the FP64 functions; the FP32 forms mirror them in
float-float (FF) arithmetic with binary32 coefficients:
  sinf     sin s = s + s t (c1 + t P(t)), |s| <= pi/2 (+slack), c1 as FF (u10)
  expf     e^r = 1 + r + r^2 u(r), |r| <= ln2/2
  logf     log m = z + z^3 P(z^2), z = 2(m-1)/(m+1), |z| <= 0.4
  expm1f   e^r - 1 = r + r^2/2 + r^3 v(r), |r| <= ln2/2 (tanh core)
  erff_a   erf x = x P(x^2) on [0, 1], the constant term as FF
  erff_b   erfc x = exp(-x^2 + L(x)) on [1, 3.95], L = log(erfc(x) e^(x^2))
           smooth and O(1) (absolute error), a polynomial in u = x - 2.475
  erfcf_a  erf x / x in t = x^2 on [0, 1] with three FF coefficients (1 - erf
           near x = 1 magnifies the error five-fold)
  erfcf_b  L on [1, 4] in u = x - 2.5 for erfc itself, the two leading
           coefficients FF (tighter than erff_b)
  erfcf_c  the same L on [3.9, 10.1] in u = x - 7 (erfc's tail)
  powlogf  the internal log of powf: log m = z + z^3 P(z^2) with the first
           coefficient FF, |z| <= 0.4
  cosf     cos s = 1 - t/2 + t^2 C(t), t = s^2, |s| <= 0.9 (pi/4 + slack)
  tanf     tan s = s + s t T(t), |s| <= 0.9, first term FF (u10)
  asinf    asin u = u + u^3 P(u^2) on [0, 0.5], first term FF (u10)
  atanf    atan s = s + s^3 P(s^2) on [0, 1], first term FF (u10)
  cbrtf    m^(-1/3) on [1, 2] in u = m - 1.5 (Newton start, about 2^-13)
  lgf_r2   lgamma(2 + e) / e on [-0.25, 0.5]; lgf_m lgamma(1.5 + u) on
           [-0.25, 0.25]; lgf_st Stirling correction in 1/x^2 for x >= 8;
           sinpif sin(pi s) / s on s^2 in [0, 1/4]; the leading terms FF
"""
import os
import sys

sys.path.insert(0, os.path.dirname(__file__))
import mpmath as mp
from remez import fit_rounded, hexf
from fit_trig import sin_g, sin_w
from fit_f64b import exp_u, exp_w, exp_v, exp_wv, log_g, log_w, LN2H

mp.mp.dps = 50


def show(name, stored, err):
    print(f"{name}: max weighted error 2^{float(mp.log(err, 2)):.2f}", flush=True)
    for e, v in stored:
        print(f"   x^{e}: {hexf(v)}", flush=True)


def erf_g(t):
    if t < mp.mpf("1e-20"):
        return 2 / mp.sqrt(mp.pi) * (1 - t / 3)
    x = mp.sqrt(t)
    return mp.erf(x) / x


def erf_w(t):
    x = mp.sqrt(t)
    return x / mp.erf(x) if t != 0 else 1 / (2 / mp.sqrt(mp.pi))


def erfc_r(x):
    return mp.erfc(x) * mp.exp(x * x)


def inv(f):
    return lambda x: 1 / f(x)


ERF_C = mp.mpf("2.475")


def erfc_r_u(u):
    return erfc_r(u + ERF_C)


def log_r_u(u):
    return mp.log(erfc_r(u + ERF_C))


def one(u):
    return mp.mpf(1)


# |s| bound: pi/2 plus the slack of q = rint(x * RN(1/pi)) for |x| < 2^20
TS = mp.mpf("1.7") ** 2
# |s| bound on quarter turns: Q = rint(RN(x RN(2/pi))) can miss the nearest
# integer for |x| < 2^20 (the product's rounding, up to 2^-5, and the
# constant's), so |s| <= (0.5 + 0.06) pi/2 < 0.9
TQ = mp.mpf("0.9") ** 2


def cos_g(t):
    if t < mp.mpf("1e-20"):
        return mp.mpf(1) / 24 - t / 720
    s = mp.sqrt(t)
    return (mp.cos(s) - 1 + t / 2) / (t * t)


def cos_w(t):
    return t * t / mp.cos(mp.sqrt(t))


def tan_g(t):
    if t < mp.mpf("1e-20"):
        return mp.mpf(1) / 3 + 2 * t / 15
    s = mp.sqrt(t)
    return (mp.tan(s) / s - 1) / t


def tan_w(t):
    s = mp.sqrt(t)
    return t * s / mp.tan(s) if t != 0 else mp.mpf(0)


def asin_g(t):
    if t < mp.mpf("1e-20"):
        return mp.mpf(1) / 6 + 3 * t / 40
    u = mp.sqrt(t)
    return (mp.asin(u) - u) / (u * t)


def asin_w(t):
    u = mp.sqrt(t)
    return u * t / mp.asin(u) if t != 0 else mp.mpf(0)


def atan_g(t):
    if t < mp.mpf("1e-20"):
        return -mp.mpf(1) / 3 + t / 5
    s = mp.sqrt(t)
    return (mp.atan(s) - s) / (s * t)


def atan_w(t):
    s = mp.sqrt(t)
    return s * t / mp.atan(s) if t != 0 else mp.mpf(0)


def lg_r2(e):
    if abs(e) < mp.mpf("1e-25"):
        return 1 - mp.euler + (mp.zeta(2) - 1) / 2 * e
    return mp.loggamma(2 + e) / e


def lg_st(w):
    if w < mp.mpf("1e-30"):
        return mp.mpf(1) / 12 - w / 360
    x = 1 / mp.sqrt(w)
    return x * (mp.loggamma(x) - ((x - mp.mpf(0.5)) * mp.log(x) - x + mp.log(2 * mp.pi) / 2))


def sinpi_g(t):
    if t < mp.mpf("1e-30"):
        return mp.pi - mp.pi ** 3 / 6 * t
    s = mp.sqrt(t)
    return mp.sin(mp.pi * s) / s


JOBS = {
    "sinf_u10": lambda: fit_rounded(sin_g, sin_w, range(5), ["ff"] + ["f"] * 4, 0, TS),
    "sinf_u35": lambda: fit_rounded(sin_g, sin_w, range(5), ["f"] * 5, 0, TS),
    "expf_u10": lambda: fit_rounded(exp_u, exp_w, range(6), ["f"] * 6, -LN2H, LN2H),
    "expf_u35": lambda: fit_rounded(exp_u, exp_w, range(5), ["f"] * 5, -LN2H, LN2H),
    "logf_u10": lambda: fit_rounded(log_g, log_w, range(4), ["f"] * 4, 0, mp.mpf("0.4001") ** 2),
    "logf_u35": lambda: fit_rounded(log_g, log_w, range(3), ["f"] * 3, 0, mp.mpf("0.4001") ** 2),
    "expm1f": lambda: fit_rounded(exp_v, exp_wv, range(5), ["f"] * 5, -LN2H, LN2H),
    "erff_a": lambda: fit_rounded(erf_g, erf_w, range(8), ["ff"] + ["f"] * 7, 0, 1),
    "erff_b": lambda: fit_rounded(log_r_u, one, range(12), ["ff"] + ["f"] * 11, 1 - ERF_C,
                                  mp.mpf("3.95") - ERF_C),
    "powlogf": lambda: fit_rounded(log_g, log_w, range(6), ["ff"] + ["f"] * 5, 0, mp.mpf("0.4001") ** 2),
    "erfcf_b": lambda: fit_rounded(lambda u: mp.log(erfc_r(u + mp.mpf("2.5"))), one, range(16),
                                   ["ff", "ff"] + ["f"] * 14, mp.mpf("-1.5"), mp.mpf("1.5")),
    "erfcf_a": lambda: fit_rounded(erf_g, erf_w, range(9), ["ff", "ff", "ff"] + ["f"] * 6, 0, 1),
    "erfcf_c": lambda: fit_rounded(lambda u: mp.log(erfc_r(u + 7)), one, range(13), ["ff", "ff"] + ["f"] * 11,
                                   mp.mpf("-3.1"), mp.mpf("3.1")),
    "cosf_u10": lambda: fit_rounded(cos_g, cos_w, range(3), ["f"] * 3, 0, TQ),
    "cosf_u35": lambda: fit_rounded(cos_g, cos_w, range(3), ["f"] * 3, 0, TQ),
    "tanf_u10": lambda: fit_rounded(tan_g, tan_w, range(9), ["ff"] + ["f"] * 8, 0, TQ),
    "tanf_u35": lambda: fit_rounded(tan_g, tan_w, range(8), ["f"] * 8, 0, TQ),
    "asinf_u10": lambda: fit_rounded(asin_g, asin_w, range(5), ["ff"] + ["f"] * 4, 0, mp.mpf("0.25")),
    "asinf_u35": lambda: fit_rounded(asin_g, asin_w, range(5), ["f"] * 5, 0, mp.mpf("0.25")),
    "atanf_u10": lambda: fit_rounded(atan_g, atan_w, range(10), ["ff"] + ["f"] * 9, 0, 1),
    "atanf_u35": lambda: fit_rounded(atan_g, atan_w, range(9), ["f"] * 9, 0, 1),
    "cbrtf": lambda: fit_rounded(lambda u: (u + mp.mpf(1.5)) ** (-mp.mpf(1) / 3),
                                 lambda u: (u + mp.mpf(1.5)) ** (mp.mpf(1) / 3), range(4), ["f"] * 4,
                                 -mp.mpf(0.5), mp.mpf(0.5)),
    "lgf_r2": lambda: fit_rounded(lg_r2, lambda e: 1 / abs(lg_r2(e)), range(10), ["ff", "ff"] + ["f"] * 8,
                                  -mp.mpf("0.25"), mp.mpf("0.5")),
    "lgf_m": lambda: fit_rounded(lambda u: mp.loggamma(mp.mpf("1.5") + u),
                                 lambda u: 1 / abs(mp.loggamma(mp.mpf("1.5") + u)), range(10),
                                 ["ff", "ff", "ff"] + ["f"] * 7, -mp.mpf("0.25"), mp.mpf("0.25")),
    "lgf_st": lambda: fit_rounded(lg_st, lambda w: 1 / lg_st(w), range(4), ["f"] * 4, 0, mp.mpf(1) / 64),
    "sinpif": lambda: fit_rounded(sinpi_g, lambda t: 1 / sinpi_g(t), range(7), ["ff", "ff"] + ["f"] * 5, 0,
                                  mp.mpf("0.25")),
}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(JOBS):
        show(name, *JOBS[name]())
