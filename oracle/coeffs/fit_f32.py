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
}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(JOBS):
        show(name, *JOBS[name]())
