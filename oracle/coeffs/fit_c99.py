"""Coefficient design for sinpi and cospi (both formats).

Run:  python oracle/coeffs/fit_c99.py [name ...]
Prints hex-float literals for the oracle and the CUDA sources.

After the exact reduction to s in [-1/4, 1/4] (t = s^2 in [0, 1/16]):
  sinpi   sin(pi s) = s g(t), g(t) = c0 + t (c1 + t Q(t)); c0 (about pi) and
          c1 as DD pairs (FF for the binary32 set), the rest plain
  cospi   cos(pi s) = 1 + t f(t), f(t) = (cos(pi sqrt t) - 1) / t =
          c1 + t R(t); c1 as a DD pair (FF), the rest plain
The 0.5-ULP entry points evaluate the leading terms in DD (FF) arithmetic;
the 3.5-ULP ones take the head of every pair and plain Horner steps.
"""
import os
import sys

sys.path.insert(0, os.path.dirname(__file__))
import mpmath as mp
from remez import fit_rounded, hexf

mp.mp.dps = 60
T16 = mp.mpf(1) / 16


def show(name, stored, err):
    print(f"{name}: max weighted error 2^{float(mp.log(err, 2)):.2f}", flush=True)
    for e, v in stored:
        print(f"   x^{e}: {hexf(v)}", flush=True)


def sin_g(t):
    if t < mp.mpf("1e-40"):
        return mp.pi - mp.pi ** 3 / 6 * t
    s = mp.sqrt(t)
    return mp.sin(mp.pi * s) / s


def cos_f(t):
    if t < mp.mpf("1e-40"):
        return -mp.pi ** 2 / 2 + mp.pi ** 4 / 24 * t
    return (mp.cos(mp.pi * mp.sqrt(t)) - 1) / t


JOBS = {
    "sinpi_f64": lambda: fit_rounded(sin_g, lambda t: 1 / sin_g(t), range(8), ["dd", "dd"] + ["d"] * 6, 0, T16,
                                     n_grid=2000),
    "cospi_f64": lambda: fit_rounded(cos_f, lambda t: 1 / abs(cos_f(t)), range(8), ["dd"] + ["d"] * 7, 0, T16,
                                     n_grid=2000),
    "sinpi_f32": lambda: fit_rounded(sin_g, lambda t: 1 / sin_g(t), range(6), ["ff", "ff"] + ["f"] * 4, 0, T16,
                                     n_grid=1000),
    "cospi_f32": lambda: fit_rounded(cos_f, lambda t: 1 / abs(cos_f(t)), range(5), ["ff"] + ["f"] * 4, 0, T16,
                                     n_grid=1000),
}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(JOBS):
        show(name, *JOBS[name]())
