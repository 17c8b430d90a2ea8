"""Coefficient design for the trigonometric polynomials (FP64 and FP32).

Run:  python oracle/coeffs/fit_trig.py
Prints the hex-float literals used in the oracle and the CUDA sources.

Shapes (Section 5.1: one sine polynomial on [-pi/2, pi/2], 9 non-zero terms):
  sin_u10   sin s = s + s t (c1 + c2 t + ... + c8 t^7),  t = s^2, |s| <= 1.61,
            c1 stored as a DD pair (the term is evaluated in DD).
  sin_u35   same shape, doubles only, fewer terms.
  sc_sin    sin on |s| <= 0.81 (sincos reduces by quarter turns).
  sc_cos    cos s = 1 - t/2 + t^2 (d2 + d3 t + ...), |s| <= 0.81.
The interval bounds include the slack of q = rint(x * RN(1/pi)) for
|x| < 1e14 (at most 0.006 half turns past the ideal bound).
"""
import sys
import os
sys.path.insert(0, os.path.dirname(__file__))
import mpmath as mp
from remez import fit_rounded, hexf, to_float

mp.mp.dps = 50


def sin_g(t):
    if t < mp.mpf("1e-8"):
        return -mp.mpf(1) / 6 + t / 120 - t * t / 5040
    s = mp.sqrt(t)
    return (mp.sin(s) - s) / (s * t)


def sin_w(t):
    s = mp.sqrt(t)
    return s * t / mp.sin(s) if t != 0 else mp.mpf(0)


def cos_g(t):
    if t < mp.mpf("1e-8"):
        return mp.mpf(1) / 24 - t / 720
    s = mp.sqrt(t)
    return (mp.cos(s) - 1 + t / 2) / (t * t)


def cos_w(t):
    s = mp.sqrt(t)
    return t * t / mp.cos(s) if t != 0 else mp.mpf(0)


def show(name, stored, err):
    print(f"{name}: max weighted error 2^{float(mp.log(err, 2)):.2f}")
    for e, v in stored:
        print(f"   t^{e}: {hexf(v)}")


def main():
    which = sys.argv[1:] or ["sin_u10", "sin_u35", "sc_sin_u10", "sc_cos_u10",
                             "sc_sin_u35", "sc_cos_u35", "sinf_u10", "sinf_u35",
                             "scf_sin", "scf_cos"]
    T = mp.mpf("1.61") ** 2
    T2 = mp.mpf("0.81") ** 2
    if "sin_u10" in which:
        show("sin_u10", *fit_rounded(sin_g, sin_w, range(8), ["dd"] + ["d"] * 7, 0, T))
    if "sin_u35" in which:
        show("sin_u35", *fit_rounded(sin_g, sin_w, range(8), ["d"] * 8, 0, T))
    if "sc_sin_u10" in which:
        show("sc_sin_u10", *fit_rounded(sin_g, sin_w, range(6), ["dd"] + ["d"] * 5, 0, T2))
    if "sc_cos_u10" in which:
        show("sc_cos_u10", *fit_rounded(cos_g, cos_w, range(6), ["d"] * 6, 0, T2))
    if "sc_sin_u35" in which:
        show("sc_sin_u35", *fit_rounded(sin_g, sin_w, range(6), ["d"] * 6, 0, T2))
    if "sc_cos_u35" in which:
        show("sc_cos_u35", *fit_rounded(cos_g, cos_w, range(6), ["d"] * 6, 0, T2))
    # FP32: sin on |s| <= pi/2 (+slack), float-float leading term for u10
    Tf = mp.mpf("1.58") ** 2
    if "sinf_u10" in which:
        show("sinf_u10", *fit_rounded(sin_g, sin_w, range(5), ["ff"] + ["f"] * 4, 0, Tf))
    if "sinf_u35" in which:
        show("sinf_u35", *fit_rounded(sin_g, sin_w, range(4), ["f"] * 4, 0, Tf))
    T2f = mp.mpf("0.79") ** 2
    if "scf_sin" in which:
        show("scf_sin", *fit_rounded(sin_g, sin_w, range(4), ["f"] * 4, 0, T2f))
    if "scf_cos" in which:
        show("scf_cos", *fit_rounded(cos_g, cos_w, range(4), ["f"] * 4, 0, T2f))


if __name__ == "__main__":
    main()
