"""Algorithmic FP64 / FP32 operation counts per element, by reduction path.

One operation = one IEEE add, subtract, multiply, fused multiply-add,
round-to-integer, division or square root of the method's sequence (the
oracle's sequence, which the kernels reproduce; each division or square root
counts once although the device expands it into several pipe instructions).
Sign changes, comparisons, exponent handling and selects are integer work and
are not counted.  Counted by hand from the operation sequences; the
derivation of each line is in the design doc.

The roofline of these FP-pipe-bound kernels divides (ops per element x
elements) by the kernel time and compares it with the measured FMA-pipe peak.
"""
import numpy as np

# path keys: trig: "cw1" |x| < 15, "cw2" |x| < 1e14, "ph" otherwise
OPS = {
    "sin_u10_f64": {"cw1": 39, "cw2": 45, "ph": 93.5},
    "cos_u10_f64": {"cw1": 39, "cw2": 45, "ph": 93.5},
    "sin_u35_f64": {"cw1": 17, "cw2": 18, "ph": 75.5},
    "cos_u35_f64": {"cw1": 17, "cw2": 18, "ph": 75.5},
    "tan_u10_f64": {"cw1": 52, "cw2": 58, "ph": 105},
    "tan_u35_f64": {"cw1": 21, "cw2": 22, "ph": 78},
    "sincos_u10_f64": {"cw1": 54, "cw2": 60, "ph": 107},
    "sincos_u35_f64": {"cw1": 21, "cw2": 22, "ph": 78},
    "exp_u10_f64": {"all": 26},
    "exp_u35_f64": {"all": 18},
    "log_u10_f64": {"all": 36},
    "log_u35_f64": {"all": 17},
    "pow_u10_f64": {"all": 107},
    "pow_u35_f64": {"all": 107},
    # asin/acos: "small" |x| <= 0.5, "big" otherwise ("bigneg" x < -0.5 for acos)
    "asin_u10_f64": {"small": 23, "big": 36},
    "asin_u35_f64": {"small": 18, "big": 22},
    "acos_u10_f64": {"small": 28, "big": 31, "bigneg": 36},
    "acos_u35_f64": {"small": 20, "big": 21, "bigneg": 22},
    # atan: "small" |x| < 1, "big" otherwise
    "atan_u10_f64": {"small": 46, "big": 54},  # 22-term polynomial
    "atan_u35_f64": {"small": 25, "big": 27},
    # atan2: base + 5 (u35: 1) when |x| > |y| and again when y < 0
    "atan2_u10_f64": {"base": 52, "swap": 5, "yneg": 5},
    "atan2_u35_f64": {"base": 26, "swap": 1, "yneg": 1},
    # fmod / remainder: 4 setup ops (division, nextafter-free scaling) plus
    # 17 per step of the long division (trunc product 2, 3D and 2D 2, exact
    # q*D 2, DD add 8, renormalization 3), steps counted by the kernel's loop
    "fmod_u10_f64": {"setup": 4, "step": 17},
    "fmod_u35_f64": {"setup": 4, "step": 17},
    "remainder_u10_f64": {"setup": 9, "step": 17},
    "remainder_u35_f64": {"setup": 9, "step": 17},
    # functions on the exp/log cores.  Building blocks: exp tail (u10) 20,
    # DD exp core (k, e^r - 1 as a DD) 46, 2^k s + 2^k - 1 in DD 16, log core
    # on a DD argument 42 (u35 form 20), DD log 52; DD ops: TwoSum 6,
    # FastTwoSum 3, DD+DD 8 (fast 5), d+DD 7 (fast 4), DD*d 3, DD*DD 4,
    # DD/DD 6, 1/DD 4, sqrt of a DD 5; a polynomial of n coefficients costs
    # n-1 fma plus the squarings of Estrin's scheme
    "exp2_u10_f64": {"all": 25},
    "exp2_u35_f64": {"all": 18},
    "exp10_u10_f64": {"all": 30},
    "exp10_u35_f64": {"all": 20},
    "expm1_u10_f64": {"all": 63},
    "expm1_u35_f64": {"all": 20},
    "log2_u10_f64": {"all": 54},
    "log2_u35_f64": {"all": 44},
    "log10_u10_f64": {"all": 57},
    "log10_u35_f64": {"all": 45},
    "log1p_u10_f64": {"all": 59},
    "log1p_u35_f64": {"all": 27},
    "cbrt_u10_f64": {"all": 29},
    "cbrt_u35_f64": {"all": 24},
    # sinh/cosh: "small" |x| <= 22 (DD formula), "big" otherwise (e^|x|/2)
    "sinh_u10_f64": {"small": 85, "big": 51},
    "cosh_u10_f64": {"small": 63, "big": 51},
    "tanh_u10_f64": {"all": 77},
    "sinh_u35_f64": {"small": 24, "big": 19},
    "cosh_u35_f64": {"small": 23, "big": 19},
    "tanh_u35_f64": {"all": 23},
    # asinh/acosh: "big" |x| > 2^500 skips the square root
    "asinh_u10_f64": {"small": 74, "big": 61},
    "asinh_u35_f64": {"small": 74, "big": 61},
    "acosh_u10_f64": {"small": 81, "big": 61},
    "acosh_u35_f64": {"small": 81, "big": 61},
    "atanh_u10_f64": {"all": 72},
    "atanh_u35_f64": {"all": 72},
    # erf/erfc: "a" |x| < 1 (DD erf kernel 45: erf 49, erfc 56), "f" 1 <= |x|
    # < 6 (erf) or 8 (erfc) (interval polynomial in DD 45 + DD exp core 46 +
    # x^2, 1 + s and the product 10: erf 111, erfc 104 for x > 0 and 111 for
    # x < 0), "g" 8 <= |x| <= 27.5 (asymptotic form 42: erfc 101), "sat"
    # beyond (no arithmetic); u35 erf: 17 and 52
    "erf_u10_f64": {"a": 49, "f": 111, "g": 0, "sat": 0},
    "erfc_u10_f64": {"a": 56, "f": 104, "fneg": 111, "g": 101, "sat": 0},
    "erfc_u35_f64": {"a": 56, "f": 104, "fneg": 111, "g": 101, "sat": 0},
    "erf_u35_f64": {"a": 17, "f": 52, "g": 0, "sat": 0},
    # tgamma/lgamma by path class: "st" x >= 8 (Stirling with the DD log of
    # pow, 119), "r2" [1.75, 2.5) (52), "m" [1.25, 1.75) (59), "lo" [0.5, 1.25)
    # (polynomial and a DD log, 136), "sh" other x > 0 (shift: up to seven DD
    # products, a DD log and Stirling, ~240), "rs" x < -7 (reflection: exact
    # sin(pi x) 42, DD log, Stirling on 1 - x, 253), "rn" -7 <= x < 0 (~330),
    # "sp" specials; tgamma adds the DD exponential (51)
    "lgamma_u10_f64": {"st": 119, "r2": 52, "m": 59, "lo": 136, "sh": 240, "rs": 253, "rn": 330, "sp": 0},
    "lgamma_u35_f64": {"st": 119, "r2": 52, "m": 59, "lo": 136, "sh": 240, "rs": 253, "rn": 330, "sp": 0},
    "tgamma_u10_f64": {"st": 170, "r2": 103, "m": 110, "lo": 187, "sh": 291, "rs": 304, "rn": 381, "sp": 0},
    "tgamma_u35_f64": {"st": 170, "r2": 103, "m": 110, "lo": 187, "sh": 291, "rs": 304, "rn": 381, "sp": 0},
}


def path_mix(name, x, y=None, steps=None):
    """Number of elements of x on each path of entry point `name` (for
    fmod/remainder: `steps` = total long-division steps of the launch, as
    counted by the kernel's own loop)."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    fn = name.split("_")[0]
    if fn in ("sin", "cos", "tan", "sincos"):
        small = ax < 15
        mid = (ax >= 15) & (ax < 1e14)
        return {"cw1": int(small.sum()), "cw2": int(mid.sum()), "ph": int(ax.size - small.sum() - mid.sum())}
    if fn == "asin":
        big = int((~(ax <= 0.5)).sum())
        return {"small": ax.size - big, "big": big}
    if fn == "acos":
        big = ~(ax <= 0.5)
        bn = int((big & (x < 0)).sum())
        return {"small": int(ax.size - big.sum()), "big": int(big.sum()) - bn, "bigneg": bn}
    if fn == "atan":
        big = int((~(ax < 1)).sum())
        return {"small": ax.size - big, "big": big}
    if fn in ("fmod", "remainder"):
        if steps is None:
            raise ValueError(f"{name}: pass the total long-division step count (sleefcu_fmod_steps_f64)")
        return {"setup": ax.size, "step": int(steps)}
    if fn == "atan2":
        ay = np.abs(np.asarray(y, dtype=np.float64))
        return {"base": ax.size, "swap": int((ax > ay).sum()), "yneg": int((np.asarray(y) < 0).sum())}
    if fn in ("sinh", "cosh"):
        small = int((ax <= 22).sum())
        return {"small": small, "big": ax.size - small}
    if fn in ("erf", "erfc"):
        a = ax < 1
        f = (ax >= 1) & (ax < (6 if fn == "erf" else 8))
        g = (ax >= 8) & (ax <= 27.5) if fn == "erfc" else np.zeros_like(a)
        out = {"a": int(a.sum()), "g": int(g.sum()), "sat": int(ax.size - a.sum() - f.sum() - g.sum())}
        if fn == "erfc":
            out["f"] = int((f & (x > 0)).sum())
            out["fneg"] = int((f & ~(x > 0)).sum())
        else:
            out["f"] = int(f.sum())
        return out
    if fn in ("tgamma", "lgamma"):
        fin = np.isfinite(x) & (x != 0) & ~((x < 0) & (x == np.rint(x)))
        big = ax > 2.0 ** 1015
        pos, neg = fin & (x > 0) & ~big, fin & (x < 0)
        st = pos & (x >= 8)
        r2 = pos & (x >= 1.75) & (x < 2.5)
        m = pos & (x >= 1.25) & (x < 1.75)
        lo = pos & (x >= 0.5) & (x < 1.25)
        sh = pos & ~st & ~r2 & ~m & ~lo
        rs, rn = neg & (x < -7), neg & (x >= -7)
        if fn == "tgamma":
            rs, rn = rs & (x >= -190), rn
        c = {"st": st, "r2": r2, "m": m, "lo": lo, "sh": sh, "rs": rs, "rn": rn}
        out = {k: int(v.sum()) for k, v in c.items()}
        out["sp"] = int(ax.size - sum(out.values()))
        return out
    if fn in ("asinh", "acosh"):
        big = int((ax > 2.0 ** 500).sum())
        return {"small": ax.size - big, "big": big}
    return {"all": int(ax.size)}


def ops_per_launch(name, x, y=None, steps=None):
    tbl = OPS[name]
    return float(sum(tbl[k] * v for k, v in path_mix(name, x, y, steps).items()))
