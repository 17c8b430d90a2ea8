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
}


def path_mix(name, x):
    """Number of elements of x on each path of entry point `name`."""
    ax = np.abs(np.asarray(x, dtype=np.float64))
    fn = name.split("_")[0]
    if fn in ("sin", "cos", "tan", "sincos"):
        small = ax < 15
        mid = (ax >= 15) & (ax < 1e14)
        return {"cw1": int(small.sum()), "cw2": int(mid.sum()), "ph": int(ax.size - small.sum() - mid.sum())}
    return {"all": int(ax.size)}


def ops_per_launch(name, x):
    tbl = OPS[name]
    return float(sum(tbl[k] * v for k, v in path_mix(name, x).items()))
