"""Algorithmic FP64 / FP32 operation counts per element, by reduction path.

One operation = one IEEE add, subtract, multiply, fused multiply-add,
round-to-integer, division or square root of the method's sequence (each
division or square root counts once although the device expands it into
several pipe instructions; they are also reported on their own).  Sign
changes, comparisons, exponent handling and selects are not counted.

The counts are those of the oracle's own operation sequence (which the
kernels reproduce bit for bit), tallied by its counting build over samples
of each path class of the benchmark's workloads and stored in opcounts.json
next to this file; this module only reads that table and classifies the
arrays of a launch by path.

The roofline of these FP-pipe-bound kernels divides (ops per element x
elements) by the kernel time and compares it with the measured FMA-pipe peak.
"""
import json
import os

import numpy as np

_TABLE = None


def table():
    global _TABLE
    if _TABLE is None:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "opcounts.json")) as f:
            _TABLE = json.load(f)
    return _TABLE


class _Ops(dict):
    """OPS[name][path] -> operations per element (binary64 entry points)"""
    def __missing__(self, name):
        v = {k: e["ops"] for k, e in table()["f64"][name].items()}
        self[name] = v
        return v


OPS = _Ops()


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
        # b<swap><yneg>: swap when |x| > |y|, yneg when y < 0
        sw = ax > np.abs(np.asarray(y, dtype=np.float64))
        yn = np.asarray(y, dtype=np.float64) < 0
        return {"b00": int((~sw & ~yn).sum()), "b10": int((sw & ~yn).sum()),
                "b01": int((~sw & yn).sum()), "b11": int((sw & yn).sum())}
    if fn in ("sinh", "cosh"):
        small = int((ax <= 22).sum())
        return {"small": small, "big": ax.size - small}
    if fn == "erf":
        a = ax < 1
        f = (ax >= 1) & (ax < 6)
        return {"a": int(a.sum()), "f": int(f.sum()), "sat": int(ax.size - a.sum() - f.sum())}
    if fn == "erfc":
        a = ax < 1
        f = (ax >= 1) & (ax < 8)
        g = (ax >= 8) & (ax <= 27.5)
        return {"a": int(a.sum()), "f": int((f & (x > 0)).sum()), "fneg": int((f & ~(x > 0)).sum()),
                "g": int(g.sum()), "sat": int(ax.size - a.sum() - f.sum() - g.sum())}
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
        if fn == "lgamma":                         # x >= 2^60: the shorter Stirling form
            c["stb"] = st & (x >= 2.0 ** 60)
            c["st"] = st & ~(x >= 2.0 ** 60)
        out = {k: int(v.sum()) for k, v in c.items()}
        out["sp"] = int(ax.size - sum(out.values()))
        return out
    if fn in ("asinh", "acosh"):
        big = int((ax > 2.0 ** 500).sum())
        return {"small": ax.size - big, "big": big}
    return {"all": int(ax.size)}


def _per_launch(name, x, y, steps, key):
    tbl = table()["f64"][name]
    return float(sum(tbl[k][key] * v for k, v in path_mix(name, x, y, steps).items()))


def ops_per_launch(name, x, y=None, steps=None):
    """algorithmic operations of one launch of a binary64 entry point"""
    return _per_launch(name, x, y, steps, "ops")


def mul_rnd_per_launch(name, x, y=None, steps=None):
    """(multiplications, roundings to integral) of one launch of a binary64
    entry point: the operations the single-array kernels run in software on
    the integer pipe (all FP64 families but tgamma / lgamma)"""
    return _per_launch(name, x, y, steps, "mul"), _per_launch(name, x, y, steps, "rnd")


# entry points whose multiplications stay on the FP64 pipe (their translation
# unit is compiled with SLEEFCU_SOFT_MUL 0): none of the single-array kernels
HW_MUL_FUNCS = ()


def div_sqrt_per_launch(name, x, y=None, steps=None):
    """(divisions, square roots) of one launch of a binary64 entry point"""
    return _per_launch(name, x, y, steps, "div"), _per_launch(name, x, y, steps, "sqrt")


def ops_per_element_f32(name):
    """mean algorithmic operations per element of a binary32 or 16-bit entry
    point over its workload (the 16-bit forms compute in binary32)"""
    t = table()
    return (t["f32"].get(name) or t["lowp"][name])["ops"]
