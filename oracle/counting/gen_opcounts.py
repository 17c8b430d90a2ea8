"""Write the algorithmic operation counts of the benchmark's workloads from
the counting build of the oracle (test infrastructure: the table it writes,
measure/opcounts.json, is data for the roofline of bench.py;
nothing in the package imports or runs this file).

Binary64 entry points are counted per reduction path (path classes defined
below; opcounts.py classifies the benchmark's arrays with the same bounds):
the table holds, per class, the mean count over up to SAMPLE_PER_CLASS
elements of that class drawn from the function's workload (the mixed C2
workload, plus the large-argument workload for the trig and remainder
functions).  fmod and remainder are counted per element and fitted exactly
as setup + step * (long-division steps).  Binary32 and 16-bit entry points
are counted as a mean per element over a sample of their own workloads.

Algorithmic operations are add/sub, mul, fma, div, sqrt and round-to-integer
(one each); divisions and square roots are also listed on their own, since
the device expands each into several pipe instructions.

    python -m oracle.counting.gen_opcounts      # rewrites the table
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2001_09258_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(ROOT, "measure", "opcounts.json")
SAMPLE = 1 << 17            # workload sample drawn per function
SAMPLE_PER_CLASS = 2048     # elements counted per path class
FMOD_SAMPLE = 512           # elements counted one by one per fmod workload


def classes(fn, x, y=None):
    """Path classes of a binary64 entry point: {class: boolean mask}."""
    ax = np.abs(x)
    if fn in ("sin", "cos", "tan", "sincos"):
        cw1 = ax < 15
        cw2 = (ax >= 15) & (ax < 1e14)
        return {"cw1": cw1, "cw2": cw2, "ph": ~(cw1 | cw2)}
    if fn == "asin":
        return {"small": ax <= 0.5, "big": ~(ax <= 0.5)}
    if fn == "acos":
        big = ~(ax <= 0.5)
        return {"small": ~big, "big": big & ~(x < 0), "bigneg": big & (x < 0)}
    if fn == "atan":
        return {"small": ax < 1, "big": ~(ax < 1)}
    if fn == "atan2":
        sw = ax > np.abs(y)
        yn = y < 0
        return {"b00": ~sw & ~yn, "b10": sw & ~yn, "b01": ~sw & yn, "b11": sw & yn}
    if fn in ("sinh", "cosh"):
        return {"small": ax <= 22, "big": ~(ax <= 22)}
    if fn in ("asinh", "acosh"):
        big = ax > 2.0 ** 500
        return {"small": ~big, "big": big}
    if fn == "erf":
        a = ax < 1
        f = (ax >= 1) & (ax < 6)
        return {"a": a, "f": f, "sat": ~(a | f)}
    if fn == "erfc":
        a = ax < 1
        f = (ax >= 1) & (ax < 8)
        g = (ax >= 8) & (ax <= 27.5)
        return {"a": a, "f": f & (x > 0), "fneg": f & ~(x > 0), "g": g, "sat": ~(a | f | g)}
    if fn in ("tgamma", "lgamma"):
        with np.errstate(invalid="ignore"):
            fin = np.isfinite(x) & (x != 0) & ~((x < 0) & (x == np.rint(x)))
        pos = fin & (x > 0) & ~(ax > 2.0 ** 1015)
        neg = fin & (x < 0)
        if fn == "tgamma":
            neg = neg & (x >= -190)
        c = {"st": pos & (x >= 8), "r2": pos & (x >= 1.75) & (x < 2.5), "m": pos & (x >= 1.25) & (x < 1.75),
             "lo": pos & (x >= 0.5) & (x < 1.25)}
        c["sh"] = pos & ~(c["st"] | c["r2"] | c["m"] | c["lo"])
        if fn == "lgamma":                         # Stirling without its two smallest terms
            c["stb"] = c["st"] & (x >= 2.0 ** 60)
            c["st"] = c["st"] & ~(x >= 2.0 ** 60)
        c["rs"] = neg & (x < -7)
        c["rn"] = neg & (x >= -7)
        rest = np.ones_like(pos)
        for v in c.values():
            rest &= ~v
        c["sp"] = rest
        return c
    return {"all": np.ones(x.shape, dtype=bool)}


def _binary(name):
    return oracle.kind(name) in (oracle.K_B64, oracle.K_B32)


def _entry(t, n, prec=None):
    if prec is None:
        prec = "f64" if t["f64"]["add"] + t["f64"]["mul"] + t["f64"]["fma"] else "f32"
    f = t[prec]
    ops = sum(f[c] for c in oracle.ALGO_CATS)
    return {"ops": round(ops / n, 4), "div": round(f["div"] / n, 4), "sqrt": round(f["sqrt"] / n, 4),
            "mul": round(f["mul"] / n, 4), "rnd": round(f["rnd"] / n, 4), "n": n}


def _count_f64(name, fn):
    xs = [I.workload(fn, SAMPLE, key="opcount", operand=0)]
    ys = [I.workload(fn, SAMPLE, key="opcount", operand=1)] if _binary(name) else [None]
    if fn in I.STRESS_FNS:
        xs.append(I.stress(fn, SAMPLE, key="opcount5"))
        ys.append(I.stress(fn, SAMPLE, key="opcount5", operand=1) if _binary(name) else None)
    x = np.concatenate(xs)
    y = np.concatenate(ys) if ys[0] is not None else None
    out = {}
    for cls, mask in classes(fn, x, y).items():
        idx = np.flatnonzero(mask)[:SAMPLE_PER_CLASS]
        if idx.size == 0:
            out[cls] = {"ops": 0.0, "div": 0.0, "sqrt": 0.0, "mul": 0.0, "rnd": 0.0, "n": 0}
            continue
        _, t = oracle.count(name, x[idx], None if y is None else y[idx])
        out[cls] = _entry(t, idx.size)
    return out


def _count_fmod(name, fn):
    """per-element counts over both workloads, as setup + step * steps: every
    long-division step costs the same whole number of operations (the
    least-squares slope, which must come out integral); the setup is the
    mean of the rest (it differs only by the fix-ups of rare cases)."""
    xs = np.concatenate([I.workload(fn, FMOD_SAMPLE, key="opcount"), I.stress(fn, FMOD_SAMPLE, key="opcount5")])
    ys = np.concatenate([I.workload(fn, FMOD_SAMPLE, key="opcount", operand=1),
                         I.stress(fn, FMOD_SAMPLE, key="opcount5", operand=1)])
    rows = []
    for a, b in zip(xs, ys):
        _, t = oracle.count(name, np.array([a]), np.array([b]))
        ops = sum(t["f64"][c] for c in oracle.ALGO_CATS)
        d = abs(b)
        if fn == "remainder" and np.isfinite(2 * d):
            d = 2 * d
        rows.append((oracle.fmod_iters(abs(a), d), ops, t["f64"]["div"], t["f64"]["mul"], t["f64"]["rnd"]))
    rows = np.array(rows, dtype=np.float64)
    fin = np.isfinite(xs) & np.isfinite(ys) & (ys != 0)
    it, ops = rows[fin, 0], rows[fin, 1]
    # the step cost: x = 1.5 * 2^(40 k), y = 1 needs more steps for larger k
    # with the same setup; the count must grow by the same amount per step
    pts = []
    for k in range(1, 12):
        a = 1.5 * 2.0 ** (40 * k)
        _, t = oracle.count(name, np.array([a]), np.array([1.0]))
        pts.append((oracle.fmod_iters(a, 2.0 if fn == "remainder" else 1.0),
                    sum(t["f64"][c] for c in oracle.ALGO_CATS), t["f64"]["mul"], t["f64"]["rnd"]))
    pts = np.array(sorted(set(pts)), dtype=np.float64)
    per = []
    for col in (1, 2, 3):                      # ops, mul, rnd per step
        slopes = np.diff(pts[:, col]) / np.diff(pts[:, 0])
        v = float(slopes[0])
        if not np.all(slopes == v) or v != int(v):
            raise RuntimeError(f"{name}: long-division steps do not cost a fixed count ({slopes})")
        per.append(v)
    step, step_mul, step_rnd = per
    setup = ops - step * it
    smul = rows[fin, 3] - step_mul * it
    srnd = rows[fin, 4] - step_rnd * it
    return {"setup": {"ops": round(float(setup.mean()), 4), "div": round(float(rows[fin, 2].mean()), 4),
                      "sqrt": 0.0, "mul": round(float(smul.mean()), 4), "rnd": round(float(srnd.mean()), 4),
                      "n": int(fin.sum()), "min": float(setup.min()), "max": float(setup.max())},
            "step": {"ops": step, "div": 0.0, "sqrt": 0.0, "mul": step_mul, "rnd": step_rnd, "n": int(fin.sum())}}


def table():
    f64, f32, lowp = {}, {}, {}
    for name in oracle.names():
        parts = name.split("_")
        fn, prec = parts[0], parts[-1]
        if prec == "f64":
            f64[name] = _count_fmod(name, fn) if fn in ("fmod", "remainder") else _count_f64(name, fn)
        elif prec == "f32":
            x = I.workload(fn, SAMPLE // 4, key="opcount", dtype=np.float32)
            y = I.workload(fn, SAMPLE // 4, key="opcount", dtype=np.float32, operand=1) if _binary(name) else None
            _, t = oracle.count(name, x, y)
            f32[name] = _entry(t, x.size)
        else:
            h = I.activations("opcount/act", (128, 256), prec).reshape(-1)
            _, t = oracle.count(name, h)
            lowp[name] = _entry(t, h.size)
    c99 = {}
    for name in oracle.c99_names():
        if oracle.kind(name) in (oracle.K_UI64, oracle.K_BI64, oracle.K_SI64,
                                 oracle.K_UI32, oracle.K_BI32, oracle.K_SI32):
            continue                     # exponent handling only: no floating-point arithmetic to count
        x = I.c99_workload(name, SAMPLE // 4)
        y = I.c99_workload(name, SAMPLE // 4, operand=1) if _binary(name) else None
        _, t = oracle.count(name, x, y)
        c99[name] = _entry(t, x.size, name.split("_")[-1])
    return {"unit": "algorithmic operations per element (add/sub, mul, fma, div, sqrt, round each one)",
            "source": "counting build of the oracle (oracle/counting), python -m oracle.counting.gen_opcounts",
            "f64": f64, "f32": f32, "lowp": lowp, "c99": c99}


def main():
    t = table()
    with open(OUT, "w") as f:
        json.dump(t, f, indent=1, sort_keys=True)
        f.write("\n")
    print(OUT)


if __name__ == "__main__":
    main()
