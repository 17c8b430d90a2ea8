"""ctypes wrapper of quadref.c: __float128 reference values and ULP errors.

Available on x86-64 only (gcc's __float128 and libquadmath); tests that need
it skip elsewhere.
"""
import ctypes
import os
import platform
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build", "libquadref.so")
_lib = None


def available():
    return platform.machine() in ("x86_64", "AMD64")


def lib():
    global _lib
    if _lib is None:
        src = os.path.join(HERE, "quadref.c")
        if not os.path.exists(OUT) or os.path.getmtime(OUT) < os.path.getmtime(src):
            os.makedirs(os.path.dirname(OUT), exist_ok=True)
            tmp = OUT + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-fPIC", "-shared", src, "-o", tmp,
                            "-l:libquadmath.so.0", "-lm"], check=True)
            os.replace(tmp, OUT)
        _lib = ctypes.CDLL(OUT)
        for f in ("quad_ulp_f64", "quad_ulp_f32"):
            getattr(_lib, f).argtypes = [ctypes.c_char_p] + [ctypes.c_void_p] * 4 + [ctypes.c_size_t]
        _lib.quad_ref_f64.argtypes = [ctypes.c_char_p] + [ctypes.c_void_p] * 3 + [ctypes.c_size_t]
        _lib.quad_ulp_gen.argtypes = [ctypes.c_char_p] + [ctypes.c_void_p] * 3 + [ctypes.c_size_t] + \
            [ctypes.c_int] * 3
    return _lib


def ulp_err(fn, x, out, y=None):
    """ULP error of `out` against the __float128 value of fn(x[, y])."""
    f32 = np.asarray(out).dtype == np.float32
    dt = np.float32 if f32 else np.float64
    x = np.ascontiguousarray(x, dtype=dt)
    out = np.ascontiguousarray(out, dtype=dt)
    yp = None
    if y is not None:
        y = np.ascontiguousarray(y, dtype=dt)
        yp = y.ctypes.data
    err = np.empty(x.size, dtype=np.float64)
    f = lib().quad_ulp_f32 if f32 else lib().quad_ulp_f64
    if f(fn.encode(), x.ctypes.data, yp, out.ctypes.data, err.ctypes.data, x.size) != 0:
        raise KeyError(fn)
    return err


def ref(fn, x, y=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    yp = None
    if y is not None:
        y = np.ascontiguousarray(y, dtype=np.float64)
        yp = y.ctypes.data
    if lib().quad_ref_f64(fn.encode(), x.ctypes.data, yp, out.ctypes.data, x.size) != 0:
        raise KeyError(fn)
    return out


FORMATS = {"bf16": (8, -126, 127), "f16": (11, -14, 15)}


def ulp_err_fmt(fn, x, out, fmt):
    """ULP error of out (exact values given as doubles) in a 16-bit format."""
    p, emin, emax = FORMATS[fmt]
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.ascontiguousarray(out, dtype=np.float64)
    err = np.empty(x.size)
    if lib().quad_ulp_gen(fn.encode(), x.ctypes.data, out.ctypes.data, err.ctypes.data, x.size,
                          p, emin, emax) != 0:
        raise KeyError(fn)
    return err
