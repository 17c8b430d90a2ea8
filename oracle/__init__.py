"""ctypes access to the C oracle (oracle/_build/liboracle.so).

Test infrastructure: only tests/, the smoke check (__graft_entry__.smoke) and
the CPU-baseline leg of bench.py may import this package.  The library it
wraps is the plain scalar implementation of the method that the CUDA path is
checked against, bit for bit.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
K_U64, K_B64, K_SC64, K_U32, K_B32, K_SC32, K_U16 = 1, 2, 3, 11, 12, 13, 21
# the int32 kinds of the remaining C99 set: ilogb (x -> int), ldexp (x, int -> x),
# frexp (x -> x, int)
K_UI64, K_BI64, K_SI64, K_UI32, K_BI32, K_SI32 = 4, 5, 6, 14, 15, 16


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        _lib.oracle_apply.restype = ctypes.c_int
        _lib.oracle_apply.argtypes = [ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        _lib.oracle_kind.restype = ctypes.c_int
        _lib.oracle_kind.argtypes = [ctypes.c_char_p]
        _lib.oracle_count.restype = ctypes.c_int
        _lib.oracle_name.restype = ctypes.c_char_p
        _lib.oracle_name.argtypes = [ctypes.c_int]
        _lib.oracle_group.restype = ctypes.c_int
        _lib.oracle_group.argtypes = [ctypes.c_int]
        _lib.oracle_ph_reduce.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        _lib.oracle_ph_table_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        _lib.oracle_ph_tablef_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        _lib.oracle_fmod_recip.restype = ctypes.c_double
        _lib.oracle_fmod_recip.argtypes = [ctypes.c_double]
        _lib.oracle_fmod_iters.restype = ctypes.c_int
        _lib.oracle_fmod_iters.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib.oracle_fmod_trace.restype = ctypes.c_int
        _lib.oracle_fmod_trace.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int]
    return _lib


def names():
    """The functions of the vectorized method's set (group 0)."""
    L = lib()
    return [L.oracle_name(i).decode() for i in range(L.oracle_count()) if L.oracle_group(i) == 0]


def c99_names():
    """The remaining C99 functions (group 1)."""
    L = lib()
    return [L.oracle_name(i).decode() for i in range(L.oracle_count()) if L.oracle_group(i) == 1]


def kind(name):
    return lib().oracle_kind(name.encode())


def default_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def apply(name, x, y=None, nthreads=None):
    """Evaluate oracle function `name` elementwise.  Returns out, or
    (sin, cos) for sincos."""
    k = kind(name)
    if k == 0:
        raise KeyError(f"oracle has no function {name!r}")
    dt = np.float64 if k < 10 else (np.float32 if k < 20 else np.uint16)
    x = np.ascontiguousarray(x, dtype=dt)
    n = x.size
    out = np.empty(n, dtype=np.int32) if k in (K_UI64, K_UI32) else np.empty_like(x)
    out2 = np.empty_like(x) if k in (K_SC64, K_SC32) else None
    if k in (K_SI64, K_SI32):
        out2 = np.empty(n, dtype=np.int32)
    yp = None
    if k in (K_B64, K_B32, K_BI64, K_BI32):
        y = np.ascontiguousarray(y, dtype=np.int32 if k in (K_BI64, K_BI32) else dt)
        assert y.size == n
        yp = y.ctypes.data
    rc = lib().oracle_apply(name.encode(), x.ctypes.data, yp, out.ctypes.data,
                            out2.ctypes.data if out2 is not None else None, n,
                            nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"oracle_apply({name}) failed: {rc}")
    return (out, out2) if out2 is not None else out


def fmod_trace(x, y, maxk=64):
    qs = np.zeros(maxk)
    rs = np.zeros(maxk)
    k = lib().oracle_fmod_trace(float(x), float(y), qs.ctypes.data, rs.ctypes.data, maxk)
    return qs[:k], rs[:k]


def fmod_recip(d):
    """The reciprocal fmod's long division multiplies by (reading R33)."""
    return lib().oracle_fmod_recip(float(d))


def fmod_iters(x, y):
    return lib().oracle_fmod_iters(float(x), float(y))


def ph_reduce(x):
    q = ctypes.c_int()
    hi = ctypes.c_double()
    lo = ctypes.c_double()
    lib().oracle_ph_reduce(float(x), ctypes.byref(q), ctypes.byref(hi), ctypes.byref(lo))
    return q.value, hi.value, lo.value


def ph_tablef():
    tab = np.empty(512, dtype=np.float32)
    ib = np.empty(128, dtype=np.uint8)
    lib().oracle_ph_tablef_copy(tab.ctypes.data, ib.ctypes.data)
    return tab, ib


def ph_table():
    tab = np.empty(4096, dtype=np.float64)
    ib = np.empty(1024, dtype=np.uint8)
    lib().oracle_ph_table_copy(tab.ctypes.data, ib.ctypes.data)
    return tab, ib


# ---- counting build (oracle/counting): operation tallies of the same sources ----
COUNT_CATS = ("add", "mul", "fma", "div", "sqrt", "rnd", "cmp", "cvt", "scl")
ALGO_CATS = ("add", "mul", "fma", "div", "sqrt", "rnd")
_clib = None


def count_lib():
    global _clib
    if _clib is None:
        _clib = ctypes.CDLL(_build.build_count())
        _clib.oracle_count_apply.restype = ctypes.c_int
        _clib.oracle_count_apply.argtypes = [ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.c_void_p]
        _clib.oracle_count_ph.restype = None
        _clib.oracle_count_ph.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
        _clib.oracle_count_ncat.restype = ctypes.c_int
        assert _clib.oracle_count_ncat() == len(COUNT_CATS)
    return _clib


def _tally_dict(t):
    t = t.reshape(2, len(COUNT_CATS))
    return {p: dict(zip(COUNT_CATS, (int(v) for v in t[i]))) for i, p in enumerate(("f64", "f32"))}


def count(name, x, y=None):
    """Run the counting build of `name` over x (and y) on one thread.
    Returns (outputs as apply() returns them, tallies) with tallies =
    {"f64": {category: total}, "f32": {...}} summed over all elements."""
    k = kind(name)
    if k == 0:
        raise KeyError(f"oracle has no function {name!r}")
    dt = np.float64 if k < 10 else (np.float32 if k < 20 else np.uint16)
    x = np.ascontiguousarray(x, dtype=dt)
    out = np.empty_like(x)
    out2 = np.empty_like(x) if k in (K_SC64, K_SC32) else None
    yp = None
    if k in (K_B64, K_B32):
        y = np.ascontiguousarray(y, dtype=dt)
        assert y.size == x.size
        yp = y.ctypes.data
    t = np.zeros(2 * len(COUNT_CATS), dtype=np.uint64)
    rc = count_lib().oracle_count_apply(name.encode(), x.ctypes.data, yp, out.ctypes.data,
                                        out2.ctypes.data if out2 is not None else None, x.size,
                                        t.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_count_apply({name}) failed: {rc}")
    return ((out, out2) if out2 is not None else out), _tally_dict(t)


def count_ph(x):
    """Tallies of the binary64 Payne-Hanek reduction alone over x."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.zeros(2 * len(COUNT_CATS), dtype=np.uint64)
    count_lib().oracle_count_ph(x.ctypes.data, x.size, t.ctypes.data)
    return _tally_dict(t)


def algo_ops(tally, prec="f64"):
    """Algorithmic operation count: add + mul + fma + div + sqrt + rnd."""
    return sum(tally[prec][c] for c in ALGO_CATS)
