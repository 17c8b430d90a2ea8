"""sleefcu: GB300-native elementwise C99 math functions (SLEEF's method).

Thin Python binding over the C ABI in include/sleefcu.h (libsleefcu.so, built
in-tree by _build.py).  This module only marshals arguments: every step of
the computation runs in the CUDA kernels.  There is no CPU fallback: if the
library is missing or fails to load, every call raises.

    import paper_2001_09258_gb300 as sleefcu
    y = sleefcu.sin(x)                # x: CUDA float64 tensor, 1-ULP variant
    y = sleefcu.sin(x, ulp=35)        # 3.5-ULP variant
    s, c = sleefcu.sincos(x)
    sleefcu.call("pow_u10_f64", x, y, out=z)   # any entry point by name
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsleefcu.so")
LIB_CHECKED_PATH = os.path.join(_HERE, "_build", "libsleefcu_checked.so")

# (function, kind) for every entry point; kind: "u" unary, "b" binary (x, y),
# "sc" one input two outputs.  Each is exported for the listed accuracies and
# precisions as sleefcu_<fn>_<acc>_<prec>.
FUNCS = {
    "sin": "u", "cos": "u", "tan": "u", "sincos": "sc",
    "asin": "u", "acos": "u", "atan": "u", "atan2": "b",
    "exp": "u", "log": "u", "pow": "b",
    "fmod": "b", "remainder": "b",
    "log1p": "u", "tanh": "u", "erf": "u",
    "exp2": "u", "exp10": "u", "expm1": "u", "log2": "u", "log10": "u", "cbrt": "u",
    "sinh": "u", "cosh": "u", "asinh": "u", "acosh": "u", "atanh": "u", "erfc": "u",
    "tgamma": "u", "lgamma": "u",
}
PRECS = {fn: ("f64", "f32") for fn in FUNCS}
for _fn in ("erf", "tanh", "exp", "log1p"):
    PRECS[_fn] = PRECS[_fn] + ("bf16", "f16")
ACCS = ("u10", "u35")

# The remaining C99 real functions, both formats (binary64, binary32): kind as
# above plus "ui" (int32 result: ilogb), "bi" (int32 second operand: ldexp)
# and "si" (int32 second result: frexp).  Exact functions carry no accuracy
# tag (sleefcu_<fn>_<prec>); the approximated ones have a 0.5-ULP and a
# 3.5-ULP form (sleefcu_<fn>_<u05|u35>_<prec>).
C99_FUNCS = {
    "fabs": "u", "trunc": "u", "floor": "u", "ceil": "u", "round": "u", "rint": "u", "logb": "u",
    "copysign": "b", "fmax": "b", "fmin": "b", "fdim": "b", "nextafter": "b",
    "modf": "sc", "ilogb": "ui", "ldexp": "bi", "frexp": "si",
    "sqrt": "u", "hypot": "b", "sinpi": "u", "cospi": "u",
}
C99_ACCS = {"sqrt": ("u05", "u35"), "hypot": ("u05", "u35"), "sinpi": ("u05", "u35"), "cospi": ("u05", "u35")}

_lib = None
_lib_checked = None


class SleefcuError(RuntimeError):
    pass


def entry_points():
    """All C-ABI entry point names this binding knows (without the prefix)."""
    out = []
    for fn, kind in FUNCS.items():
        for prec in PRECS[fn]:
            for acc in ACCS:
                out.append(f"{fn}_{acc}_{prec}")
    return out


def c99_entry_points():
    """The entry points of the remaining C99 functions (without the prefix)."""
    out = []
    for fn in C99_FUNCS:
        for prec in ("f64", "f32"):
            if fn in C99_ACCS:
                out += [f"{fn}_{a}_{prec}" for a in C99_ACCS[fn]]
            else:
                out.append(f"{fn}_{prec}")
    return out


def masked_entry_points():
    """The masked FP64 entry points (sleefcu_<name>_masked), by the name of
    the entry point they mask."""
    return [e for e in entry_points() if e.endswith("_f64")]


def _declare(L):
    """Declare the argument and result types of every exported function."""
    L.sleefcu_last_error.restype = ctypes.c_char_p
    L.sleefcu_version.restype = ctypes.c_char_p
    L.sleefcu_is_checked.restype = ctypes.c_int
    L.sleefcu_is_checked.argtypes = []
    L.sleefcu_checked_error_count.restype = ctypes.c_int
    L.sleefcu_checked_error_count.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]
    L.sleefcu_fmod_steps_f64.restype = ctypes.c_int
    L.sleefcu_fmod_steps_f64.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_size_t, ctypes.c_void_p]
    for name in entry_points():
        fn = name.split("_")[0]
        f = getattr(L, "sleefcu_" + name)
        f.restype = ctypes.c_int
        nptr = {"u": 2, "b": 3, "sc": 3}[FUNCS[fn]]
        f.argtypes = [ctypes.c_void_p] * nptr + [ctypes.c_size_t, ctypes.c_void_p]
    for name in c99_entry_points():
        f = getattr(L, "sleefcu_" + name)
        f.restype = ctypes.c_int
        nptr = {"u": 2, "b": 3, "sc": 3, "ui": 2, "bi": 3, "si": 3}[C99_FUNCS[name.split("_")[0]]]
        f.argtypes = [ctypes.c_void_p] * nptr + [ctypes.c_size_t, ctypes.c_void_p]
    for name in masked_entry_points():
        fn = name.split("_")[0]
        f = getattr(L, "sleefcu_" + name + "_masked")
        f.restype = ctypes.c_int
        nptr = {"u": 3, "b": 4, "sc": 4}[FUNCS[fn]]          # the mask comes after the inputs
        f.argtypes = [ctypes.c_void_p] * nptr + [ctypes.c_size_t, ctypes.c_void_p]
    L.sleefcu_batch_create.argtypes = [ctypes.POINTER(BatchItem), ctypes.c_size_t, ctypes.c_char_p,
                                       ctypes.POINTER(ctypes.c_void_p)]
    for f in ("sleefcu_batch_launch", "sleefcu_batch_launch_graph"):
        getattr(L, f).argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.sleefcu_batch_autotune.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p]
    L.sleefcu_batch_set_config.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4
    L.sleefcu_batch_get_config.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 4
    L.sleefcu_batch_launch_static.argtypes = [ctypes.POINTER(BatchItem), ctypes.c_size_t, ctypes.c_void_p]
    L.sleefcu_eval_host.argtypes = [ctypes.POINTER(BatchItem), ctypes.c_size_t]
    L.sleefcu_eval_host_many.argtypes = [ctypes.POINTER(BatchItem), ctypes.c_size_t, ctypes.c_size_t]
    L.sleefcu_batch_destroy.argtypes = [ctypes.c_void_p]
    L.sleefcu_batch_destroy.restype = None
    return L


def _load(path):
    if not os.path.exists(path):
        from . import _build
        _build.build()
    try:
        return _declare(ctypes.CDLL(path))
    except OSError as e:
        raise SleefcuError(f"cannot load {path}: {e}") from e


def lib():
    """Load libsleefcu.so (building it first if it does not exist)."""
    global _lib
    if _lib is None:
        _lib = _load(LIB_PATH)
    return _lib


def lib_checked():
    """Load the checked build, libsleefcu_checked.so: the same entry points
    and results, plus device-pointer checks before every launch and a device
    error word (sleefcu_checked_error_count)."""
    global _lib_checked
    if _lib_checked is None:
        _lib_checked = _load(LIB_CHECKED_PATH)
    return _lib_checked


def last_error():
    return lib().sleefcu_last_error().decode()


def raw(name):
    """The ctypes function of entry point sleefcu_<name>.  Every function
    handed out has its argument types declared: an undeclared ctypes call
    would pass 64-bit device pointers as C ints."""
    f = getattr(lib(), "sleefcu_" + name)
    if f.argtypes is None:
        raise SleefcuError(f"sleefcu_{name}: no declared signature in the binding")
    return f


def _check(rc, name):
    if rc != 0:
        raise SleefcuError(f"sleefcu_{name} returned {rc}: {last_error()}")


def call(name, x, y=None, out=None, out2=None, stream=None):
    """Call entry point `name` on CUDA tensors; allocates outputs with
    empty_like when not given.  Returns out, or (out, out2) for sincos."""
    import torch
    fn = name.split("_")[0]
    kind = FUNCS[fn]
    if not x.is_cuda:
        raise SleefcuError("sleefcu works on CUDA tensors only")
    x = x.contiguous()
    if out is None:
        out = torch.empty_like(x)
    if kind == "sc" and out2 is None:
        out2 = torch.empty_like(x)
    st = stream if stream is not None else torch.cuda.current_stream(x.device)
    sp = ctypes.c_void_p(st.cuda_stream)
    f = raw(name)
    if kind == "u":
        rc = f(x.data_ptr(), out.data_ptr(), x.numel(), sp)
    elif kind == "b":
        y = y.contiguous()
        rc = f(x.data_ptr(), y.data_ptr(), out.data_ptr(), x.numel(), sp)
    else:
        rc = f(x.data_ptr(), out.data_ptr(), out2.data_ptr(), x.numel(), sp)
    _check(rc, name)
    return (out, out2) if kind == "sc" else out


def call_masked(name, x, mask, y=None, out=None, out2=None, stream=None):
    """sleefcu_<name>_masked on CUDA tensors: out[i] (and out2[i]) is
    computed where mask[i] != 0 (a uint8/bool tensor of x's length) and left
    as it is elsewhere.  Allocates outputs with empty_like when not given."""
    import torch
    fn = name.split("_")[0]
    kind = FUNCS[fn]
    if not x.is_cuda or not mask.is_cuda:
        raise SleefcuError("sleefcu works on CUDA tensors only")
    if mask.numel() != x.numel():
        raise SleefcuError("call_masked: mask and x differ in length")
    x = x.contiguous()
    m = mask.contiguous().view(torch.uint8) if mask.dtype == torch.bool else mask.contiguous()
    if out is None:
        out = torch.empty_like(x)
    if kind == "sc" and out2 is None:
        out2 = torch.empty_like(x)
    st = stream if stream is not None else torch.cuda.current_stream(x.device)
    sp = ctypes.c_void_p(st.cuda_stream)
    f = raw(name + "_masked")
    if kind == "u":
        rc = f(x.data_ptr(), m.data_ptr(), out.data_ptr(), x.numel(), sp)
    elif kind == "b":
        y = y.contiguous()
        rc = f(x.data_ptr(), y.data_ptr(), m.data_ptr(), out.data_ptr(), x.numel(), sp)
    else:
        rc = f(x.data_ptr(), m.data_ptr(), out.data_ptr(), out2.data_ptr(), x.numel(), sp)
    _check(rc, name + "_masked")
    return (out, out2) if kind == "sc" else out


def call_c99(name, x, y=None, out=None, out2=None, stream=None):
    """Call a C99-set entry point (c99_entry_points()) on CUDA tensors.
    ldexp takes an int32 tensor y; ilogb returns an int32 tensor; frexp and
    modf return two tensors (frexp: mantissa and int32 exponent; modf:
    fractional and integral part)."""
    import torch
    kind = C99_FUNCS[name.split("_")[0]]
    if not x.is_cuda:
        raise SleefcuError("sleefcu works on CUDA tensors only")
    x = x.contiguous()
    if out is None:
        out = torch.empty_like(x, dtype=torch.int32) if kind == "ui" else torch.empty_like(x)
    if kind in ("sc", "si") and out2 is None:
        out2 = torch.empty_like(x, dtype=torch.int32) if kind == "si" else torch.empty_like(x)
    st = stream if stream is not None else torch.cuda.current_stream(x.device)
    sp = ctypes.c_void_p(st.cuda_stream)
    f = raw(name)
    if kind in ("u", "ui"):
        rc = f(x.data_ptr(), out.data_ptr(), x.numel(), sp)
    elif kind in ("b", "bi"):
        y = y.contiguous()
        if y.numel() != x.numel():
            raise SleefcuError(f"{name}: x and y differ in length")
        rc = f(x.data_ptr(), y.data_ptr(), out.data_ptr(), x.numel(), sp)
    else:
        rc = f(x.data_ptr(), out.data_ptr(), out2.data_ptr(), x.numel(), sp)
    _check(rc, name)
    return (out, out2) if kind in ("sc", "si") else out


def _prec_of(x):
    import torch
    return {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16",
            torch.float16: "f16"}[x.dtype]


def _mk(fn):
    def f(x, y=None, ulp=10, out=None, out2=None):
        name = f"{fn}_u{ulp}_{_prec_of(x)}"
        if FUNCS[fn] == "b":
            return call(name, x, y, out=out)
        if FUNCS[fn] == "sc":
            return call(name, x, out=out, out2=out2)
        return call(name, x, out=out)
    f.__name__ = fn
    f.__doc__ = f"Elementwise {fn} via sleefcu_{fn}_u<ulp>_<prec>."
    return f


for _fn in FUNCS:
    globals()[_fn] = _mk(_fn)


def _mk_c99(fn):
    def f(x, y=None, ulp=5, out=None, out2=None):
        prec = _prec_of(x)
        name = f"{fn}_u{ulp:02d}_{prec}" if fn in C99_ACCS else f"{fn}_{prec}"
        return call_c99(name, x, y, out=out, out2=out2)
    f.__name__ = fn
    f.__doc__ = f"Elementwise {fn} via sleefcu_{fn}_<prec> (ulp=5 or 35 where the function has accuracy forms)."
    return f


for _fn in C99_FUNCS:
    globals()[_fn] = _mk_c99(_fn)


# ---------------- batched mixed launch ----------------
FN_IDS = {name: i for i, name in enumerate(
    ["sin", "cos", "tan", "sincos", "asin", "acos", "atan", "atan2", "exp", "log", "pow", "fmod",
     "remainder", "log1p", "tanh", "erf", "exp2", "exp10", "expm1", "log2", "log10", "cbrt", "sinh",
     "cosh", "asinh", "acosh", "atanh", "erfc", "tgamma", "lgamma"])}
DTYPE_IDS = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}


class BatchItem(ctypes.Structure):
    _fields_ = [("fn", ctypes.c_uint16), ("dtype", ctypes.c_uint8), ("ulp", ctypes.c_uint8),
                ("reserved", ctypes.c_uint32), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("out2", ctypes.c_void_p), ("n", ctypes.c_size_t)]


def _batch_lib():
    return lib()


def _items_array(items):
    arr = (BatchItem * max(len(items), 1))()
    for i, (name, x, y, out, out2) in enumerate(items):
        fn, acc, prec = name.split("_")
        arr[i] = BatchItem(FN_IDS[fn], DTYPE_IDS[prec], int(acc[1:]), 0,
                           x.data_ptr(), y.data_ptr() if y is not None else None,
                           out.data_ptr(), out2.data_ptr() if out2 is not None else None, x.numel())
    return arr


def batch_launch_static(items, stream=None):
    """sleefcu_batch_launch_static on (entry point name, x, y, out, out2)
    items: the batched evaluation without any device allocation."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    arr = _items_array(items)
    _check(_batch_lib().sleefcu_batch_launch_static(arr, len(items), ctypes.c_void_p(st.cuda_stream)),
           "batch_launch_static")


def eval_host(name, x, y=None, out=None, out2=None, chunk=0):
    """sleefcu_eval_host on host arrays (numpy arrays or raw addresses): the
    library copies chunks in, runs entry point `name` and copies results out,
    overlapped; returns when out holds every result."""
    import numpy as np
    fn, acc, prec = name.split("_")
    ptr = lambda a: None if a is None else (a.ctypes.data if isinstance(a, np.ndarray) else int(a))
    n = x.size if isinstance(x, np.ndarray) else None
    if n is None:
        raise SleefcuError("eval_host: pass numpy arrays")
    item = BatchItem(FN_IDS[fn], DTYPE_IDS[prec], int(acc[1:]), 0, ptr(x), ptr(y), ptr(out), ptr(out2), n)
    _check(_batch_lib().sleefcu_eval_host(ctypes.byref(item), chunk), "eval_host")
    return out


def eval_host_many(items, chunk=0):
    """sleefcu_eval_host_many on (entry point name, x, y, out, out2) items of
    host numpy arrays (y / out2 None where unused): one overlapped pipeline
    over all items; returns when every out holds its results."""
    import numpy as np
    arr = (BatchItem * max(len(items), 1))()
    ptr = lambda a: None if a is None else a.ctypes.data
    for i, (name, x, y, out, out2) in enumerate(items):
        if not isinstance(x, np.ndarray):
            raise SleefcuError("eval_host_many: pass numpy arrays")
        fn, acc, prec = name.split("_")
        arr[i] = BatchItem(FN_IDS[fn], DTYPE_IDS[prec], int(acc[1:]), 0, ptr(x), ptr(y), ptr(out), ptr(out2),
                           x.size)
    _check(_batch_lib().sleefcu_eval_host_many(arr, len(items), chunk), "eval_host_many")


class Batch:
    """A plan for sleefcu_batch_*: items are (entry point name, x, y, out, out2)
    with CUDA tensors (y / out2 None where unused).  tune_file: None keeps the
    default configuration; a path (or "" for no cache file) autotunes the
    plan inside sleefcu_batch_create."""

    def __init__(self, items, tune_file=None):
        L = _batch_lib()
        arr = (BatchItem * len(items))()
        self._keep = items
        for i, (name, x, y, out, out2) in enumerate(items):
            fn, acc, prec = name.split("_")
            arr[i] = BatchItem(FN_IDS[fn], DTYPE_IDS[prec], int(acc[1:]), 0,
                               x.data_ptr(), y.data_ptr() if y is not None else None,
                               out.data_ptr(), out2.data_ptr() if out2 is not None else None, x.numel())
        h = ctypes.c_void_p()
        tf = None if tune_file is None else tune_file.encode()
        _check(L.sleefcu_batch_create(arr, len(items), tf, ctypes.byref(h)), "batch_create")
        self.handle = h

    def _stream(self, stream):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(st.cuda_stream)

    def launch(self, stream=None, graph=False):
        f = _batch_lib().sleefcu_batch_launch_graph if graph else _batch_lib().sleefcu_batch_launch
        _check(f(self.handle, self._stream(stream)), "batch_launch")

    def autotune(self, cache_file=None, stream=None):
        c = cache_file.encode() if cache_file else None
        _check(_batch_lib().sleefcu_batch_autotune(self.handle, c, self._stream(stream)), "batch_autotune")

    def config(self):
        v = [ctypes.c_int() for _ in range(4)]
        _check(_batch_lib().sleefcu_batch_get_config(self.handle, *[ctypes.byref(a) for a in v]), "batch_get_config")
        return dict(zip(("block", "tile", "grid_mult", "vec"), (a.value for a in v)))

    def set_config(self, block, tile, grid_mult, vec):
        _check(_batch_lib().sleefcu_batch_set_config(self.handle, block, tile, grid_mult, vec), "batch_set_config")

    def close(self):
        if self.handle:
            _batch_lib().sleefcu_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
