"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

Holds no arithmetic of the method: only random bit generation and the
mapping of random bits onto each function's argument domain.  Every array is
a pure function of (key, n, domain) and is built from integer operations and
exact power-of-two scalings, so the same bytes come out on x86-64 and Arm.

Recipe (the paper's workloads are uniform random arguments over stated
domains, Section 7, Table 3):
  uniform(a, b)       a + (b - a) * u,  u = (r >> 11) * 2^-53, r from PCG64
  loguniform(lo, hi)  binade chosen uniformly among those covering [lo, hi],
                      mantissa uniform within it, random sign if asked,
                      clamped into [lo, hi]
  mix                 per element: 89% main domain, 10% tail (log-uniform huge
                      arguments for the trig functions), 1% from SPECIALS_F64
"""
import hashlib
import math
import os

import numpy as np

_MASK53 = (1 << 53) - 1


def seed_of(key):
    return int.from_bytes(hashlib.sha256(str(key).encode()).digest()[:8], "little")


def raw(key, n):
    """n uint64 values of the PCG64 stream seeded by key (stream stable
    across numpy versions: only the bit generator is used)."""
    bg = np.random.PCG64(seed_of(key))
    return bg.random_raw(n).astype(np.uint64)


def unit(key, n):
    """n doubles uniform in [0, 1) with 53 random bits."""
    return (raw(key, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(key, n, a, b, dtype=np.float64):
    u = unit(key, n)
    x = a + (b - a) * u
    return x.astype(dtype)


def loguniform(key, n, lo, hi, signed=True, dtype=np.float64):
    r = raw(key, n)
    elo = math.frexp(lo)[1] - 1
    ehi = math.frexp(hi)[1] - 1
    nb = ehi - elo + 1
    e = elo + (r % np.uint64(nb)).astype(np.int64)
    mant = 1.0 + ((r >> np.uint64(11)) & np.uint64(_MASK53 >> 1)).astype(np.float64) * 2.0 ** -52
    x = np.ldexp(mant, e.astype(np.int32))
    x = np.clip(x, lo, hi)
    if signed:
        s = (raw(str(key) + "/sign", n) >> np.uint64(63)).astype(bool)
        x = np.where(s, -x, x)
    return x.astype(dtype)


def _pi_half_int(bits):
    """floor(pi/2 * 2^bits) from Machin's formula in integers (input
    generation only: used to place arguments next to multiples of pi/2)."""
    guard = bits + 16
    one = 1 << guard

    def atan_inv(k):
        s, t, n, k2 = 0, one // k, 0, k * k
        while t:
            s += t // (2 * n + 1) if n % 2 == 0 else -(t // (2 * n + 1))
            t //= k2
            n += 1
        return s
    pi = 16 * atan_inv(5) - 4 * atan_inv(239)
    return (pi >> 1) >> 16


def near_pi_half(ks):
    """RN(k pi/2) for integers k, as doubles."""
    P = _pi_half_int(1200)
    out = []
    for k in ks:
        v = k * P                      # k pi/2 * 2^1200
        e = v.bit_length() - 53        # keep 53 bits
        m = v >> e
        rem = v - (m << e)
        half = 1 << (e - 1)
        if rem > half or (rem == half and (m & 1)):
            m += 1
        out.append(math.ldexp(float(m), e - 1200))
    return np.array(out, dtype=np.float64)


def _specials():
    d = np.float64
    tiny = np.nextafter(d(0), d(1))
    maxsub = d(2.0 ** -1022) - tiny
    base = [0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, tiny, -tiny, maxsub, -maxsub,
            2.0 ** -1022, -(2.0 ** -1022), np.finfo(d).max, -np.finfo(d).max,
            1.0, -1.0, 0.5, -0.5, 2.0, -2.0, 15.0, -15.0,
            float(np.nextafter(d(15), d(0))), float(np.nextafter(d(15), d(20))),
            1e14, -1e14, float(np.nextafter(d(1e14), d(0))), float(np.nextafter(d(1e14), d(1e15))),
            2.0 ** 1023, 3 * 2.0 ** -1022, 0.75, 1.5, 3.0, 0.1,
            1e-300, -1e-300, 700.0, -700.0, 710.0, -745.5, 1e300, -1e300,
            math.pi, -math.pi, math.pi / 2, -math.pi / 2, 6.283185307179586, 1e22, -1e22, 100.0]
    k0 = int(1e22 * 2 / math.pi)
    near = list(near_pi_half(range(k0, k0 + 14)))
    vals = np.array(base + near, dtype=np.float64)
    assert vals.size == 64
    return vals


SPECIALS_F64 = _specials()


def specials_f32():
    """The FP64 specials rounded to binary32 (out-of-range values become
    infinities, tiny ones zeros or subnormals)."""
    with np.errstate(over="ignore", under="ignore"):
        return SPECIALS_F64.astype(np.float32)


# argument domains (main part) per function; trig tail = log-uniform huge
# arguments through the Payne-Hanek path.  Trig main domain [-100, 100]; the
# others follow Table 3 of the paper where it gives one.
DOMAINS_F64 = {
    "sin": (-100.0, 100.0), "cos": (-100.0, 100.0), "tan": (-100.0, 100.0),
    "sincos": (-100.0, 100.0),
    "asin": (-1.0, 1.0), "acos": (-1.0, 1.0), "atan": (-700.0, 700.0),
    "atan2": (-100.0, 100.0),
    "exp": (-700.0, 700.0), "exp2": (-1075.0, 1024.0), "exp10": (-324.0, 308.0),
    "expm1": (-700.0, 709.0),
    "log": (0.0, 1e300), "log2": (0.0, 1e300), "log10": (0.0, 1e300), "log1p": (-1.0, 1e300),
    "pow": (-30.0, 30.0), "cbrt": (-1e300, 1e300),
    "sinh": (-709.0, 709.0), "cosh": (-709.0, 709.0), "tanh": (-20.0, 20.0),
    "asinh": (-1e300, 1e300), "acosh": (1.0, 1e300), "atanh": (-1.0, 1.0),
    "erf": (-6.0, 6.0), "erfc": (-6.0, 27.3), "tgamma": (-170.0, 171.6),
    "lgamma": (-1e3, 2.5e305), "fmod": (-1e25, 1e25), "remainder": (-1e25, 1e25),
}
TRIG = ("sin", "cos", "tan", "sincos")
# FP32: the same mixes scaled to the binary32 range
DOMAINS_F32 = {
    "sin": (-100.0, 100.0), "cos": (-100.0, 100.0), "tan": (-100.0, 100.0), "sincos": (-100.0, 100.0),
    "asin": (-1.0, 1.0), "acos": (-1.0, 1.0), "atan": (-700.0, 700.0), "atan2": (-100.0, 100.0),
    "exp": (-87.0, 88.0), "exp2": (-150.0, 128.0), "exp10": (-45.0, 38.0), "expm1": (-87.0, 88.0),
    "log": (0.0, 3.4e38), "log2": (0.0, 3.4e38), "log10": (0.0, 3.4e38), "log1p": (-1.0, 3.4e38),
    "pow": (-30.0, 30.0), "cbrt": (-3.4e38, 3.4e38),
    "sinh": (-89.0, 89.0), "cosh": (-89.0, 89.0), "tanh": (-9.0, 9.0),
    "asinh": (-3.4e38, 3.4e38), "acosh": (1.0, 3.4e38), "atanh": (-1.0, 1.0),
    "erf": (-4.0, 4.0), "erfc": (-4.0, 10.0), "tgamma": (-40.0, 35.0), "lgamma": (-1e3, 4e36),
    "fmod": (-1e10, 1e10), "remainder": (-1e10, 1e10),
}
SPECIALS_F32_TAIL = (1e5, 3.4e38)


_BLOCK = 1 << 22


def _blocked(n, dtype, make):
    """Arrays above 2^22 elements are built block by block, each block from
    its own keyed streams (key + "#i"), on all host cores: the values depend
    only on the keys, never on the thread count."""
    if n <= _BLOCK:
        return make(n, "")
    from concurrent.futures import ThreadPoolExecutor
    out = np.empty(n, dtype=dtype)
    nb = (n + _BLOCK - 1) // _BLOCK

    def job(i):
        lo = i * _BLOCK
        m = min(_BLOCK, n - lo)
        out[lo:lo + m] = make(m, f"#{i}")
    with ThreadPoolExecutor(max_workers=min(nb, os.cpu_count() or 1)) as ex:
        list(ex.map(job, range(nb)))
    return out


def workload(fn, n, key="c2", dtype=np.float64, operand=0):
    """The mixed workload of one function: 89% uniform over the main domain,
    10% log-uniform tail, 1% specials, interleaved by a seeded choice.
    dtype float32 uses the binary32 domains (trig tail up to 3.4e38)."""
    return _blocked(n, dtype, lambda m, sfx: _workload_block(fn, m, key + sfx, dtype, operand))


def _workload_block(fn, n, key, dtype, operand):
    f32 = dtype == np.float32
    a, b = (DOMAINS_F32 if f32 else DOMAINS_F64)[fn]
    k = f"{key}/{fn}/{operand}" + ("/f32" if f32 else "")
    main = uniform(k + "/main", n, a, b)
    if fn in TRIG:
        tail = loguniform(k + "/tail", n, 1e5, 3.4e38 if f32 else 1e300)
    else:
        lo = max(1e-300, 0.0 if a <= 0 <= b else min(abs(a), abs(b)))
        hi = max(abs(a), abs(b))
        tail = loguniform(k + "/tail", n, max(lo, 1e-300), hi, signed=a < 0)
    specials = specials_f32().astype(np.float64) if f32 else SPECIALS_F64
    spec = specials[(raw(k + "/spec", n) % np.uint64(64)).astype(np.int64)]
    c = raw(k + "/cat", n) % np.uint64(100)
    x = np.where(c < 89, main, np.where(c < 99, tail, spec))
    if f32:
        with np.errstate(over="ignore", under="ignore"):
            x = x.astype(np.float32)
    return x


STRESS_FNS = ("sin", "cos", "tan", "sincos", "fmod", "remainder")


def stress(fn, n, key="c5", operand=0):
    """The large-argument stress workload: |x| log-uniform over [1e5, DBL_MAX]
    with a random sign (every trig lane takes the Payne-Hanek path); the
    divisor of fmod/remainder log-uniform over [1e-300, 1e300], random sign."""
    k = f"{key}/{fn}/{operand}"
    lo, hi = (1e5, 1.7976931348623157e308) if operand == 0 else (1e-300, 1e300)
    return _blocked(n, np.float64, lambda m, sfx: loguniform(k + sfx, m, lo, hi))


def fmod_sweep(r, n, key="sweep"):
    """The remainder workload of Section 7.1: d uniform in [1, 100] and the
    dividend uniform in [0.95 r d, 1.05 r d], for a quotient size r."""
    d = uniform(f"{key}/{r:g}/d", n, 1.0, 100.0)
    u = uniform(f"{key}/{r:g}/u", n, 0.95, 1.05)
    return u * (r * d), d


def c99_workload(name, n, key="c99", operand=0):
    """Inputs of the remaining C99 functions: x uniform in [-100, 100] with
    the 64 specials mixed in at the front (binary32 values rounded from
    binary64), the second operand independent the same way; sqrt takes |x|;
    hypot takes magnitudes log-uniform over [1e-300, 1e300] ([1e-35, 1e35]
    in binary32); ldexp's exponents are int32 uniform in [-60, 60]."""
    parts = name.split("_")
    fn, prec = parts[0], parts[-1]
    dt = np.float64 if prec == "f64" else np.float32
    cls = fn if fn in ("hypot", "ldexp") and operand == 1 or fn == "hypot" else "x"
    k = f"{key}/{cls}/{prec}/{operand}"          # the same arrays for every function of a class
    if fn == "ldexp" and operand == 1:
        return (raw(k, n) % np.uint64(121)).astype(np.int64).astype(np.int32) - 60
    if fn == "hypot":
        span = (1e-300, 1e300) if prec == "f64" else (1e-35, 1e35)
        return loguniform(k, n, *span, dtype=dt)
    x = uniform(k, n, -100.0, 100.0, dtype=dt)
    m = min(n, SPECIALS_F64.size)
    with np.errstate(over="ignore"):
        x[:m] = SPECIALS_F64[:m].astype(dt)
    return np.abs(x) if fn == "sqrt" else x


def to_bf16_bits(x32):
    """binary32 -> bf16 bit patterns, round-to-nearest-even (input preparation)."""
    b = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return r.astype(np.uint16)


def bits16_to_f64(h, fmt):
    """exact double values of bf16 / binary16 bit patterns."""
    h = np.asarray(h, dtype=np.uint16)
    if fmt == "bf16":
        return (h.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    return h.view(np.float16).astype(np.float64)


def activations(key, shape, fmt, sigma=3.0):
    """N(0, sigma) activations of the given shape as bf16 / binary16 bit
    patterns (Box-Muller in double, then binary32, then the 16-bit format)."""
    n = int(np.prod(shape))

    def block(m, sfx):
        u1 = (raw(key + sfx + "/u1", m) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 + 2.0 ** -54
        u2 = (raw(key + sfx + "/u2", m) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        return (sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).astype(np.float32)
    x32 = _blocked(n, np.float32, block)
    if fmt == "bf16":
        return to_bf16_bits(x32).reshape(shape)
    return x32.astype(np.float16).view(np.uint16).reshape(shape)
