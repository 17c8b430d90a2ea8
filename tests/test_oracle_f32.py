"""Pins of the FP32 (float-float) oracle: ULP bounds against __float128,
C99 Annex F special values against the host C library, the FP32
Payne-Hanek reduction against exact integer arithmetic, and its table
against an independent computation."""
import ctypes
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import quadref
from paper_2001_09258_gb300 import inputs as I

needs_quad = pytest.mark.skipif(not quadref.available(), reason="__float128 needs x86-64")
BOUND = {"u10": 1.0, "u35": 3.5}
N = 80000
F = np.float32


def _sets():
    trig = np.concatenate([I.uniform("fs1", N, -125, 125), I.loguniform("fs2", N, 125, 2 ** 20),
                           I.loguniform("fs3", N, 2 ** 20, 3.4e38), I.loguniform("fs4", N, 1e-45, 1),
                           I.uniform("fs5", N, -1, 1)])
    return {
        "sin": trig, "cos": trig,
        "exp": np.concatenate([I.uniform("fe1", N, -104, 89), I.uniform("fe2", N, -1, 1),
                               I.uniform("fe3", N, -103.9, -87)]),
        "log": np.concatenate([I.loguniform("fl1", N, 1e-45, 3.4e38, signed=False), I.uniform("fl2", N, 0.5, 2)]),
        "log1p": np.concatenate([I.uniform("fp1", N, -1, 1), I.loguniform("fp2", N, 1e-45, 3.4e38),
                                 I.uniform("fp3", N, -0.999, -0.5)]),
        "tanh": np.concatenate([I.uniform("ft1", N, -10, 10), I.loguniform("ft2", N, 1e-45, 20)]),
        "erf": np.concatenate([I.uniform("fr1", N, -4.5, 4.5), I.loguniform("fr2", N, 1e-45, 5),
                               I.uniform("fr3", N, 0.95, 1.05)]),
    }


SETS = _sets()
FUNCS = list(SETS)


@needs_quad
@pytest.mark.parametrize("fn", FUNCS)
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_f32_ulp_bound(fn, acc):
    x = SETS[fn].astype(F)
    x = x[np.isfinite(x)]
    x = np.concatenate([x, I.specials_f32()])
    y = oracle.apply(f"{fn}_{acc}_f32", x)
    err = quadref.ulp_err(fn, x, y)
    i = int(np.argmax(err))
    assert err.max() <= BOUND[acc], (fn, acc, x[i], y[i], err.max())


_libm = ctypes.CDLL("libm.so.6")
for _f in ("sinf", "cosf", "expf", "logf", "log1pf", "tanhf", "erff"):
    getattr(_libm, _f).restype = ctypes.c_float
    getattr(_libm, _f).argtypes = [ctypes.c_float]
SPEC = [0.0, -0.0, 1.0, -1.0, math.inf, -math.inf, math.nan, 1e-40, -1e-40, 3.4e38, -3.4e38, 0.5, -0.5]


@pytest.mark.parametrize("fn", FUNCS)
@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_f32_special_values(fn, acc):
    x = np.array(SPEC, dtype=F)
    y = oracle.apply(f"{fn}_{acc}_f32", x)
    for xi, yi in zip(x, y):
        ref = getattr(_libm, fn + "f")(float(xi))
        if math.isnan(ref):
            assert math.isnan(yi) and np.array([yi], dtype=F).view(np.uint32)[0] == 0x7FC00000, (fn, xi, yi)
        elif ref == 0 or math.isinf(ref) or abs(ref) == 1.0:
            if not (abs(ref) == 1.0 and abs(xi) not in (0.0, math.inf) and fn != "exp"):
                assert yi == ref and math.copysign(1, yi) == math.copysign(1, ref), (fn, xi, yi, ref)


@pytest.mark.parametrize("acc", ["u10", "u35"])
def test_f32_odd_symmetry_bitwise(acc):
    x = SETS["sin"][:50000].astype(F)
    for fn in ("sin", "tanh", "erf"):
        a = oracle.apply(f"{fn}_{acc}_f32", x)
        b = oracle.apply(f"{fn}_{acc}_f32", -x)
        assert np.array_equal(a.view(np.uint32), (-b).view(np.uint32)), fn


def test_f32_payne_hanek_bruteforce():
    """The FF Payne-Hanek reduction against x - k pi/2 with pi/2 to 400 bits."""
    f = oracle.lib().oracle_ph_reduce_f32
    f.argtypes = [ctypes.c_float, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                  ctypes.POINTER(ctypes.c_float)]
    B = 400
    P = I._pi_half_int(B)
    Pf = Fraction(P, 2 ** B)
    xs = list(I.loguniform("fph", 3000, 2 ** 20, 3.4e38).astype(F)) + [F(16367173 * 2.0 ** 72)]
    for x in xs:
        x = float(x)
        q, hi, lo = ctypes.c_int(), ctypes.c_float(), ctypes.c_float()
        f(x, ctypes.byref(q), ctypes.byref(hi), ctypes.byref(lo))
        X = Fraction(x)
        k = round(X / Pf)
        r = X - k * Pf
        d = (q.value - k) % 4
        if d:
            assert d in (1, 3) and abs(float(r)) > 0.78
            kk = k + (1 if d == 1 else -1)
            r = r - (kk - k) * Pf
        err = abs(Fraction(hi.value) + Fraction(lo.value) - r) / abs(r)
        assert err < 2.0 ** -40, (x, float(err))


def test_f32_payne_hanek_table_definition():
    mp = pytest.importorskip("mpmath")
    tab, ib = oracle.ph_tablef()
    assert np.all((tab.view(np.uint32) & np.uint32(1)) == 0)
    with mp.workprec(800):
        twoopi = 2 / mp.pi
        for E in range(0, 128, 3):
            M = -64 if E > 64 else 0
            v = twoopi * mp.mpf(2) ** (E - 24)
            ipart = mp.floor(v)
            m = (v - ipart) * mp.mpf(2) ** (-(E - 24 + M))
            for i in range(4):
                with mp.workprec(24):
                    t = float(+m)
                b = np.array([t], dtype=F).view(np.uint32)[0] & ~np.uint32(1)
                t = float(np.array([b], dtype=np.uint32).view(F)[0])
                assert tab[4 * E + i] == F(t), (E, i)
                m = m - t
            assert ib[E] == int(ipart) % 2
