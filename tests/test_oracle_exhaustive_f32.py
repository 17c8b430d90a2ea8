"""Exhaustive accuracy pin of the binary32 u10 oracle (P7 of the accuracy
plan): sin, exp and log u10 in binary32 over all 2^32 inputs, against the
binary64 u10 oracle of the same function (itself pinned within 1.0 binary64
ulp of the exact value by the quad tests, i.e. 2^-29 binary32 ulp).  The
bound asserted is the 1.0-ulp contract plus that slack; the measured maxima
are printed.  The loop runs in C on all host threads
(tests/exhaustive/f32_vs_f64.c) over the oracle's scalar entry points."""
import ctypes
import os
import subprocess

import pytest

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exhaustive")


@pytest.fixture(scope="module")
def helper(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("exh") / "libf32_vs_f64.so")
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", out, os.path.join(HERE, "f32_vs_f64.c"),
                    "-ldl", "-lpthread", "-lm"], check=True)
    L = ctypes.CDLL(out)
    L.exhaustive_max_ulp.restype = ctypes.c_double
    L.exhaustive_max_ulp.argtypes = [ctypes.c_char_p] * 3 + [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                                             ctypes.POINTER(ctypes.c_uint32)]
    return L


@pytest.mark.parametrize("fn", ["sin", "exp", "log"])
def test_every_binary32_input(helper, fn):
    lib = oracle.lib()._name.encode()
    am = ctypes.c_uint32(0)
    hi = int(os.environ.get("EXHAUSTIVE_F32_END", 1 << 32))
    err = helper.exhaustive_max_ulp(lib, f"oracle_{fn}_u10_f32".encode(), f"oracle_{fn}_u10_f64".encode(),
                                    0, hi, os.cpu_count() or 1, ctypes.byref(am))
    assert err >= 0, err
    print(f"{fn}_u10_f32: max {err:.4f} ulp over [0, {hi:#x}) at 0x{am.value:08x}")
    assert err <= 1.0 + 2.0 ** -28, (fn, err, hex(am.value))
