"""Exact binary64 arithmetic on the integer pipe (csrc/softfp64.cuh).

Correctly rounded IEEE operations are unique (the bit-consistency argument of
Section 4), so the software fma, add, mul, rint and trunc must equal the host
processor's hardware operations bit for bit (NaN results: NaN-ness on the
host, whose NaN payload rules differ) and the GPU's FP64 pipe bit for bit
(NaN bits included).  Pinned on:
  * structured random operands (tests/softfp/softfp_gen.h): uniform bit
    patterns, cancellation against RN(a b), subnormal and near-overflow
    ranges, few-bit significands that produce exact ties, specials mixed with
    finite values, additions with close exponents, products with a zero
    addend -- 2^29 triples x 5 operations on the host cores
    (SOFTFP_CASES=<per mode per thread> for larger runs);
  * directed cases: ties to even in the normal and subnormal range, exact
    cancellation to +0, signed zeros, overflow to infinity at the tie above
    DBL_MAX, underflow ties around 2^-1075, invalid operations;
  * on the GPU, 1.3e9 structured triples against __fma_rn, __dadd_rn,
    __dmul_rn, rint and trunc."""
import ctypes
import concurrent.futures as cf
import os
import struct
import subprocess

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "softfp")


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("softfp") / "libsoftfp_check.so")
    subprocess.run(["g++", "-O2", "-shared", "-fPIC", "-ffp-contract=off", "-o", out,
                    os.path.join(HERE, "softfp_check.cc")], check=True)
    L = ctypes.CDLL(out)
    L.sfp_check.restype = ctypes.c_int64
    L.sfp_check.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    for nm in ("sfp_fma_n", "ref_fma_n"):
        getattr(L, nm).argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64]
    for nm in ("sfp_rint_n", "ref_rint_n"):
        getattr(L, nm).argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int64]
    return L


MODES = ["uniform bits", "cancellation", "subnormal", "overflow", "few-bit ties", "specials",
         "additions", "products"]


@pytest.mark.parametrize("mode", range(8), ids=MODES)
def test_structured_random(host, mode):
    per = int(os.environ.get("SOFTFP_CASES", 1 << 23))
    threads = min(8, os.cpu_count() or 1)
    bads = [np.zeros(6, np.uint64) for _ in range(threads)]
    with cf.ThreadPoolExecutor(threads) as ex:
        errs = list(ex.map(lambda t: host.sfp_check(0x5EED0000 + 97 * mode + t, per, 1 << mode,
                                                    bads[t].ctypes.data), range(threads)))
    for e, bad in zip(errs, bads):
        assert e == 0, (MODES[mode], [hex(int(v)) for v in bad])


def d2u(*vals):
    return np.array([struct.unpack("<Q", struct.pack("<d", v))[0] for v in vals], dtype=np.uint64)


def run_fma(host, a, b, c):
    n = a.size
    got, want = np.empty(n, np.uint64), np.empty(n, np.uint64)
    host.sfp_fma_n(a.ctypes.data, b.ctypes.data, c.ctypes.data, got.ctypes.data, n)
    host.ref_fma_n(a.ctypes.data, b.ctypes.data, c.ctypes.data, want.ctypes.data, n)
    return got, want


def test_directed(host):
    M, m, tiny = 1.7976931348623157e308, 2.2250738585072014e-308, 5e-324
    e = 2.0 ** -53
    cases = [
        (1.0, 1.0, e), (1.0, 1.0, 3 * e), (1.0, 1.0, -e / 2), (1.0 + 2 * e, 1.0, e),     # ties to even
        (1.0 + 2 * e, 1.0 - e, 0.0), (3.0, 1.0 / 3.0, -1.0),                            # product ties, residual
        (1.0, -1.0, 1.0), (-0.0, 1.0, -0.0), (0.0, -1.0, 0.0), (-0.0, -0.0, -0.0),       # zeros
        (2.0, -1.0, 2.0), (1e300, 1e-300, -1.0),
        (M, 2.0, -M), (M, 1.0, 2.0 ** 970), (M, 1.0, 2.0 ** 969), (M, 1.0 + 2 * e, 0.0),  # overflow edge
        (M, -1.0, -(2.0 ** 970)), (2.0 ** 1023, 2.0, 0.0),
        (tiny, 0.5, 0.0), (tiny, 1.5, 0.0), (tiny, 2.5, 0.0), (3 * tiny, 0.5, 0.0),      # underflow ties
        (m, 0.5, 0.0), (m, 1.0 - e, 0.0), (m, 1.0 - e, tiny), (m - tiny, 1.0, tiny),
        (-tiny, 0.5, 0.0), (-tiny, 0.5, -0.0), (1e-200, 1e-200, -0.0), (1e-160, 1e-160, tiny),
        (float("inf"), 0.0, 1.0), (float("inf"), 1.0, float("-inf")), (float("inf"), -2.0, float("-inf")),
        (1.0, 2.0, float("inf")), (float("nan"), 0.0, 1.0), (0.0, 0.0, float("nan")),
    ]
    a, b, c = (d2u(*[t[k] for t in cases]) for k in range(3))
    got, want = run_fma(host, a, b, c)
    for i in range(len(cases)):
        w = want[i]
        if (int(w) & 0x7FFFFFFFFFFFFFFF) > 0x7FF0000000000000:
            assert (int(got[i]) & 0x7FFFFFFFFFFFFFFF) > 0x7FF0000000000000, cases[i]
        else:
            assert got[i] == w, (cases[i], hex(int(got[i])), hex(int(w)))


def test_rint_directed(host):
    vals = [0.5, 1.5, 2.5, -0.5, -1.5, -2.5, 0.49999999999999994, -0.0, 0.0, 4503599627370495.5,
            4503599627370496.0, -4503599627370495.5, 1e300, 5e-324, -5e-324, 0.7, 1.0, 2.0 ** 52 - 1,
            float("inf"), float("-inf"), 3.5, 4.5, 1.0 - 2.0 ** -53, 2.0 ** 51 + 0.5]
    a = d2u(*vals)
    got, want = np.empty_like(a), np.empty_like(a)
    host.sfp_rint_n(a.ctypes.data, got.ctypes.data, a.size)
    host.ref_rint_n(a.ctypes.data, want.ctypes.data, a.size)
    assert np.array_equal(got, want), [(v, hex(int(g)), hex(int(w))) for v, g, w in zip(vals, got, want) if g != w]


@pytest.fixture(scope="module")
def device(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    nvcc = next((c for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc") if c and os.path.exists(c)), "nvcc")
    out = str(tmp_path_factory.mktemp("softfp_gpu") / "libsoftfp_gpu.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-fmad=false",
                    "-Xcompiler", "-fPIC", "-shared", "-o", out, os.path.join(HERE, "softfp_gpu.cu")], check=True)
    L = ctypes.CDLL(out)
    L.softfp_check_gpu.argtypes = [ctypes.c_uint64, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return L


@pytest.mark.gpu
def test_gpu_bit_exact_against_fp64_pipe(device):
    import torch
    err = torch.zeros(2, dtype=torch.int64, device="cuda")
    bad = torch.zeros(6, dtype=torch.int64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    blocks = torch.cuda.get_device_properties(0).multi_processor_count * 8
    assert device.softfp_check_gpu(0xC0FFEE, 512, blocks, 0xFF, err.data_ptr(), bad.data_ptr(), st) == 0
    torch.cuda.synchronize()
    b = [hex(int(v) & 0xFFFFFFFFFFFFFFFF) for v in bad.cpu().tolist()]
    e = err.cpu().tolist()
    assert e[1] == 0, ("non-NaN differences", e, b)
    assert e[0] == 0, ("NaN payload differences", e, b)
