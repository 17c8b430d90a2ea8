"""Measurement support for bench.py (not part of the library).

* opcounts: algorithmic operation counts per element (the roofline's unit),
  read from opcounts.json, which the oracle's counting build writes;
* probe library (probe.cu -> _build/libsleefcu_probe.so): FMA-chain kernels
  that measure the FP64 and FP32 pipe peaks the roofline is quoted against.
"""
import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
PROBE_LIB = os.path.join(BUILD, "libsleefcu_probe.so")
_probe = None


def build(force=False):
    """Compile probe.cu for sm_103a into _build/libsleefcu_probe.so."""
    src = os.path.join(HERE, "probe.cu")
    if not force and os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(src):
        return PROBE_LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = next((c for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc") if c and os.path.exists(c)), "nvcc")
    tmp = PROBE_LIB + f".tmp{os.getpid()}"
    cmd = [nv, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false", "-shared",
           "-Xcompiler", "-fPIC", src, "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def probe_lib():
    global _probe
    if _probe is None:
        build()
        L = ctypes.CDLL(PROBE_LIB)
        for nm in ("probe_dfma", "probe_ffma"):
            getattr(L, nm).restype = ctypes.c_int
            getattr(L, nm).argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        _probe = L
    return _probe
