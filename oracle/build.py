"""Build the C oracle into oracle/_build/liboracle.so, and its counting
build (the same sources compiled as C++ with oracle/counting/opcount.hpp forced
in) into oracle/_build/liboracle_count.so.

Test infrastructure: only tests/, the smoke check and the CPU-baseline leg of
the benchmark may use anything under oracle/.

Flags: -O2 -ffp-contract=off -fno-fast-math (no fused multiply-add unless
fma() is written; Section 4's bit-consistent build disables contraction),
plus -mfma -msse4.1 on x86-64 so that fma() and rint() are single
instructions.  No -march=native: the same source builds on x86-64 and Arm.
"""
import glob
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build", "liboracle.so")
OUT_COUNT = os.path.join(HERE, "_build", "liboracle_count.so")


def flags():
    f = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
         "-fno-math-errno", "-Wall", "-Wno-unused-function"]
    if platform.machine() in ("x86_64", "AMD64"):
        f += ["-mfma", "-msse4.1"]
    return f


def build(force=False):
    srcs = sorted(glob.glob(os.path.join(HERE, "src", "*.c")))
    deps = srcs + sorted(glob.glob(os.path.join(HERE, "src", "*.h"))) + \
        sorted(glob.glob(os.path.join(HERE, "src", "*.inc"))) + [os.path.abspath(__file__)]
    if not force and os.path.exists(OUT):
        t = os.path.getmtime(OUT)
        if all(os.path.getmtime(d) <= t for d in deps):
            return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = ["gcc"] + flags() + ["-I", os.path.join(HERE, "src")] + srcs + ["-o", tmp, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build_count(force=False):
    """Counting build: every translation unit of the oracle except the C
    registry (api.c) is compiled as C++17 with the counting header, in
    parallel, and linked with oracle/counting/count_api.cc."""
    from concurrent.futures import ThreadPoolExecutor
    srcs = [s for s in sorted(glob.glob(os.path.join(HERE, "src", "*.c")))
            if os.path.basename(s) != "api.c"]
    hdr = os.path.join(HERE, "counting", "opcount.hpp")
    api = os.path.join(HERE, "counting", "count_api.cc")
    deps = srcs + [hdr, api, os.path.abspath(__file__)] + \
        sorted(glob.glob(os.path.join(HERE, "src", "*.h"))) + sorted(glob.glob(os.path.join(HERE, "src", "*.inc")))
    if not force and not _stale(OUT_COUNT, deps):
        return OUT_COUNT
    odir = os.path.join(HERE, "_build", f"count_obj{os.getpid()}")
    os.makedirs(odir, exist_ok=True)
    cflags = ["g++", "-x", "c++", "-std=gnu++17", "-O1", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
              "-fno-math-errno", "-w", "-include", hdr, "-I", os.path.join(HERE, "src")]
    objs = []

    def compile_one(src):
        obj = os.path.join(odir, os.path.basename(src) + ".o")
        subprocess.run(cflags + ["-c", src, "-o", obj], check=True)
        return obj

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, srcs + [api]))
    tmp = OUT_COUNT + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-shared", "-o", tmp] + objs + ["-lm", "-lpthread"], check=True)
    os.replace(tmp, OUT_COUNT)
    for o in objs:
        os.remove(o)
    os.rmdir(odir)
    return OUT_COUNT


if __name__ == "__main__":
    print(build(force=True))
    print(build_count(force=True))
