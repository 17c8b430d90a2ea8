"""Build the C oracle into oracle/_build/liboracle.so.

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


if __name__ == "__main__":
    print(build(force=True))
