"""Build libsleefcu.so and libsleefcu_checked.so in-tree
(paper_2001_09258_gb300/_build/).

nvcc for sm_103a only, one object per .cu and build compiled in parallel,
then one shared link per library.  Floating-point flags: -fmad=false (no contraction: a multiply
is fused into an add only where __fma_rn is written, as in the paper's
bit-consistent build, Section 4), IEEE division and square root, no
flush-to-zero, no fast math.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(BUILD, "libsleefcu.so")
LIB_CHECKED = os.path.join(BUILD, "libsleefcu_checked.so")
ROOT = os.path.dirname(HERE)

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
    "--expt-relaxed-constexpr",
]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps():
    return (sorted(glob.glob(os.path.join(CSRC, "*"))) +
            [os.path.join(ROOT, "include", "sleefcu.h"), os.path.abspath(__file__)])


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _link(objs, lib):
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force=False, verbose=False, extra_flags=()):
    """Build libsleefcu.so and the checked build libsleefcu_checked.so (the
    same sources with -DSLEEFCU_CHECKED: device-pointer checks before every
    launch and a device error word for clamped table indices).  Both sets of
    objects compile in one pool, largest translation unit first."""
    deps = _deps()
    if not force and not _stale(LIB, deps) and not _stale(LIB_CHECKED, deps):
        return LIB
    os.makedirs(GEN, exist_ok=True)
    os.makedirs(os.path.join(BUILD, "checked"), exist_ok=True)
    phtab = os.path.join(GEN, "sleefcu_phtab.inc")
    gen = os.path.join(CSRC, "gen_phtab.py")
    if force or _stale(phtab, [gen]):
        subprocess.run([sys.executable, gen, phtab], check=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")), key=lambda f: -os.path.getsize(f))
    srcs.sort(key=lambda f: os.path.basename(f) != "batch.cu")     # the longest compile first
    flags = NVCC_FLAGS + ["-I", CSRC, "-I", GEN, "-I", os.path.join(ROOT, "include")] + list(extra_flags)
    jobs = [(src, False) for src in srcs] + [(src, True) for src in srcs]
    jobs.sort(key=lambda j: os.path.basename(j[0]) != "batch.cu")

    def compile_one(job):
        src, checked = job
        obj = os.path.join(BUILD, "checked" if checked else "", os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc()] + flags + (["-DSLEEFCU_CHECKED"] if checked else []) + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}{' (checked)' if checked else ''}:\n{r.stdout}\n{r.stderr}")
        return obj, checked, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(2, min(len(jobs), os.cpu_count() or 8))) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose:
        for _, _, err in results:
            if err.strip():
                print(err)
    _link([o for o, c, _ in results if not c], LIB)
    _link([o for o, c, _ in results if c], LIB_CHECKED)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []))
