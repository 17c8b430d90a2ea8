"""Launch every entry point of one family once, in a fixed order, on a sample
of its benchmark workload (for per-kernel ncu captures: `ncu -s K -c 1`
profiles exactly the K-th launch).

    python measure/launch_each.py --family f32 --n 4194304 [--list] [--only NAME]

family: f64 (the full FP64 set, C2 mixes) or f32 (the binary32 family, C3
mixes).  --list prints "index name" for every launch and exits without a
GPU.  One launch per entry point: the sorted / deferred / plain kernel the
entry point itself chooses for a 16-byte-aligned array of n elements.
"""
import argparse
import ctypes
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def names(family):
    import paper_2001_09258_gb300 as sleefcu
    return [e for e in sleefcu.entry_points() if e.endswith("_" + family)]


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--family", choices=["f64", "f32"], default="f32")
    p.add_argument("--n", type=int, default=1 << 22)
    p.add_argument("--list", action="store_true")
    p.add_argument("--only", default="", help="launch this one entry point")
    a = p.parse_args()
    order = [a.only] if a.only else names(a.family)
    if a.list:
        for i, nm in enumerate(order):
            print(i, nm)
        return
    import numpy as np
    import torch
    import paper_2001_09258_gb300 as sleefcu
    from paper_2001_09258_gb300 import inputs as I
    dt = np.float64 if a.family == "f64" else np.float32
    key = "c2/rank0" if a.family == "f64" else "c3"
    st = torch.cuda.current_stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    for nm in order:
        fn = nm.split("_")[0]
        kind = sleefcu.FUNCS[fn]
        ins = [torch.from_numpy(I.workload(fn, a.n, key=key, operand=k, dtype=dt)).cuda()
               for k in range(2 if kind == "b" else 1)]
        outs = [torch.empty_like(ins[0]) for _ in range(2 if kind == "sc" else 1)]
        f = sleefcu.raw(nm)
        args = [t.data_ptr() for t in ins + outs] + [a.n, sp]
        rc = f(*args)
        if rc != 0:
            raise RuntimeError(f"{nm}: {sleefcu.last_error()}")
        torch.cuda.synchronize()
    print(f"launched {len(order)} entry points of family {a.family}, n = {a.n}")


if __name__ == "__main__":
    main()
