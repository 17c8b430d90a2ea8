#!/usr/bin/env python
"""Benchmark of the elementwise math hot path on GB300.

One step = one pass of every FP64 entry point of the library over its own
2^26-element synthetic array of the full-FP64-set workload (89% uniform over
the function's main domain, 10% log-uniform tail -- Payne-Hanek arguments
for the trig functions -- and 1% special values; inputs resident in HBM,
each array larger than L2).  Metric: Gelem/s (all elements of the step /
step time) with the per-function Gelem/s and the roofline fraction of the
dominant kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU, each rank on its own arrays
(weak scaling, no collective on the data path).  --impl reference times the
scalar C oracle on the host cores on a bounded sample of the same workload.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=1 << 26, help="elements per function")
    p.add_argument("--fns", default="", help="comma list of entry points (default: every FP64 one)")
    p.add_argument("--cpu-sample", type=int, default=1 << 18, help="oracle sample per function")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the FP32 / bf16 / f16 family measurements")
    p.add_argument("--n32", type=int, default=1 << 28, help="elements per FP32 entry point")
    p.add_argument("--n5", type=int, default=1 << 28, help="elements of the large-argument stress")
    p.add_argument("--detail", default=os.path.join(ROOT, "bench_detail.json"),
                   help="file for the per-entry-point rows and the families' tables (stdout gets "
                        "one compact line)")
    return p.parse_args()


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v, device):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip() == "Active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def default_fns(sleefcu):
    return [e for e in sleefcu.entry_points() if e.endswith("_f64")]


def build_inputs(sleefcu, names, n, rank, torch, device):
    from paper_2001_09258_gb300 import inputs as I
    host, dev = {}, {}
    for name in names:
        fn = name.split("_")[0]
        if fn in host:
            continue
        xs = [I.workload(fn, n, key=f"c2/rank{rank}", operand=0)]
        if sleefcu.FUNCS[fn] == "b":
            xs.append(I.workload(fn, n, key=f"c2/rank{rank}", operand=1))
        host[fn] = xs
        dev[fn] = [torch.from_numpy(a).to(device) for a in xs]
    return host, dev


def launch(sleefcu, name, ins, outs, stream_ptr):
    f = sleefcu.raw(name)
    kind = sleefcu.FUNCS[name.split("_")[0]]
    n = ins[0].numel()
    if kind == "u":
        rc = f(ins[0].data_ptr(), outs[0].data_ptr(), n, stream_ptr)
    elif kind == "b":
        rc = f(ins[0].data_ptr(), ins[1].data_ptr(), outs[0].data_ptr(), n, stream_ptr)
    else:
        rc = f(ins[0].data_ptr(), outs[0].data_ptr(), outs[1].data_ptr(), n, stream_ptr)
    if rc != 0:
        raise RuntimeError(f"{name}: {sleefcu.last_error()}")


E2E_CHUNK = 1 << 24          # elements per host-pipeline chunk of the end-to-end step


def csrc_sha(sources=None):
    """hash of the CUDA sources a stored ncu figure was taken on: the given
    .cu files and every shared header of csrc/ (all of csrc/ when sources is
    None); the figure is used only while they are unchanged"""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2001_09258_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        fp = os.path.join(csrc, f)
        if os.path.isfile(fp) and (sources is None or f in sources or not f.endswith(".cu")):
            h.update(f.encode())
            h.update(open(fp, "rb").read())
    return h.hexdigest()[:16]


def measured_inst_table(fname):
    """per-entry-point ncu counts from profiles/<fname> (measure/ncu_table.py):
    the entries whose kernel sources are unchanged since the capture"""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", fname)))
    except (OSError, ValueError):
        return None
    return {k: v for k, v in rec.get("per_entry_point", {}).items()
            if v.get("csrc_sha") == csrc_sha([v.get("source")])}


def measured_pipe_counts():
    """FP64 instructions per element measured by ncu for each FP64 entry point
    (profiles/fp64_inst.json), or None when the kernel sources have changed
    since the capture (the file records a hash of the CUDA sources)."""
    return measured_inst_table("fp64_inst.json")


def pipe_peak(sleefcu, torch, device, pipe="fp64"):
    """Measured FMA-pipe throughput (ops/s) with the bench's probe kernels
    (measure/probe.cu: 8 independent FMA chains per thread, 8 blocks of 256
    per SM)."""
    import measure
    props = torch.cuda.get_device_properties(device)
    blocks = props.multi_processor_count * 8
    P = measure.probe_lib()
    dt, probe, iters = ((torch.float64, P.probe_dfma, 2048) if pipe == "fp64"
                        else (torch.float32, P.probe_ffma, 16384))
    out = torch.empty(blocks * 256, dtype=dt, device=device)
    st = torch.cuda.current_stream(device)
    sp = ctypes.c_void_p(st.cuda_stream)
    for _ in range(2):
        probe(ctypes.c_void_p(out.data_ptr()), blocks, iters, sp)
    best = None
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        probe(ctypes.c_void_p(out.data_ptr()), blocks, iters, sp)
        b.record(st)
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    return blocks * 256.0 * iters * 8 / (best * 1e-3)


def fp64_pipe_peak(sleefcu, torch, device):
    return pipe_peak(sleefcu, torch, device, "fp64")


def time_calls(torch, st, fn, reps=5):
    """average ms of fn() over reps launches, CUDA events on stream st"""
    fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(reps):
        fn()
    b.record(st)
    b.synchronize()
    return a.elapsed_time(b) / reps


def extras(sleefcu, torch, device, st, sp, per_fn_f64, peaks, n32):
    """FP32 family (2^28 floats) and bf16/f16 activation forms ([8192, 28672]),
    each with its speedup over the plain FP64 / FP32 form of the function."""
    from paper_2001_09258_gb300 import inputs as I
    from measure import opcounts
    import numpy as np
    hbm = peaks.get("hbm_gbs")
    peak_fp32 = pipe_peak(sleefcu, torch, device, "fp32")
    # issue-slot bound: 4 warp instructions per clock per SM
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    issue_peak = 4.0 * sms * float(peaks.get("sm_max_mhz") or 2070.0) * 1e6
    inst32 = measured_inst_table("fp32_inst.json") or {}
    f32 = {}
    cache = {}
    for name in [e for e in sleefcu.entry_points() if e.endswith("_f32")]:
        fn = name.split("_")[0]
        kind = sleefcu.FUNCS[fn]
        if fn not in cache:                 # u10 and u35 share the workload
            cache.clear()
            torch.cuda.empty_cache()
            cache[fn] = [torch.from_numpy(I.workload(fn, n32, key="c3", operand=k, dtype=np.float32)).to(device)
                         for k in range(2 if kind == "b" else 1)]
        ins = cache[fn]
        outs = [torch.empty_like(ins[0]) for _ in range(2 if kind == "sc" else 1)]
        ms = time_calls(torch, st, lambda: launch(sleefcu, name, ins, outs, sp))
        g = n32 / (ms * 1e-3) / 1e9
        nbytes = 4 * (len(ins) + len(outs))
        acc = name.split("_")[1]
        base = per_fn_f64.get(f"{fn}_{acc}_f64")
        ope = opcounts.ops_per_element_f32(name)
        f32[name] = {"gelem_s": round(g, 2), "hbm_gbs": round(nbytes * n32 / (ms * 1e-3) / 1e9, 1),
                     "hbm_frac": round(nbytes * n32 / (ms * 1e-3) / 1e9 / hbm, 4) if hbm else None,
                     "ops_per_element": round(ope, 2),
                     "fp32_frac": round(ope * g * 1e9 / peak_fp32, 4),
                     "speedup_vs_f64": round(g / base, 2) if base else None}
        w = inst32.get(name, {}).get("warp_inst_per_element")
        if w:
            f32[name]["warp_inst_per_element"] = w
            f32[name]["issue_frac"] = round(g * 1e9 * w / issue_peak, 4)
        del outs
    low = {}
    shape = (8192, 28672)
    n16 = shape[0] * shape[1]
    for name in [e for e in sleefcu.entry_points() if e.endswith(("_bf16", "_f16"))]:
        fn, acc, fmt = name.split("_")
        h = I.activations("c3/act", shape, fmt).reshape(-1)
        x = torch.from_numpy(h.view(np.int16)).to(device)
        o = torch.empty_like(x)
        f = sleefcu.raw(name)
        ms = time_calls(torch, st, lambda: f(x.data_ptr(), o.data_ptr(), n16, sp))
        g = n16 / (ms * 1e-3) / 1e9
        base = f32.get(f"{fn}_{acc}_f32", {}).get("gelem_s")
        ope = opcounts.ops_per_element_f32(name)
        low[name] = {"gelem_s": round(g, 2), "hbm_gbs": round(4 * n16 / (ms * 1e-3) / 1e9, 1),
                     "hbm_frac": round(4 * n16 / (ms * 1e-3) / 1e9 / hbm, 4) if hbm else None,
                     "ops_per_element": round(ope, 2),
                     "fp32_frac": round(ope * g * 1e9 / peak_fp32, 4),
                     "speedup_vs_f32": round(g / base, 2) if base else None}
        del x, o
    return {"fp32_family": {"n": n32, "workload": "same mixes scaled to binary32 (trig tail to 3.4e38)",
                            "fp32_pipe_peak_tops": round(peak_fp32 / 1e12, 3),
                            "fp32_frac_note": "algorithmic binary32 ops per element (oracle counting build, "
                                              "mean over the workload) x Gelem/s / measured FFMA peak "
                                              "(measure/probe.cu probe_ffma)",
                            "issue_frac_note": "executed warp instructions per element (ncu, "
                                               "profiles/fp32_inst.json) x Gelem/s / (4 warp instructions "
                                               "per clock per SM x SMs x max SM clock); null when the "
                                               "kernels changed since the capture",
                            "entry_points": f32},
            "bf16_f16_forms": {"shape": list(shape), "inputs": "N(0,3) rounded to the 16-bit format",
                               "entry_points": low}}


def fmod_steps(sleefcu, torch, x, y, remainder, sp):
    """Per-element long-division step counts of the fmod kernel (int64 numpy
    array), from sleefcu_fmod_steps_f64 on the device operands; remainder
    divides by 2|y| where that is finite."""
    import numpy as np
    yy = y.abs()
    if remainder:
        big = float.fromhex("0x1.fffffffffffffp+1022")
        yy = torch.where(yy <= big, 2 * yy, yy)
    o = torch.empty_like(x)
    rc = sleefcu.raw("fmod_steps_f64")(x.data_ptr(), yy.data_ptr(), o.data_ptr(), x.numel(), sp)
    if rc != 0:
        raise RuntimeError(sleefcu.last_error())
    torch.cuda.synchronize()
    return o.cpu().numpy().astype(np.int64)


def stress(sleefcu, torch, device, st, sp, n5, peak_fp64):
    """Large-argument stress: 2^28 doubles with |x| log-uniform in
    [1e5, DBL_MAX] through sin/cos/tan/sincos u10 (every lane on the
    Payne-Hanek path) and fmod/remainder with the divisor log-uniform in
    [1e-300, 1e300] (up to ~42 long-division steps).  Per entry point:
    Gelem/s and the FP64-pipe roofline fraction; for fmod/remainder also
    the histogram of long-division steps per element and per warp (the
    kernel groups a tile's elements by step count, so a warp's time is
    its largest count after that grouping)."""
    from paper_2001_09258_gb300 import inputs as I
    from measure import opcounts
    import numpy as np
    out = {}
    for fn in I.STRESS_FNS:
        name = f"{fn}_u10_f64"
        hx = I.stress(fn, n5)
        hy = I.stress(fn, n5, operand=1) if fn in ("fmod", "remainder") else None
        ins = [torch.from_numpy(hx).to(device)] + ([torch.from_numpy(hy).to(device)] if hy is not None else [])
        outs = [torch.empty_like(ins[0]) for _ in range(2 if fn == "sincos" else 1)]
        ms = time_calls(torch, st, lambda: launch(sleefcu, name, ins, outs, sp), reps=3)
        it = None
        if hy is not None:
            it = fmod_steps(sleefcu, torch, ins[0], ins[1], fn == "remainder", sp)
        ops = opcounts.ops_per_launch(name, hx, hy, None if it is None else int(it.sum()))
        rec = {"gelem_s": round(n5 / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3),
               "ops_per_element": round(ops / n5, 2),
               "fp64_frac": round(ops / (ms * 1e-3) / peak_fp64, 4)}
        if it is not None:
            # the kernel groups each 1024-element tile by the class
            # ceil((ilogb x - ilogb y) / 52); a warp takes the largest count
            # of its 32 grouped elements
            ex = np.frexp(np.abs(hx))[1].astype(np.int64)
            ey = np.frexp(np.abs(hy))[1].astype(np.int64)
            cls = np.clip((ex - ey + 51) // 52, 0, 47)
            m = (n5 // 1024) * 1024
            order = np.argsort(cls[:m].reshape(-1, 1024), axis=1, kind="stable")
            grouped = np.take_along_axis(it[:m].reshape(-1, 1024), order, axis=1)
            warp = grouped.reshape(-1, 32).max(axis=1)
            rec["steps_per_element"] = {int(k): int(v) for k, v in zip(*np.unique(it, return_counts=True))}
            rec["steps_per_warp"] = {int(k): int(v) for k, v in zip(*np.unique(warp, return_counts=True))}
        out[name] = rec
        del ins, outs
        torch.cuda.empty_cache()
    return {"n": n5, "workload": "|x| log-uniform [1e5, DBL_MAX], random sign; divisor log-uniform "
                                 "[1e-300, 1e300]", "entry_points": out}


def fmod_sweep(sleefcu, torch, device, st, sp, peak_fp64, n=1 << 22):
    """Section 7.1's remainder workload: throughput of fmod u10 as the
    quotient size r grows from 1 to 1e25 (d uniform in [1, 100], dividend
    uniform in [0.95 r d, 1.05 r d]); per r the Gelem/s, the long-division
    steps per element counted by the kernel's own loop, and the FP64-pipe
    fraction.  The steps grow by one every 52 bits of quotient, so the
    throughput falls in steps."""
    from paper_2001_09258_gb300 import inputs as I
    from measure import opcounts
    pts = []
    for e in range(0, 26):
        r = 10.0 ** e
        hx, hy = I.fmod_sweep(r, n)
        ins = [torch.from_numpy(hx).to(device), torch.from_numpy(hy).to(device)]
        outs = [torch.empty_like(ins[0])]
        ms = time_calls(torch, st, lambda: launch(sleefcu, "fmod_u10_f64", ins, outs, sp), reps=5)
        steps = int(fmod_steps(sleefcu, torch, ins[0], ins[1], False, sp).sum())
        ops = opcounts.ops_per_launch("fmod_u10_f64", hx, hy, steps)
        pts.append({"r": r, "gelem_s": round(n / (ms * 1e-3) / 1e9, 3), "steps_per_element": round(steps / n, 3),
                    "fp64_frac": round(ops / (ms * 1e-3) / peak_fp64, 4)})
        del ins, outs
    return {"n": n, "workload": "d uniform [1, 100], x uniform [0.95 r d, 1.05 r d] (Section 7.1)",
            "points": pts}


def masked(sleefcu, torch, device, st, sp, n=1 << 26):
    """The masked entry points (the paper's whole-function opmask) on the C2
    arrays with a tenth and a half of the elements selected: time against
    the unmasked call, which evaluates every element."""
    from paper_2001_09258_gb300 import inputs as I
    import numpy as np
    out = {}
    for name in ("sin_u10_f64", "tgamma_u10_f64", "pow_u10_f64"):
        fn = name.split("_")[0]
        ins = [torch.from_numpy(I.workload(fn, n, key="c2/rank0", operand=k)).to(device)
               for k in range(2 if sleefcu.FUNCS[fn] == "b" else 1)]
        o = torch.empty_like(ins[0])
        full = time_calls(torch, st, lambda: launch(sleefcu, name, ins, [o], sp), reps=3)
        rec = {"unmasked_ms": round(full, 3)}
        r = (I.raw("c2/mask", n) % np.uint64(10)).astype(np.uint8)
        for label, keep in (("tenth", 1), ("half", 5)):
            m = torch.from_numpy((r < keep).astype(np.uint8)).to(device)
            y = ins[1] if len(ins) > 1 else None
            ms = time_calls(torch, st, lambda: sleefcu.call_masked(name, ins[0], m, y=y, out=o, stream=st), reps=3)
            sel = keep / 10
            rec[label] = {"ms": round(ms, 3), "time_vs_unmasked": round(ms / full, 3),
                          "selected_gelem_s": round(sel * n / (ms * 1e-3) / 1e9, 3)}
        out[name] = rec
        del ins, o
        torch.cuda.empty_cache()
    return {"n": n, "workload": "C2 arrays, mask bytes from a seeded stream", "entry_points": out}


def c99(sleefcu, torch, device, st, sp, peaks, peak_fp64, n=1 << 26):
    """The remaining C99 functions, both formats, on the C99 workload (2^26
    elements per entry point, larger than L2): Gelem/s, HBM bytes and
    algorithmic pipe operations per element, and the fraction of the
    roofline (the slower of the HBM bound and the FP-pipe bound)."""
    from paper_2001_09258_gb300 import inputs as I
    from measure import opcounts
    cnt = opcounts.table().get("c99", {})
    hbm = peaks.get("hbm_gbs")
    peak_fp32 = pipe_peak(sleefcu, torch, device, "fp32")
    out = {}
    host = {}

    def arr(name, operand):
        # functions of one input class share their arrays (inputs.c99_workload)
        fn, prec = name.split("_")[0], name.split("_")[-1]
        cls = (fn if fn in ("hypot", "sqrt") or (fn == "ldexp" and operand == 1) else "x", prec, operand)
        if cls not in host:
            host[cls] = torch.from_numpy(I.c99_workload(name, n, operand=operand)).to(device)
        return host[cls]

    for name in sleefcu.c99_entry_points():
        kd = sleefcu.C99_FUNCS[name.split("_")[0]]
        prec = name.split("_")[-1]
        x = arr(name, 0)
        y = arr(name, 1) if kd in ("b", "bi") else None
        o = torch.empty_like(x, dtype=torch.int32) if kd == "ui" else torch.empty_like(x)
        o2 = None
        if kd in ("sc", "si"):
            o2 = torch.empty_like(x, dtype=torch.int32) if kd == "si" else torch.empty_like(x)
        ms = time_calls(torch, st, lambda: sleefcu.call_c99(name, x, y, out=o, out2=o2, stream=st), reps=5)
        g = n / (ms * 1e-3) / 1e9
        nbytes = sum(t.element_size() for t in (x, y, o, o2) if t is not None)
        ops = cnt.get(name, {}).get("ops", 0.0)
        rec = {"gelem_s": round(g, 2), "bytes_per_element": nbytes, "hbm_gbs": round(g * nbytes, 1),
               "ops_per_element": ops}
        hfrac = g * nbytes / hbm if hbm else None
        pfrac = g * 1e9 * ops / (peak_fp64 if prec == "f64" else peak_fp32)
        rec["hbm_frac"] = round(hfrac, 4) if hfrac is not None else None
        rec["pipe_frac"] = round(pfrac, 4)
        rec["bound"] = "hbm" if hfrac is not None and hfrac >= pfrac else ("fp64" if prec == "f64" else "fp32")
        rec["roofline_frac"] = round(max(pfrac, hfrac or 0.0), 4)
        out[name] = rec
        del o, o2
    del host
    torch.cuda.empty_cache()
    return {"n": n, "workload": "x uniform [-100, 100] with the specials, y independent; sqrt |x|; hypot "
                                "log-uniform magnitudes; ldexp exponents uniform in [-60, 60]",
            "peaks": {"hbm_gbs": hbm, "fp64_pipe_tops": round(peak_fp64 / 1e12, 4),
                      "fp32_pipe_tops": round(peak_fp32 / 1e12, 3)},
            "entry_points": out}


def batched(sleefcu, torch, device, st, sp, narrays=4096, peak_fp64=None, peak_fp32=None, hbm=None):
    """4096 arrays, lengths log-uniform in [1, 2^20], each assigned an FP64 or
    FP32 entry point uniformly at random: one autotuned persistent launch (plain
    and graph replay) against one launch per array (plain and captured in a
    CUDA graph)."""
    import math
    import numpy as np
    from paper_2001_09258_gb300 import inputs as I
    names_all = [e for e in sleefcu.entry_points() if e.endswith(("_f64", "_f32"))]
    u = (I.raw("c4/len", narrays) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    lens = np.clip(np.floor(np.exp(u * math.log(2 ** 20))), 1, 2 ** 20).astype(np.int64)
    pick = (I.raw("c4/fn", narrays) % np.uint64(len(names_all))).astype(np.int64)
    items = []
    for k in range(narrays):
        name = names_all[pick[k]]
        fn, acc, prec = name.split("_")
        dt = np.float64 if prec == "f64" else np.float32
        n = int(lens[k])
        x = torch.from_numpy(I.workload(fn, n, key=f"c4/{k}", dtype=dt)).to(device)
        y = torch.from_numpy(I.workload(fn, n, key=f"c4/{k}", operand=1, dtype=dt)).to(device) \
            if sleefcu.FUNCS[fn] == "b" else None
        out = torch.empty_like(x)
        out2 = torch.empty_like(x) if sleefcu.FUNCS[fn] == "sc" else None
        items.append((name, x, y, out, out2))
    total = int(lens.sum())
    # algorithmic work of the mix: FP64 operations (per path class, fmod /
    # remainder with the kernel's own step counts), FP32 operations, bytes
    from measure import opcounts
    ops64 = ops32 = 0.0
    nbytes = 0
    for name, x, y, out, out2 in items:
        n = x.numel()
        nbytes += sum(t.numel() * t.element_size() for t in (x, y, out, out2) if t is not None)
        if name.endswith("_f64"):
            fn = name.split("_")[0]
            stp = None
            if fn in ("fmod", "remainder"):
                stp = int(fmod_steps(sleefcu, torch, x, y, fn == "remainder", sp).sum())
            ops64 += opcounts.ops_per_launch(name, x.cpu().numpy(), None if y is None else y.cpu().numpy(), stp)
        else:
            ops32 += opcounts.ops_per_element_f32(name) * n
    b = sleefcu.Batch(items, tune_file=os.path.join(ROOT, "paper_2001_09258_gb300", "_build", "batch_tune.jsonl"))
    cfg = b.config()
    ms_plain = time_calls(torch, st, lambda: b.launch(st), reps=5)
    ms_graph = time_calls(torch, st, lambda: b.launch(st, graph=True), reps=5)
    # the tuned shape with each vector width (why the tuner picked its width)
    vec_ms = {}
    for v in (1, 2):
        b.set_config(cfg["block"], cfg["tile"], cfg["grid_mult"], v)
        vec_ms[f"vec{v}"] = round(time_calls(torch, st, lambda: b.launch(st), reps=5), 3)
    b.set_config(cfg["block"], cfg["tile"], cfg["grid_mult"], cfg["vec"])

    def singles():
        for name, x, y, out, out2 in items:
            launch(sleefcu, name, [x] + ([y] if y is not None else []), [out] + ([out2] if out2 is not None else []), sp)
    ms_single = time_calls(torch, st, singles, reps=2)
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream(device)
    with torch.cuda.stream(cs):
        csp = ctypes.c_void_p(cs.cuda_stream)
        with torch.cuda.graph(g, stream=cs):
            for name, x, y, out, out2 in items:
                launch(sleefcu, name, [x] + ([y] if y is not None else []),
                       [out] + ([out2] if out2 is not None else []), csp)
    ms_single_graph = time_calls(torch, st, lambda: g.replay(), reps=3)
    b.close()
    # host-side latency of the allocation-free launch over the same 4096
    # items, on an idle stream and behind a 50 ms busy kernel (the call must
    # return without waiting for the stream)
    lat = {}
    arr = sleefcu._items_array(items)                 # descriptors built once: the C call alone is timed
    fst = sleefcu.lib().sleefcu_batch_launch_static
    for label, busy in (("idle_stream_us", False), ("busy_stream_us", True)):
        fst(arr, len(items), sp)
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            if busy:
                torch.cuda._sleep(100_000_000)
            t = time.perf_counter()
            rc = fst(arr, len(items), sp)
            ts.append((time.perf_counter() - t) * 1e6)
            torch.cuda.synchronize()
            if rc != 0:
                raise RuntimeError(sleefcu.last_error())
        lat[label] = round(statistics.median(ts), 1)
    gel = lambda ms: round(total / (ms * 1e-3) / 1e9, 3)
    # roofline of the mixed launch: the slowest of the three bounds at peak
    t64 = ops64 / peak_fp64 if peak_fp64 else 0.0
    t32 = ops32 / peak_fp32 if peak_fp32 else 0.0
    thbm = nbytes / (hbm * 1e9) if hbm else 0.0
    troof = max(t64, t32, thbm)
    roof = {"fp64_ops": ops64, "fp32_ops": ops32, "bytes": nbytes,
            "bound": ["fp64", "fp32", "hbm"][[t64, t32, thbm].index(troof)],
            "t_fp64_ms": round(t64 * 1e3, 3), "t_fp32_ms": round(t32 * 1e3, 3), "t_hbm_ms": round(thbm * 1e3, 3),
            "frac": round(troof / (ms_graph * 1e-3), 4) if troof else None}
    return {"arrays": narrays, "elements": total, "entry_points": len(names_all), "config": cfg,
            "roofline": roof, "vec_width_ms": vec_ms, "fp_frac": roof["frac"],
            "batched_ms": round(ms_plain, 3), "batched_graph_ms": round(ms_graph, 3),
            "single_launches_ms": round(ms_single, 3), "single_launches_graph_ms": round(ms_single_graph, 3),
            "batched_gelem_s": gel(ms_plain), "batched_graph_gelem_s": gel(ms_graph),
            "single_launches_gelem_s": gel(ms_single), "single_launches_graph_gelem_s": gel(ms_single_graph),
            "speedup_vs_single_launches": round(ms_single / ms_graph, 2),
            "speedup_vs_single_launch_graph": round(ms_single_graph / ms_graph, 2),
            "static_launch_host_latency": lat}


def cpu_baseline(names, n_sample, rank, threads=None):
    """The oracle as it stands, on the host cores (all of them unless
    `threads` is given), on a bounded sample."""
    import oracle
    from paper_2001_09258_gb300 import inputs as I
    threads = threads or oracle.default_threads()
    total_el, total_s = 0, 0.0
    for name in names:
        fn = name.split("_")[0]
        x = I.workload(fn, n_sample, key=f"c2/rank{rank}", operand=0)
        y = I.workload(fn, n_sample, key=f"c2/rank{rank}", operand=1) if oracle.kind(name) in (2, 12) else None
        oracle.apply(name, x[:1024], None if y is None else y[:1024], nthreads=threads)
        t = time.perf_counter()
        oracle.apply(name, x, y, nthreads=threads)
        total_s += time.perf_counter() - t
        total_el += n_sample
    return total_el, total_s, threads


def run_reference(args, ws, rank):
    names = args.fns.split(",") if args.fns else None
    import paper_2001_09258_gb300 as sleefcu
    names = names or default_fns(sleefcu)
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(names, max(1024, args.cpu_sample // 16), 0)
    times = []
    el = 0
    thr = 1
    for _ in range(args.steps):
        e, s, thr = cpu_baseline(names, args.cpu_sample, 0)
        times.append(s)
        el = e
    t = sum(times)
    val = el * args.steps / t / 1e9
    line = {
        "impl": "reference", "metric": "Gelem/s (full FP64 C99 set, u10+u35) at max-ULP <=1.0/3.5",
        "value": round(val, 6), "unit": "Gelem/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"full FP64 set mixed workload, oracle sample of {args.cpu_sample} "
                               f"elements per entry point", "entry_points": names},
        "cpu_baseline": {"value": round(val, 6), "unit": "Gelem/s", "cores": thr, "kind": "oracle",
                         "sample": f"{args.cpu_sample} elements per entry point of the same workload"},
        "e2e": {"value": round(val, 6), "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    ws, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    import paper_2001_09258_gb300 as sleefcu
    from measure import opcounts
    device = torch.device(f"cuda:{local}")
    torch.cuda.set_device(device)
    names = args.fns.split(",") if args.fns else default_fns(sleefcu)
    n = args.n
    host, dev = build_inputs(sleefcu, names, n, rank, torch, device)
    outs = {}
    for name in names:
        fn = name.split("_")[0]
        k = 2 if sleefcu.FUNCS[fn] == "sc" else 1
        outs[name] = [torch.empty(n, dtype=torch.float64, device=device) for _ in range(k)]
    st = torch.cuda.current_stream(device)
    sp = ctypes.c_void_p(st.cuda_stream)

    def step(evs=None):
        for i, name in enumerate(names):
            if evs is not None:
                evs[i].record(st)
            launch(sleefcu, name, dev[name.split("_")[0]], outs[name], sp)
        if evs is not None:
            evs[len(names)].record(st)

    for _ in range(max(args.warmup, 3) if args.warmup >= 3 else 3):
        step()
    torch.cuda.synchronize()
    peak_fp64 = fp64_pipe_peak(sleefcu, torch, device) if rank == 0 else None

    per_fn_ms = {name: [] for name in names}
    with Clocks(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        allev = []
        t0.record(st)
        for _ in range(args.steps):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
            step(evs)
            allev.append(evs)
        t1.record(st)
        torch.cuda.synchronize()
        barrier(ws)
    ms = t0.elapsed_time(t1)
    for evs in allev:
        for i, name in enumerate(names):
            per_fn_ms[name].append(evs[i].elapsed_time(evs[i + 1]))
    ms_max = allmax(ws, ms, device)
    total_el = n * len(names) * args.steps * ws
    value = total_el / (ms_max * 1e-3) / 1e9

    # e2e: the library's host-memory entry point (sleefcu_eval_host_many, one
    # call per step over all 60 arrays) on pinned host arrays: every step
    # copies each input in, evaluates and copies each result out, overlapped
    # chunk by chunk inside the library; host clock around whole steps (the
    # call returns with every result in host memory)
    e2e = None
    if not args.no_e2e:
        hin = {fn: [torch.from_numpy(a).pin_memory() for a in xs] for fn, xs in host.items()}
        hout = {name: [torch.empty(n, dtype=torch.float64).pin_memory() for _ in outs[name]] for name in names}
        h2d = sum(sum(a.numel() * 8 for a in hin[nm.split("_")[0]]) for nm in names)
        d2h = sum(sum(a.numel() * 8 for a in hout[nm]) for nm in names)
        hin_np = {fn: [t.numpy() for t in ts] for fn, ts in hin.items()}
        hout_np = {nm: [t.numpy() for t in ts] for nm, ts in hout.items()}

        e2e_items = []
        for name in names:
            xs, os_ = hin_np[name.split("_")[0]], hout_np[name]
            e2e_items.append((name, xs[0], xs[1] if len(xs) > 1 else None, os_[0], os_[1] if len(os_) > 1 else None))

        def e2e_step():
            # 2^24-element chunks: whole multiples of the sorted kernels' tiles
            # over the grid, so a chunk's last wave of tiles is a small share
            sleefcu.eval_host_many(e2e_items, chunk=E2E_CHUNK)
        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - t0) * 1e3
        barrier(ws)
        e_ms = allmax(ws, e_ms, device)
        e2e = {"value": round(total_el / (e_ms * 1e-3) / 1e9, 4), "unit": "Gelem/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "sleefcu_eval_host_many (one call per step over the 60 pinned host arrays, "
                      "up to 6 chunks of 2^24 in flight)",
               "timer": "host clock around whole steps"}

    if rank != 0:
        return
    avg = {name: statistics.mean(v) for name, v in per_fn_ms.items()}
    per_fn = {name: round(n / (avg[name] * 1e-3) / 1e9, 3) for name in names}
    # per-entry-point roofline: algorithmic FP64 ops of each launch's path mix
    per_roof = {}
    pipe_counts = measured_pipe_counts()
    for name in names:
        fn = name.split("_")[0]
        hx = host[fn]
        st_ = None
        if fn in ("fmod", "remainder"):
            st_ = int(fmod_steps(sleefcu, torch, dev[fn][0], dev[fn][1], fn == "remainder", sp).sum())
        o = opcounts.ops_per_launch(name, hx[0], hx[1] if len(hx) > 1 else None, st_)
        dv, sq = opcounts.div_sqrt_per_launch(name, hx[0], hx[1] if len(hx) > 1 else None, st_)
        mu, rn = opcounts.mul_rnd_per_launch(name, hx[0], hx[1] if len(hx) > 1 else None, st_)
        # the operations left on the FP64 pipe: multiplications and roundings
        # run in software on the integer pipe (except where a translation
        # unit keeps them on the FP64 pipe, opcounts.HW_MUL_FUNCS)
        pipe_ops = o if fn in opcounts.HW_MUL_FUNCS else o - mu - rn
        per_roof[name] = {"ops_per_element": round(o / n, 2),
                          "div_per_element": round(dv / n, 3), "sqrt_per_element": round(sq / n, 3),
                          "mul_rnd_per_element": round((mu + rn) / n, 3),
                          "fp64_frac": round(o / (avg[name] * 1e-3) / peak_fp64, 4),
                          "fp64_pipe_frac": round(pipe_ops / (avg[name] * 1e-3) / peak_fp64, 4)}
        if pipe_counts and name in pipe_counts:
            per_roof[name]["fp64_inst_per_element"] = pipe_counts[name]["fp64_inst"]
    ext = None
    if not args.no_extras:
        del dev, outs
        torch.cuda.empty_cache()
        ext = extras(sleefcu, torch, device, st, sp, per_fn, measured_peaks(), args.n32)
        torch.cuda.empty_cache()
        ext["batched"] = batched(sleefcu, torch, device, st, sp, peak_fp64=peak_fp64,
                                 peak_fp32=ext["fp32_family"]["fp32_pipe_peak_tops"] * 1e12,
                                 hbm=measured_peaks().get("hbm_gbs"))
        torch.cuda.empty_cache()
        ext["stress"] = stress(sleefcu, torch, device, st, sp, args.n5, peak_fp64)
        torch.cuda.empty_cache()
        ext["fmod_sweep"] = fmod_sweep(sleefcu, torch, device, st, sp, peak_fp64)
        torch.cuda.empty_cache()
        ext["masked"] = masked(sleefcu, torch, device, st, sp)
        torch.cuda.empty_cache()
        ext["c99"] = c99(sleefcu, torch, device, st, sp, measured_peaks(), peak_fp64)
    dom = max(names, key=lambda nm: avg[nm])
    hx = host[dom.split("_")[0]]
    steps = None
    if dom.split("_")[0] in ("fmod", "remainder"):
        dx = [torch.from_numpy(a).to(device) for a in hx]
        steps = int(fmod_steps(sleefcu, torch, dx[0], dx[1], dom.startswith("remainder"), sp).sum())
        del dx
    ops = opcounts.ops_per_launch(dom, hx[0], hx[1] if len(hx) > 1 else None, steps)
    dv, sq = opcounts.div_sqrt_per_launch(dom, hx[0], hx[1] if len(hx) > 1 else None, steps)
    achieved = ops / (avg[dom] * 1e-3)
    roof = {"kernel": dom, "bound": "alu", "pipe": "fp64",
            "achieved": round(achieved / 1e12, 5), "peak": round(peak_fp64 / 1e12, 5),
            "unit": "Tops/s (FP64 pipe: add, mul, fma, rint, div, sqrt each one op)",
            "frac": round(achieved / peak_fp64, 4),
            "peak_source": "measured in this run with measure/probe.cu probe_dfma (8 independent FMA chains "
                           "per thread, all SMs)",
            "ops_per_element": round(ops / n, 3), "div_per_element": round(dv / n, 3),
            "sqrt_per_element": round(sq / n, 3),
            "ops_source": "oracle counting build, per path class (measure/opcounts.json), "
                          "weighted by this launch's path mix",
            "fp64_inst_per_element": (pipe_counts or {}).get(dom, {}).get("fp64_inst"),
            "fp64_inst_source": "ncu sm__sass_thread_inst_executed_op_fp64_pred_on on the C2 mix "
                                "(profiles/fp64_inst.json; null when the kernels changed since)",
            "traffic": None}
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            tr = json.load(open(prof)).get(dom)
            if tr and tr.get("csrc_sha") == csrc_sha([tr["source"]]):   # null once its sources changed
                roof["traffic"] = tr["bytes_per_launch"] * n / tr["n"]
        except (OSError, ValueError, KeyError):
            pass
    cpu = None
    if not args.no_cpu_baseline:
        el, s, thr = cpu_baseline(names, args.cpu_sample, rank)
        el1, s1, _ = cpu_baseline(names, max(1024, args.cpu_sample // 16), rank, threads=1)
        cpu = {"value": round(el / s / 1e9, 6), "unit": "Gelem/s", "cores": thr, "kind": "oracle",
               "sample": f"{args.cpu_sample} elements of each entry point's workload array "
                         f"({len(names)} entry points)",
               "single_core_value": round(el1 / s1 / 1e9, 6),
               "single_core_sample": f"{max(1024, args.cpu_sample // 16)} elements per entry point, one thread"}
    detail = {
        "metric": "Gelem/s (full FP64 C99 set, u10+u35) at max-ULP <=1.0/3.5",
        "value": round(value, 4), "unit": "Gelem/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "full FP64 C99 set, mixed 89% main domain / 10% log-uniform tail "
                               "(trig: Payne-Hanek arguments 1e5..1e300) / 1% specials",
                   "n_per_function": n, "entry_points": names, "l2": "inputs larger than L2 (no flush)"},
        "per_function_gelem_s": per_fn,
        "per_function_roofline": per_roof,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": len(names) * args.steps,
        "forms": ext,
        "clocks": clk.summary(),
    }
    path = os.path.abspath(args.detail)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(detail, f, indent=1)
    print(json.dumps(headline(detail, path)))


def _spread(vals):
    vals = sorted(v for v in vals if v is not None)
    if not vals:
        return None
    return {"min": vals[0], "median": round(statistics.median(vals), 4), "max": vals[-1], "count": len(vals)}


def headline(d, detail_path):
    """The one JSON line bench.py prints: the contract's keys, the dominant
    kernel's roofline, the CPU baseline, the end-to-end figure, the clocks
    and one summary per family; the per-entry-point rows and the families'
    tables stay in the detail file."""
    roof = {k: d["roofline"][k] for k in ("kernel", "bound", "pipe", "achieved", "peak", "frac",
                                          "ops_per_element", "div_per_element", "fp64_inst_per_element",
                                          "traffic")}
    roof["unit"] = "Tops/s"
    roof["unit_note"] = "FP64 pipe ops: add, mul, fma, rint, div, sqrt one each (oracle counting build)"
    roof["peak_source"] = "measured DFMA peak, this run (measure/probe.cu)"
    fr = [r["fp64_frac"] for r in d["per_function_roofline"].values()]
    pf = [r["fp64_pipe_frac"] for r in d["per_function_roofline"].values()]
    summ = {"fp64_entry_points": {"gelem_s": _spread(list(d["per_function_gelem_s"].values())),
                                  "roofline_frac": _spread(fr),
                                  "at_or_above_0.8": sum(1 for v in fr if v >= 0.8),
                                  "pipe_only_frac": _spread(pf),
                                  "frac_note": "roofline_frac: all algorithmic FP64 operations against the DFMA "
                                               "peak (can pass 1: multiplications and roundings run on the "
                                               "integer pipe); pipe_only_frac: the operations left on the FP64 "
                                               "pipe against the same peak"}}
    ext = d.get("forms") or {}
    if ext:
        f32 = ext["fp32_family"]["entry_points"]
        low = ext["bf16_f16_forms"]["entry_points"]
        summ["fp32_family"] = {"gelem_s": _spread([r["gelem_s"] for r in f32.values()]),
                               "hbm_frac": _spread([r["hbm_frac"] for r in f32.values()]),
                               "issue_frac": _spread([r.get("issue_frac") for r in f32.values()]),
                               "speedup_vs_f64": _spread([r["speedup_vs_f64"] for r in f32.values()])}
        summ["bf16_f16_forms"] = {"gelem_s": _spread([r["gelem_s"] for r in low.values()]),
                                  "hbm_frac": _spread([r["hbm_frac"] for r in low.values()]),
                                  "speedup_vs_f32": _spread([r["speedup_vs_f32"] for r in low.values()])}
        b = ext["batched"]
        summ["batched"] = {k: b.get(k) for k in ("batched_graph_gelem_s", "speedup_vs_single_launches",
                                                 "speedup_vs_single_launch_graph", "fp_frac")}
        stv = ext["stress"]["entry_points"]
        summ["stress"] = {"gelem_s": _spread([r["gelem_s"] for r in stv.values()]),
                          "fp64_frac": _spread([r["fp64_frac"] for r in stv.values()])}
        summ["c99"] = {"roofline_frac": _spread([r["roofline_frac"] for r in ext["c99"]["entry_points"].values()])}
    cfg = dict(d["config"])
    cfg["entry_points"] = len(cfg["entry_points"])
    out = {k: d[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                             "higher_is_better", "scaling", "vs_baseline", "dtype", "data")}
    out.update({"config": cfg, "roofline": roof, "cpu_baseline": d["cpu_baseline"], "e2e": d["e2e"],
                "gpu_launches": d["gpu_launches"], "clocks": d["clocks"], "summary": summ,
                "detail": os.path.relpath(detail_path, ROOT) if detail_path.startswith(ROOT) else detail_path})
    return out


if __name__ == "__main__":
    main()
