"""Turn an ncu CSV of `measure/launch_each.py` (one launch per entry point,
in its --list order) into the per-entry-point table bench.py reads:

    python measure/ncu_table.py --family f32 --n 4194304 launches.csv > profiles/fp32_inst.json
    python measure/ncu_table.py --family f64 --n 33554432 captures_dir > profiles/fp64_inst.json

For each entry point: executed warp instructions per element
(smsp__inst_executed.sum / n) and, when captured, FP64 thread instructions
per element (sm__sass_thread_inst_executed_op_fp64_pred_on.sum / n).  The
table records, per entry point, a hash of the kernel's .cu file and the
shared headers; bench.py ignores an entry once they change.  The hashes are
those of the sources the captures ran: write them beside the captures, on
the machine that runs them, before capturing,

    python measure/ncu_table.py --stamp captures_dir

and the table takes them from captures_dir/csrc_sha.json (or from the
csrc_sha.json beside a single CSV); --assume-local-sources takes the local
sources' hashes instead, for captures made from the local tree unchanged."""
import argparse
import csv
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "measure"))


SOURCES = {"f32": ["trig_f32.cu", "explog_f32.cu", "derived_f32.cu"],
           "f64": ["trig_f64.cu", "explog_f64.cu", "invtrig_f64.cu", "fmod_f64.cu", "derived_f64.cu",
                   "gamma_f64.cu", "pow_f64.cu"]}


def source_of(name):
    """the .cu file that holds an entry point's kernel"""
    fn, prec = name.split("_")[0], name.split("_")[-1]
    if prec == "f64":
        if fn in ("sin", "cos", "tan", "sincos"):
            return "trig_f64.cu"
        if fn in ("asin", "acos", "atan", "atan2"):
            return "invtrig_f64.cu"
        if fn in ("exp", "log"):
            return "explog_f64.cu"
        if fn == "pow":
            return "pow_f64.cu"
        if fn in ("fmod", "remainder"):
            return "fmod_f64.cu"
        if fn in ("tgamma", "lgamma"):
            return "gamma_f64.cu"
        return "derived_f64.cu"
    if fn in ("sin", "cos", "tan", "sincos"):
        return "trig_f32.cu"
    if fn in ("exp", "log", "log1p", "tanh", "erf"):
        return "explog_f32.cu"
    return "derived_f32.cu"


def csrc_sha(sources):
    """the hash bench.py checks: the family's .cu files and every shared header"""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2001_09258_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        fp = os.path.join(csrc, f)
        if os.path.isfile(fp) and (f in sources or not f.endswith(".cu")):
            h.update(f.encode())
            h.update(open(fp, "rb").read())
    return h.hexdigest()[:16]


def stamp(path):
    """record the hashes of the sources as they are now (before a capture)"""
    os.makedirs(path, exist_ok=True)
    srcs = sorted(set(SOURCES["f32"]) | set(SOURCES["f64"]))
    out = {src: csrc_sha([src]) for src in srcs}
    out.update({f"family:{k}": csrc_sha(v) for k, v in SOURCES.items()})
    with open(os.path.join(path, "csrc_sha.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


def main():
    if len(sys.argv) == 3 and sys.argv[1] == "--stamp":
        stamp(sys.argv[2])
        return
    p = argparse.ArgumentParser()
    p.add_argument("--family", choices=["f64", "f32"], required=True)
    p.add_argument("--n", type=int, required=True)
    p.add_argument("--assume-local-sources", action="store_true",
                   help="hash the local sources (no csrc_sha.json was written at capture time)")
    p.add_argument("csv", help="one CSV of every launch in --list order, or a directory of <entry point>.csv "
                                "files with one launch each")
    a = p.parse_args()
    sdir = a.csv if os.path.isdir(a.csv) else os.path.dirname(os.path.abspath(a.csv))
    spath = os.path.join(sdir, "csrc_sha.json")
    if os.path.exists(spath):
        with open(spath) as f:
            stamped = json.load(f)
        sha_of = lambda src: stamped[src]
        family_sha = stamped[f"family:{a.family}"]
    elif a.assume_local_sources:
        sha_of = lambda src: csrc_sha([src])
        family_sha = csrc_sha(SOURCES[a.family])
    else:
        raise SystemExit(f"{spath} missing: run `ncu_table.py --stamp` where the captures run, "
                         "or pass --assume-local-sources")
    from launch_each import names
    order = names(a.family)

    def read(path):
        out = {}
        with open(path) as f:
            lines = [l for l in f if l.startswith('"')]
        for r in csv.DictReader(lines):
            out.setdefault(int(r["ID"]), {})[r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
            out[int(r["ID"])]["kernel"] = r["Kernel Name"]
        return out

    if os.path.isdir(a.csv):
        rows = {i: read(os.path.join(a.csv, nm + ".csv"))[0] for i, nm in enumerate(order)}
    else:
        rows = read(a.csv)
    if len(rows) != len(order):
        raise SystemExit(f"{len(rows)} launches in {a.csv}, {len(order)} entry points")
    out = {}
    for i, nm in enumerate(order):
        m = rows[i]
        e = {"kernel": m["kernel"].split("(")[0], "time_ns": m.get("gpu__time_duration.sum")}
        if "smsp__inst_executed.sum" in m:
            e["warp_inst_per_element"] = round(m["smsp__inst_executed.sum"] / a.n, 4)
        if "sm__sass_thread_inst_executed_op_fp64_pred_on.sum" in m:
            e["fp64_inst"] = round(m["sm__sass_thread_inst_executed_op_fp64_pred_on.sum"] / a.n, 3)
        e["source"] = source_of(nm)
        e["csrc_sha"] = sha_of(e["source"])
        out[nm] = e
    json.dump({"csrc_sha": family_sha, "sources": SOURCES[a.family], "n": a.n, "family": a.family,
               "command": f"python measure/launch_each.py --family {a.family} --n {a.n} [--only NAME] under "
                          "ncu --metrics <the metrics above>,gpu__time_duration.sum --clock-control none --csv",
               "per_entry_point": out}, sys.stdout, indent=1, sort_keys=True)
    print()


if __name__ == "__main__":
    main()
