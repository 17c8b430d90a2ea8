"""The stored ncu tables the bench reads (CPU only).

measure/ncu_table.py turns per-entry-point ncu captures into
profiles/fp64_inst.json and profiles/fp32_inst.json, and bench.py uses an
entry only while the kernel's sources hash as they did when the capture ran.
These tests pin that bookkeeping: the hashes come from the machine that ran
the captures (a csrc_sha.json written before capturing), a table is not
built without them unless asked, and a stored entry whose source changed is
dropped by the bench.
"""
import csv
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "measure"))
import ncu_table  # noqa: E402
import launch_each  # noqa: E402

HEADER = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
          "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def _write_capture(path, kernel, metrics):
    with open(path, "w", newline="") as f:
        f.write("==PROF== a line ncu writes before the table\n")
        w = csv.writer(f, quoting=csv.QUOTE_ALL)
        w.writerow(HEADER)
        for name, value in metrics.items():
            w.writerow(["0", "1", "python3", "127.0.0.1", kernel + "(const float *, float *, unsigned long)",
                        "1", "7", "(256, 1, 1)", "(1216, 1, 1)", "0", "10.3", "Command line profiler metrics",
                        name, "", f"{value:,}"])


def _captures(tmp_path, n):
    d = tmp_path / "caps"
    d.mkdir()
    for i, nm in enumerate(launch_each.names("f32")):
        _write_capture(d / f"{nm}.csv", f"void k_unary32<F{i}, 1>",
                       {"smsp__inst_executed.sum": (i + 1) * n, "gpu__time_duration.sum": 1000 + i})
    return d


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "measure", "ncu_table.py"), *map(str, args)],
                          capture_output=True, text=True)


def test_stamp_records_the_hashes_of_the_sources_as_they_are(tmp_path):
    ncu_table.stamp(str(tmp_path))
    with open(tmp_path / "csrc_sha.json") as f:
        s = json.load(f)
    for fam, srcs in ncu_table.SOURCES.items():
        assert s[f"family:{fam}"] == ncu_table.csrc_sha(srcs)
        for src in srcs:
            assert s[src] == ncu_table.csrc_sha([src])


def test_table_takes_the_stamped_hashes(tmp_path):
    n = 1 << 10
    d = _captures(tmp_path, n)
    stamped = {src: f"{i:016x}" for i, src in enumerate(sorted(set(sum(ncu_table.SOURCES.values(), []))))}
    stamped.update({f"family:{k}": "f" * 16 for k in ncu_table.SOURCES})
    with open(d / "csrc_sha.json", "w") as f:
        json.dump(stamped, f)
    r = _run("--family", "f32", "--n", n, d)
    assert r.returncode == 0, r.stderr
    t = json.loads(r.stdout)
    assert t["csrc_sha"] == "f" * 16
    for i, nm in enumerate(launch_each.names("f32")):
        e = t["per_entry_point"][nm]
        assert e["csrc_sha"] == stamped[e["source"]]
        assert e["warp_inst_per_element"] == i + 1
        assert e["kernel"] == f"void k_unary32<F{i}, 1>"


def test_table_refuses_captures_without_hashes(tmp_path):
    d = _captures(tmp_path, 1 << 10)
    r = _run("--family", "f32", "--n", 1 << 10, d)
    assert r.returncode != 0 and "csrc_sha.json" in (r.stderr + r.stdout)
    r = _run("--family", "f32", "--n", 1 << 10, "--assume-local-sources", d)
    assert r.returncode == 0, r.stderr
    t = json.loads(r.stdout)
    nm = launch_each.names("f32")[0]
    assert t["per_entry_point"][nm]["csrc_sha"] == ncu_table.csrc_sha([ncu_table.source_of(nm)])


@pytest.mark.parametrize("fname", ["fp64_inst.json", "fp32_inst.json"])
def test_bench_drops_entries_whose_source_changed(tmp_path, monkeypatch, fname):
    import bench
    with open(os.path.join(ROOT, "profiles", fname)) as f:
        t = json.load(f)
    first = sorted(t["per_entry_point"])[0]
    t["per_entry_point"][first]["csrc_sha"] = "0" * 16
    prof = tmp_path / "profiles"
    prof.mkdir()
    with open(prof / fname, "w") as f:
        json.dump(t, f)
    os.symlink(os.path.join(ROOT, "paper_2001_09258_gb300"), tmp_path / "paper_2001_09258_gb300")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    kept = bench.measured_inst_table(fname)
    assert first not in kept
    for nm, e in t["per_entry_point"].items():
        if nm != first and e["csrc_sha"] == bench.csrc_sha([e["source"]]):
            assert nm in kept
