"""The algorithmic operation counts behind the roofline (CPU only).

The counting build of the oracle (oracle/counting) compiles the oracle's own
sources with floating-point types that tally each operation.  These tests pin
it: it must compute exactly what the oracle computes, reproduce the operation
counts the paper states (the Payne-Hanek table of Section 5.8, the single
reciprocal of the remainder of Section 5.9, the single DD division of the tan
listing of Appendix A), and the committed table opcounts.json must be what
the generator writes today, classified the way opcounts.py classifies the
benchmark's arrays.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle.counting import gen_opcounts as G
from paper_2001_09258_gb300 import inputs as I
from measure import opcounts as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sample(name, n=1024):
    k = oracle.kind(name)
    fn, prec = name.split("_")[0], name.split("_")[-1]
    if k == oracle.K_U16:
        return (I.raw(f"cnt/{name}", n) & np.uint64(0xFFFF)).astype(np.uint16), None
    dt = np.float64 if prec == "f64" else np.float32
    x = I.workload(fn, n, key="cnt", dtype=dt)
    bits = I.raw(f"cnt/bits/{name}", n // 4)
    xr = bits.view(np.float64) if dt == np.float64 else (bits & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    x = np.concatenate([x, xr])
    y = None
    if k in (oracle.K_B64, oracle.K_B32):
        y = np.concatenate([I.workload(fn, n, key="cnt", dtype=dt, operand=1), x[n:][::-1]])
    return x, y


@pytest.mark.parametrize("name", oracle.names())
def test_counting_build_computes_the_oracle(name):
    """Same bits as the plain build on the workload mix plus random bit
    patterns, so every count is of the pinned computation itself."""
    x, y = _sample(name)
    want = oracle.apply(name, x, y, nthreads=1)
    got, tally = oracle.count(name, x, y)
    ws = want if isinstance(want, tuple) else (want,)
    gs = got if isinstance(got, tuple) else (got,)
    for w, g in zip(ws, gs):
        assert w.tobytes() == g.tobytes(), name
    assert oracle.algo_ops(tally, "f64") + oracle.algo_ops(tally, "f32") > 0


@pytest.mark.parametrize("name", [n for n in oracle.c99_names()
                                  if oracle.kind(n) in (oracle.K_U64, oracle.K_B64, oracle.K_SC64,
                                                        oracle.K_U32, oracle.K_B32, oracle.K_SC32)])
def test_counting_build_computes_the_c99_oracle(name):
    """the remaining C99 functions: the counting build gives the plain
    build's bits on their workload and on random bit patterns"""
    prec = name.split("_")[-1]
    n = 4096
    r = I.raw(f"opc99/{name}", n)
    rb = r.view(np.float64) if prec == "f64" else (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    x = np.concatenate([I.c99_workload(name, n), rb])
    y = None
    if oracle.kind(name) in (oracle.K_B64, oracle.K_B32):
        y = np.concatenate([I.c99_workload(name, n, operand=1), rb[::-1].copy()])
    want = oracle.apply(name, x, y, nthreads=1)
    got, _ = oracle.count(name, x, y)
    ws = want if isinstance(want, tuple) else (want,)
    gs = got if isinstance(got, tuple) else (got,)
    for w, g in zip(ws, gs):
        assert w.tobytes() == g.tobytes(), name


def test_payne_hanek_counts_match_the_paper_table():
    """Section 5.8, table of FP operators in Payne-Hanek implementations:
    36 add/sub, 5 mul, 11 FMA per reduction.  The paper's 8 rounds are 2 per
    step; here q mod 4 comes from the two low bits of round(4 x.hi), so 4
    rounds remain (and 4 x.hi is an exponent step, not a multiplication)."""
    x = I.loguniform("cnt/ph", 4096, 1e14, 1.7e308)
    t = oracle.count_ph(x)["f64"]
    n = x.size
    assert t["add"] == 36 * n
    assert t["mul"] == 5 * n
    assert t["fma"] == 11 * n
    assert t["rnd"] == 4 * n
    assert t["div"] == 0 and t["sqrt"] == 0


@pytest.mark.parametrize("fn", ["fmod", "remainder"])
def test_remainder_uses_one_division(fn):
    """Section 5.9: the remainder forms one reciprocal in total, whatever
    the number of long-division steps (here up to ~40 steps): below a
    divisor of 2^1021 without any binary64 division (reading R33: one
    binary32 division and four fma), above it the listing's one division."""
    x = np.concatenate([I.workload(fn, 256, key="cnt1"), I.stress(fn, 256, key="cnt1")])
    y = np.concatenate([I.workload(fn, 256, key="cnt1", operand=1), I.stress(fn, 256, key="cnt1", operand=1)])
    ok = np.isfinite(x) & np.isfinite(y) & (y != 0)
    steps = []
    for a, b in zip(x[ok], y[ok]):
        _, t = oracle.count(f"{fn}_u10_f64", np.array([a]), np.array([b]))
        dv = abs(b) * (2 if fn == "remainder" else 1)
        if abs(a) >= abs(b) and dv < 2.0 ** 1021:
            assert t["f64"]["div"] == 0 and t["f32"]["div"] == 1, (a, b)
        else:
            assert t["f64"]["div"] + t["f32"]["div"] <= 1, (a, b)
        steps.append(oracle.fmod_iters(abs(a), abs(b)))
    assert max(steps) >= 30


def test_tan_has_one_dd_division_and_no_square_root():
    """Appendix A tan: the double-angle reconstruction ends in one DD
    division (one IEEE division) on every path."""
    x = np.concatenate([I.uniform("cnt/tan", 512, -14, 14), I.loguniform("cnt/tan2", 512, 15, 1e13),
                        I.loguniform("cnt/tan3", 512, 1e14, 1e300)])
    _, t = oracle.count("tan_u10_f64", x)
    assert t["f64"]["div"] == x.size and t["f64"]["sqrt"] == 0


def test_exact_counts_of_fixed_paths():
    """A few paths are branch-free, so their count is the same for every
    element: an exact integer mean in the table."""
    t = json.load(open(os.path.join(ROOT, "measure", "opcounts.json")))["f64"]
    for name, cls in [("sin_u10_f64", "cw1"), ("exp_u10_f64", "all"), ("tan_u10_f64", "ph"),
                      ("atan_u10_f64", "small"), ("erf_u10_f64", "f")]:
        v = t[name][cls]["ops"]
        assert v == int(v) and v > 0, (name, cls, v)
    assert t["fmod_u10_f64"]["step"]["ops"] == 17.0


def test_committed_table_is_current():
    """opcounts.json is exactly what the generator writes from the oracle as
    it stands (a change to the oracle's operation sequence must come with a
    regenerated table)."""
    want = json.loads(json.dumps(G.table(), sort_keys=True))
    with open(G.OUT) as f:
        got = json.load(f)
    assert got == want


@pytest.mark.parametrize("name", [n for n in oracle.names() if n.endswith("_f64")])
def test_path_classes_agree(name):
    """opcounts.path_mix (the benchmark side) splits an array into the same
    classes as the generator."""
    fn = name.split("_")[0]
    if fn in ("fmod", "remainder"):
        return
    x = np.concatenate([I.workload(fn, 4096, key="pm"), I.stress(fn, 512, key="pm")]) if fn in I.STRESS_FNS \
        else I.workload(fn, 4096, key="pm")
    y = I.workload(fn, x.size, key="pm", operand=1) if oracle.kind(name) == oracle.K_B64 else None
    pm = O.path_mix(name, x, y)
    gc = {k: int(v.sum()) for k, v in G.classes(fn, x, y).items()}
    assert pm == gc
    assert set(pm) == set(O.OPS[name])


@pytest.mark.parametrize("name", ["sin_u10_f64", "atan2_u10_f64", "tgamma_u10_f64", "erfc_u35_f64",
                                  "log1p_u10_f64", "acosh_u10_f64"])
def test_class_weighting_reproduces_a_direct_count(name):
    """ops_per_launch (class means weighted by the launch's path mix) agrees
    with the counting build run on the same array, within 2 %."""
    fn = name.split("_")[0]
    x = I.workload(fn, 1 << 14, key="direct")
    y = I.workload(fn, 1 << 14, key="direct", operand=1) if oracle.kind(name) == oracle.K_B64 else None
    _, t = oracle.count(name, x, y)
    direct = oracle.algo_ops(t)
    est = O.ops_per_launch(name, x, y)
    assert abs(est - direct) <= 0.02 * direct, (est, direct)


def test_fmod_weighting_with_kernel_steps():
    """fmod/remainder: setup + 17 per step with the step total the kernel's
    loop reports (here the oracle's iteration count, which the GPU tests pin
    to the kernel's) agrees with a direct count within 2 %."""
    x = I.stress("fmod", 2048, key="direct")
    y = I.stress("fmod", 2048, key="direct", operand=1)
    _, t = oracle.count("fmod_u10_f64", x, y)
    steps = sum(oracle.fmod_iters(abs(a), abs(b)) for a, b in zip(x, y))
    est = O.ops_per_launch("fmod_u10_f64", x, y, steps)
    direct = oracle.algo_ops(t)
    assert abs(est - direct) <= 0.02 * direct, (est, direct)
