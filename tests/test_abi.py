"""The C-ABI library: it loads without a GPU, exports every symbol declared in
include/sleefcu.h, and its host-side argument checks behave as documented
(these paths return before any CUDA call)."""
import ctypes
import os
import re

import pytest

import paper_2001_09258_gb300 as sleefcu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "sleefcu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sleefcu_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = sleefcu.lib()
    names = declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header():
    names = set(declared())
    for e in sleefcu.entry_points():
        assert "sleefcu_" + e in names, e
    c99 = {"sleefcu_" + e for e in sleefcu.c99_entry_points()}
    fn_decl = {n for n in names if re.match(r"sleefcu_\w+_u(10|35)_(f64|f32|bf16|f16)$", n)} - c99
    assert fn_decl == {"sleefcu_" + e for e in sleefcu.entry_points()}
    masked = {n for n in names if n.endswith("_masked")}
    assert masked == {"sleefcu_" + e + "_masked" for e in sleefcu.masked_entry_points()}
    assert c99 <= names
    other = {n for n in names if re.match(r"sleefcu_[a-z0-9]+(_u(05|35))?_(f64|f32)$", n)} - fn_decl
    assert other == c99


@pytest.mark.parametrize("name", sleefcu.c99_entry_points())
def test_c99_n_zero_and_null_pointers(name):
    f = sleefcu.raw(name)
    nptr = len(f.argtypes) - 2
    assert f(*([None] * nptr), 0, None) == 0
    assert f(*([None] * nptr), 7, None) == -1
    assert name in sleefcu.last_error()


def test_c99_set_matches_oracle_names():
    import oracle
    assert sorted(sleefcu.c99_entry_points()) == sorted(oracle.c99_names())


def test_version_and_error_text():
    assert b"sleefcu" in sleefcu.lib().sleefcu_version()
    assert isinstance(sleefcu.last_error(), str)


@pytest.mark.parametrize("name", sleefcu.entry_points())
def test_n_zero_and_null_pointers(name):
    """n == 0 is OK with null pointers; a null pointer with n > 0 is EINVAL
    and sets the thread-local error text.  Neither reaches the GPU."""
    f = sleefcu.raw(name)
    nptr = len(f.argtypes) - 2
    assert f(*([None] * nptr), 0, None) == 0
    assert f(*([None] * nptr), 5, None) == -1
    assert name in sleefcu.last_error()


def test_cuda_literals_match_paper_listing():
    """The CUDA tan kernel carries the coefficients printed in Appendix A."""
    gold = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "tan_listing.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            gold[k] = float.fromhex(v) if "0x" in v else float(v)
    src = open(os.path.join(ROOT, "paper_2001_09258_gb300", "csrc", "trig_f64.cu")).read()
    body = re.search(r"kTanC\[8\] = \{(.*?)\};", src, re.S).group(1)
    vals = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-f.]+p[-+]?\d+", body)]
    assert vals == [gold[f"estrin{i}"] for i in range(8)][::-1]
    c3 = re.search(r"TAN_C3 = (0x[0-9a-f.p+-]+);", src).group(1)
    assert float.fromhex(c3) == gold["horner"]
    for name, key in (("PIO2_A", "pio2_hi"), ("PIO2_B", "pio2_lo"), ("TWOPI_H", "twopi_hi"),
                      ("TWOPI_L", "twopi_lo")):
        v = re.search(rf"constexpr double {name} = (-?0x[0-9a-f.p+-]+);", src).group(1)
        assert float.fromhex(v) == gold[key], name


def test_phtab_generators_agree():
    """The CUDA build's Payne-Hanek table (Chudnovsky pi, Python Fractions)
    equals the oracle's (Machin pi, C bignum): two independent derivations
    of the Payne-Hanek table-generation figure."""
    import importlib.util
    import numpy as np
    import oracle
    spec = importlib.util.spec_from_file_location(
        "gen_phtab", os.path.join(ROOT, "paper_2001_09258_gb300", "csrc", "gen_phtab.py"))
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    t64, i64, t32, i32 = g.tables()
    tab, ib = oracle.ph_table()
    assert np.array_equal(np.array(t64), tab)
    assert list(ib) == i64


@pytest.mark.parametrize("name", sleefcu.masked_entry_points())
def test_masked_n_zero_and_null_pointers(name):
    """The masked entry points follow the same argument rules, the mask
    included."""
    f = sleefcu.raw(name + "_masked")
    nptr = len(f.argtypes) - 2
    assert f(*([None] * nptr), 0, None) == 0
    assert f(*([None] * nptr), 5, None) == -1
    assert name + "_masked" in sleefcu.last_error()


def test_checked_build_exports_every_declared_symbol():
    """libsleefcu_checked.so (-DSLEEFCU_CHECKED) has the whole interface and
    says which build it is; the normal build refuses the checked-only query."""
    L = sleefcu.lib_checked()
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing
    assert L.sleefcu_is_checked() == 1
    assert sleefcu.lib().sleefcu_is_checked() == 0
    assert b"checked" in L.sleefcu_version()
    c = ctypes.c_ulonglong(7)
    assert sleefcu.lib().sleefcu_checked_error_count(ctypes.byref(c), 0) == -3
    assert "checked" in sleefcu.last_error()
    assert L.sleefcu_checked_error_count(None, 0) == -1
