"""The C-ABI library builds, loads without a GPU, exports every symbol that
include/relo.h declares, and its structs match the header's layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "relo.h")


@pytest.fixture(scope="module")
def relo():
    from paper_2511_01219_gb300 import _build
    _build.build()
    import paper_2511_01219_gb300 as relo
    relo.lib()
    return relo


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(relo_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("relo_load_map", "relo_set_hypotheses", "relo_relocalize", "relo_create", "relo_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(relo):
    L = relo.lib()
    names = declared_functions()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(relo.EXPORTED) == names


def test_struct_layout_matches_header(relo, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "relo.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(relo_params), sizeof(relo_result),"
        " offsetof(relo_params, n_orient), offsetof(relo_params, hbm_budget), offsetof(relo_result, hyp),"
        " offsetof(relo_result, status)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    P, R = relo.Params, relo.Result
    assert got == [ctypes.sizeof(P), ctypes.sizeof(R), P.n_orient.offset, P.hbm_budget.offset, R.hyp.offset,
                   R.status.offset]


def test_default_params_match_the_paper_constants(relo):
    import oracle
    p = relo.default_params()
    o = oracle.Params()
    for f in ("z_hit", "sigma_hit", "z_rand", "eps", "d_max", "a_mid_min", "a_mid_max", "a_low_min", "a_low_max",
              "tau", "panoramic_ratio", "batch", "local_topk", "n_skip_beam"):
        assert getattr(p, f) == getattr(o, f), f
    assert (p.z_hit, p.sigma_hit, p.z_rand, p.eps) == (1.0, 0.2, 0.0, 1e-6)     # Sec. IV-B, Eq. 23
    assert (p.batch, p.local_topk, p.tau) == (200, 20, 0.95)                     # Sec. IV-C


def test_missing_library_fails_loudly(monkeypatch, relo):
    monkeypatch.setattr(relo, "LIB_PATH", "/nonexistent/librelo.so")
    monkeypatch.setattr(relo, "_lib", None)
    with pytest.raises(ImportError):
        relo.lib()


def test_python_constants_match_the_header_defines(relo):
    """Every RELO_* integer define has the same value in the binding (status
    codes, ranking and scoring metric codes, stage ids)."""
    text = open(HEADER).read()
    defines = {m.group(1): int(m.group(2)) for m in
               re.finditer(r"#define RELO_([A-Z0-9_]+)\s+\(?(-?\d+)\)?", text)}
    assert len(defines) >= 25
    checked = 0
    for name, value in defines.items():
        if name == "N_STAGES":
            assert len(relo.STAGES) == value
        elif hasattr(relo, name):
            assert getattr(relo, name) == value, name
        else:
            continue
        checked += 1
    skipped = sorted(n for n in defines if n != "N_STAGES" and not hasattr(relo, n))
    assert skipped == [], skipped
    assert checked == len(defines)
