"""The C-ABI library loads and exports every entry point include/rsol.h
declares; parameter validation runs on the host (no GPU needed)."""
from __future__ import annotations

import ctypes as C
import os
import re

import pytest

import paper_2111_14704_gb300 as rs
from paper_2111_14704_gb300 import build as rsbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "rsol.h")).read()
    return sorted(set(re.findall(r"^\s*(?:rsol_status|const char \*|int64_t)\s*(rsol_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    rsbuild.build()
    return rs.load_library()


def test_header_declares_the_hot_path_entry_points():
    syms = declared_symbols()
    for name in ("rsol_init", "rsol_push_gather", "rsol_deposit", "rsol_sort", "rsol_moments"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(rs.EXPORTS) | set(declared_symbols())


def test_params_struct_layout_matches_header():
    # int32 x 8 then double x 5
    assert C.sizeof(rs.CParams) == 8 * 4 + 5 * 8
    assert C.sizeof(rs.CParticles) == 8 + 8 * 8
    assert C.sizeof(rs.CBatchDesc) == 2 * 4 + 4 * 8


def test_struct_layouts_match_a_c_compiler(tmp_path):
    """Every struct the binding mirrors has the size and field offsets that gcc
    gives the header's declaration."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    pairs = [("rsol_params", rs.CParams), ("rsol_particles", rs.CParticles),
             ("rsol_batch_desc", rs.CBatchDesc), ("rsol_grad_desc", rs.CGradDesc),
             ("rsol_subcycle_desc", rs.CSubcycleDesc)]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rsol.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs:
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


@pytest.mark.parametrize("bad", [
    dict(nx=1), dict(nx=1025), dict(shape=3), dict(precision=16), dict(bin=3), dict(bin=32),
    dict(c_tilde=2.0), dict(c_tilde=0.0), dict(q=0.0), dict(q_over_m=0.0), dict(dx=-1.0),
    dict(deterministic=2), dict(c=float("nan")), dict(warps=4), dict(warps=32),
])
def test_init_rejects_invalid_params_on_host(lib, bad):
    kw = dict(nx=8, ny=8, nz=8, shape=2, precision=32, c=1.0, c_tilde=0.1)
    kw.update(bad)
    p = rs.Params(**kw).to_c()
    h = C.c_void_p(123)
    assert lib.rsol_init(C.byref(p), C.byref(h)) == 1
    assert not h.value


def test_null_arguments_rejected(lib):
    assert lib.rsol_init(None, None) == 1
    assert lib.rsol_destroy(None) == 0
    assert lib.rsol_push_gather(None, None, None, 1.0, None, None) == 1
    assert lib.rsol_sort(None, None, None, None) == 1
    assert lib.rsol_moments(None, None, None, None, None) == 1
    assert lib.rsol_deposit(None, None, None, None) == 1
    assert lib.rsol_check(None, None) == 1
