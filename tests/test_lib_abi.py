"""The C-ABI library builds, loads and exports every symbol include/wd.h declares.

CPU only: no call here launches device work. Host-only entry points
(status strings, parameter defaults, argument validation) are exercised.
"""

import ctypes as C
import os
import re

import pytest

from paper_2602_14450_gb300 import build, wd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "wd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wd_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return wd.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 13
    assert sorted(wd.SYMBOLS) == names
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    assert L.wd_status_string(wd.WD_OK) == b"WD_OK"
    assert L.wd_status_string(wd.WD_ERR_NOT_SU3) == b"WD_ERR_NOT_SU3"
    assert L.wd_status_string(99) == b"WD_ERR_UNKNOWN"


def test_param_defaults_follow_table2(L):
    p = wd.default_params("mixed_fp16")
    assert (p.s, p.sigma, p.use_shat, p.recalc_gamma, p.rescale_x) == (128.0, 64.0, 1, 1, 0)
    assert abs(p.inner_eps ** 2 - 1e-4) < 1e-18 and p.omega0 == 0.7
    p = wd.default_params("mixed_fp16_plain")
    assert (p.s, p.sigma, p.use_shat) == (1.0, 0.0, 0)
    assert L.wd_solve_params_default(77, C.byref(wd.SolveParams())) == wd.WD_ERR_INVALID_ARG


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 0, 4), (4, 4, 4, 1)])
def test_create_rejects_bad_extents(L, dims):
    h = C.c_void_p()
    rc = L.wd_create((C.c_int * 4)(*dims), 0.12, None, C.byref(h))
    assert rc == wd.WD_ERR_INVALID_ARG and not h.value


def test_create_rejects_bad_boundary_phase(L):
    h = C.c_void_p()
    rc = L.wd_create((C.c_int * 4)(4, 4, 4, 4), 0.12, (C.c_int * 4)(1, 1, 1, 2), C.byref(h))
    assert rc == wd.WD_ERR_INVALID_ARG


def test_null_handle_is_rejected(L):
    assert L.wd_set_gauge(None, None, 0) == wd.WD_ERR_INVALID_ARG
    assert L.wd_apply(None, 0, 18, 0, None, None, None) == wd.WD_ERR_INVALID_ARG
    assert L.wd_solve(None, None, None, 1e-10, 0, None, None, None) == wd.WD_ERR_INVALID_ARG
    assert L.wd_vector_bytes(None, 0) == 0


def test_arith_entry_points_check_their_arguments(L):
    assert L.wd_set_arith(None, 16) == wd.WD_ERR_INVALID_ARG
    assert L.wd_get_arith(None) == 0


STRUCTS = {"wd_solve_params": "SolveParams", "wd_solve_stats": "SolveStats", "wd_tune_result": "TuneResult"}


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's sizes
    and field offsets (a C program built against include/wd.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "wd.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in getattr(wd, pyname)._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, pyname in STRUCTS.items():
        cls = getattr(wd, pyname)
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
