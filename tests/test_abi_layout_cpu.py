"""The binding's ctypes structures match the C header's, field by field.

A small C program, generated from the ctypes field lists and compiled against
include/elas.h, prints the size of each structure and the offset and size of each field
(a field the header lacks fails to compile); the test compares them with ctypes.  The
library's own option defaults (elas_solve_opts_default, which needs no GPU) are checked
against the documented values, and the binding's keyword mapping onto the structure."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def E():
    from paper_2001_04789_gb300 import build as B
    try:
        B.build()
    except RuntimeError as e:       # no nvcc on this machine
        pytest.skip(str(e))
    from paper_2001_04789_gb300 import elas
    return elas


def _pairs(E):
    return [(E.GridDesc, "elas_grid_desc"), (E.AmrLevelDesc, "elas_amr_level"),
            (E.SolveOpts, "elas_solve_opts"), (E.SolveInfo, "elas_solve_info")]


def test_ctypes_structures_match_the_header(E, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "elas.h"', "int main(void) {"]
    for cls, cname in _pairs(E):
        lines.append(f'    printf("{cname} - %zu %zu\\n", (size_t)0, sizeof({cname}));')
        for name, _ in cls._fields_:
            lines.append(f'    printf("{cname} {name} %zu %zu\\n", offsetof({cname}, {name}), '
                         f'sizeof((({cname}*)0)->{name}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        cname, field, off, size = line.split()
        got[(cname, field)] = (int(off), int(size))
    for cls, cname in _pairs(E):
        assert got[(cname, "-")][1] == C.sizeof(cls), cname
        for name, _ in cls._fields_:
            f = getattr(cls, name)
            assert got[(cname, name)] == (f.offset, f.size), (cname, name)


def test_option_defaults_and_keyword_mapping(E):
    o = E.SolveOpts()
    E.lib().elas_solve_opts_default(C.byref(o))
    assert (o.precision, o.rel_tol, o.max_cycles, o.nu1, o.nu2) == (E.FP64, 1e-8, 100, 2, 2)
    assert (o.warm_start, o.fixed_cycles, o.use_graph, o.inner_cycles) == (0, 0, 0, 1)
    assert (o.smoother, o.cycle, o.outer_residual) == (E.SMOOTH_RB, E.CYCLE_V, E.OUTER_AUTO)
    assert o.omega == pytest.approx(2.0 / 3.0, abs=1e-15)
    m = E._opts(E.MIXED, 1e-6, 50, 1, 3, True, 7, True, 3, E.SMOOTH_GS8, E.CYCLE_F, 0.5, E.OUTER_DF)
    assert (m.precision, m.rel_tol, m.max_cycles, m.nu1, m.nu2) == (E.MIXED, 1e-6, 50, 1, 3)
    assert (m.warm_start, m.fixed_cycles, m.use_graph, m.inner_cycles) == (1, 7, 1, 3)
    assert (m.smoother, m.cycle, m.omega, m.outer_residual) == (E.SMOOTH_GS8, E.CYCLE_F, 0.5, E.OUTER_DF)
    d = E._opts()                                   # unset options keep the library's defaults
    assert (d.smoother, d.cycle, d.outer_residual) == (E.SMOOTH_RB, E.CYCLE_V, E.OUTER_AUTO)
