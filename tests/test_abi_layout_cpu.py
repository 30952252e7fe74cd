"""The binding's ctypes declarations match the C header: structures field by field, and
every function's arity and argument kinds.

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


def _header_prototypes():
    import re
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "elas.h")).read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"\n\s*([A-Za-z_][A-Za-z_ ]*?\**)\s*\b(elas_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        params = [p.strip() for p in m.group(3).split(",") if p.strip() and p.strip() != "void"]
        protos[m.group(2)] = (m.group(1).strip(), params)
    return protos


def _c_kind(decl, is_return=False):
    """Category of a C parameter declaration (or return type)."""
    if "*" in decl or "[" in decl:
        return "ptr"
    words = decl.replace("const ", "").split()
    if not is_return:
        words = words[:-1]                      # drop the parameter name
    t = " ".join(words)
    if t.startswith("elas_") and t not in ("elas_solve_opts", "elas_solve_info"):
        return "ptr"                            # handles are typedef'd pointers
    return {"int": "i32", "double": "f64", "size_t": "u64", "unsigned long long": "u64",
            "long long": "s64", "void": "void"}[t]


def _ctypes_kind(t):
    if t is None:
        return "void"
    if t in (C.c_void_p, C.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"
    return {C.c_int: "i32", C.c_double: "f64", C.c_size_t: "u64", C.c_ulonglong: "u64",
            C.c_longlong: "s64"}[t]


def test_binding_signatures_match_the_header(E):
    """Every function elas.h declares has ctypes argument and result types in the binding,
    with the header's arity and, per argument, the same kind (32-bit int, double, unsigned
    or signed 64-bit integer, pointer or handle)."""
    L = E.lib()
    protos = _header_prototypes()
    assert len(protos) > 40
    for name, (ret, params) in protos.items():
        fn = getattr(L, name)
        assert fn.argtypes is not None, f"{name}: no ctypes signature in the binding"
        assert len(fn.argtypes) == len(params), name
        assert _ctypes_kind(fn.restype) == _c_kind(ret, is_return=True), name
        for k, (decl, t) in enumerate(zip(params, fn.argtypes)):
            assert _ctypes_kind(t) == _c_kind(decl), (name, k, decl, t)
