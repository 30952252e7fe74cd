"""The C-ABI library loads without a GPU and exports every function elas.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "elas.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(elas_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2001_04789_gb300 import build as B
    try:
        return B.build()
    except RuntimeError as e:       # no nvcc on this machine
        pytest.skip(str(e))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["elas_ctx_create", "elas_grid_create", "elas_set_moduli", "elas_set_bc", "elas_solve",
              "elas_query_residual", "elas_op_apply", "elas_op_sweep", "elas_op_restrict",
              "elas_op_prolong_add", "elas_batch_solve"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (elas_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_through_ctypes_without_gpu(libpath):
    from paper_2001_04789_gb300 import elas as E
    L = E.lib()
    for n in declared_functions():
        assert hasattr(L, n)
