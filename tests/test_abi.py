"""CPU checks of the C ABI: the library builds for sm_103a, loads, and
exports every function declared in include/bopgb.h (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bopgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\s*\*)\s*(bop_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1803_07491_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bop_create", "bop_destroy", "bop_build_hamiltonian", "bop_moments", "bop_recursion",
                     "bop_energy", "bop_forces", "bop_evaluate_host", "bop_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(L, name), name
    L.bop_version.restype = ctypes.c_int
    assert L.bop_version() >= 100


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1803_07491_gb300 import bop
    saved = bop._LIB
    bop._LIB = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            bop.lib(str(tmp_path / "missing.so"))
    finally:
        bop._LIB = saved


def test_model_struct_layout_matches_header():
    """The ctypes mirror lists the C fields in the same order."""
    from paper_1803_07491_gb300 import bop
    src = open(os.path.join(ROOT, "include", "bopgb.h")).read()
    body = src[src.index("typedef struct {\n  int norb;"):src.index("} bop_model;")]
    names = re.findall(r"(\w+)(?:\[\d+\])?\s*[,;]", body)
    assert [f for f, _ in bop.bop_model._fields_] == names
