"""The C-ABI library builds, loads without a GPU and exports every function include/pic.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def libpath():
    from paper_2402_08404_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    return _build.LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pic_create", "pic_emit", "pic_step", "pic_solve_field", "pic_diagnostics", "pic_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2402_08404_gb300 import pic
    monkeypatch.setattr(pic, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pic, "_lib", None)
    with pytest.raises(ImportError):
        pic.lib()


def test_struct_layouts_match_header():
    # ctypes mirrors of the header structs: field order and sizes
    from paper_2402_08404_gb300 import pic
    assert ctypes.sizeof(pic.GridT) == 24
    assert ctypes.sizeof(pic.SpeciesT) == 24
    assert [f for f, _ in pic.Params._fields_] == ["dt", "apex_field", "V0", "T0", "work_function", "w_min",
                                                    "w_max_units", "n_heat", "seed", "flags", "mg_tol",
                                                    "mg_max_cycles", "mg_sweeps", "circuit_R", "circuit_C",
                                                    "sigma_el_en", "sigma_el_nn", "sigma_cx", "coulomb_log",
                                                    "merge_max"]
