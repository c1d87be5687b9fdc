"""The C-ABI library loads without a GPU and exports every entry point the public
header declares; the binding refuses to load when the library is missing."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pet_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for required in ("pet_plan_create", "pet_forward", "pet_back", "pet_objective_grad", "pet_rdp",
                     "pet_precond", "pet_solver_run", "pet_em_update", "pet_nrmse"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2506_04976_gb300 import build as B
    lib = ctypes.CDLL(B.build())
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    from paper_2506_04976_gb300 import build as B
    lib = ctypes.CDLL(B.build())
    lib.pet_status_str.restype = ctypes.c_char_p
    assert lib.pet_status_str(0) == b"ok"
    assert b"infeasible" in lib.pet_status_str(3)


def test_binding_refuses_to_load_without_the_library(tmp_path):
    """A copy of the binding whose library directory is empty raises ImportError at
    import: no operation can fall back to the CPU."""
    import importlib.util
    src = os.path.join(ROOT, "paper_2506_04976_gb300", "binding.py")
    pkg = tmp_path / "pkg_without_lib"
    pkg.mkdir()
    dst = pkg / "binding.py"
    dst.write_text(open(src).read())
    spec = importlib.util.spec_from_file_location("binding_without_lib", str(dst))
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError, match="is missing"):
        spec.loader.exec_module(mod)
