"""The C-ABI library builds, loads and exports every function include/rte.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "rte.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:[A-Za-z_][A-Za-z0-9_]*\s+)+\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src,
                       flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


def test_header_declares_the_boundary_calls():
    names = _declared_functions()
    for required in ("rte_problem_create", "rte_sweep", "rte_scalar_flux", "romsad_build_greedy", "romsad_apply",
                     "fgmres_solve"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2410_08735_gb300 import binding, build_lib
    path = build_lib.build()
    import ctypes
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the whole header
    assert set(_declared_functions()) <= set(binding.exported_symbols())


def test_status_strings_and_version_without_gpu():
    from paper_2410_08735_gb300 import binding
    lib = binding.load(build_if_missing=True)
    assert lib.rte_status_string(0) == b"RTE_OK"
    assert lib.rte_status_string(4) == b"RTE_ERR_NOT_CONVERGED"
    import ctypes
    a, b = ctypes.c_int(), ctypes.c_int()
    assert lib.rte_version(ctypes.byref(a), ctypes.byref(b)) == 0


def test_invalid_descriptor_rejected_before_touching_the_device():
    from paper_2410_08735_gb300 import binding
    import ctypes
    lib = binding.load(build_if_missing=True)
    d = binding.ProblemDesc()
    d.dim = 3
    h = ctypes.c_void_p()
    assert lib.rte_problem_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"dim" in lib.rte_last_error()
