"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/igamg.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "igamg.h")).read()
    return sorted(set(re.findall(r"^\s*(?:igamg_status|const char\*)\s+(igamg_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1804_02539_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("igamg_setup", "igamg_solve", "igamg_free", "igamg_apply", "igamg_smooth",
                 "igamg_restrict", "igamg_prolong", "igamg_precondition", "igamg_dof_map"):
        assert name in syms


def test_library_exports_every_declared_symbol(built_lib):
    missing = [s for s in declared_symbols() if not hasattr(built_lib, s)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(built_lib):
    from paper_1804_02539_gb300 import igamg
    lib = igamg.load_library()
    for s in declared_symbols():
        assert getattr(lib, s).restype is not None


def test_setup_rejects_bad_problems_without_gpu(built_lib):
    """Argument validation happens before any device work."""
    from paper_1804_02539_gb300 import igamg
    lib = igamg.load_library()
    h = ctypes.c_void_p()
    assert lib.igamg_setup(None, None, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert b"NULL" in lib.igamg_last_error(None) or b"problem" in lib.igamg_last_error(None)
    assert lib.igamg_free(None) == 0
