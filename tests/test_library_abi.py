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


def test_multi_and_server_reject_bad_arguments_without_gpu(built_lib):
    """igamg_solve_multi without a context and a server without workers are refused
    before any device work."""
    from paper_1804_02539_gb300 import igamg
    lib = igamg.load_library()
    b = (ctypes.c_void_p * 2)()
    x = (ctypes.c_void_p * 2)()
    assert lib.igamg_solve_multi(None, 2, b, x, 1e-8, None, None) == 1
    srv = ctypes.c_void_p()
    assert lib.igamg_server_create(None, 0, 1 << 30, ctypes.byref(srv)) == 1
    assert srv.value is None and b"workers" in lib.igamg_last_error(None)
    assert lib.igamg_server_free(None) == 0


STRUCTS = ("igamg_problem", "igamg_options", "igamg_result", "igamg_request_info", "igamg_server_counters")


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's field names, order, offsets and
    size: a C program compiled against include/igamg.h prints them (host compiler only)."""
    import shutil
    import subprocess
    from paper_1804_02539_gb300 import igamg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "igamg.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(igamg, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                          text=True).stdout.splitlines())
    for name in STRUCTS:
        cls = getattr(igamg, name)
        assert int(out[f"{name} size"]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(out[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)
    # and no header field is missing from the mirror: the header's member count per struct
    hdr = open(os.path.join(ROOT, "include", "igamg.h")).read()
    for name in STRUCTS:
        end = re.search(r"\}\s*" + name + r"\s*;", hdr).start()
        body = hdr[hdr.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        decls = [d for d in body.split(";") if d.strip()]
        count = sum(len(d.split(",")) for d in decls)
        assert count == len(getattr(igamg, name)._fields_), name


def test_missing_library_fails_loudly(tmp_path):
    """No silent fallback: without the built library the binding raises."""
    from paper_1804_02539_gb300 import igamg
    with pytest.raises(ImportError, match="not built"):
        igamg.load_library(str(tmp_path / "libigamg.so"))
