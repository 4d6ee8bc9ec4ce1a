"""The C-ABI library loads and exports every entry point the header declares
(no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "psolve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psolve_[a-z_]+)\s*\(", src)) - {"psolve_alloc_fn", "psolve_free_fn"})


@pytest.fixture(scope="module")
def libpath():
    import paper_2606_17636_gb300 as ps
    if not os.path.exists(ps.LIB_PATH):
        from paper_2606_17636_gb300 import build
        build.build()
    return ps.LIB_PATH


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    names = declared()
    assert "psolve_create" in names and "psolve_solve" in names and "psolve_destroy" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_declares_the_same_names(libpath):
    import paper_2606_17636_gb300 as ps
    L = ps.lib()
    for n in declared():
        assert getattr(L, n).argtypes is not None or n == "psolve_last_error", n


def test_invalid_arguments_fail_without_a_gpu(libpath):
    import paper_2606_17636_gb300 as ps
    L = ps.lib()
    h = ctypes.c_void_p()
    assert L.psolve_create(ctypes.byref(h), 0, 24, 16, 16, 1, 0.1, 10.0) == ps.ERR_ARG
    assert "power" in ps.last_error()
    assert L.psolve_create(ctypes.byref(h), 0, 32, 16, 16, 1, 0.0, 10.0) == ps.ERR_ARG
    assert L.psolve_solve(None, None, None, 1e-8) == ps.ERR_ARG
    L.psolve_destroy(None)


def test_static_scratch_limit_matches_the_header():
    import paper_2606_17636_gb300 as ps
    src = open(os.path.join(ROOT, "include", "psolve.h")).read()
    m = re.search(r"#define PSOLVE_STATIC_SCRATCH_BYTES \((\d+)u \* 1024u \* 1024u\)", src)
    assert m and int(m.group(1)) * 1024 * 1024 == ps.STATIC_SCRATCH_BYTES


def test_static_entry_point_rejects_bad_arguments_without_a_gpu(libpath):
    import paper_2606_17636_gb300 as ps
    L = ps.lib()
    assert L.psolve_stage_smooth_static(None, 0, 0, None, None, 1) == ps.ERR_ARG
    assert "null" in ps.last_error()
