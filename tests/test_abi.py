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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of psolve_desc, psolve_stats and psolve_schedule
    have the C layout (sizes and field offsets, from gcc on the header)."""
    import shutil
    import subprocess
    import paper_2606_17636_gb300 as ps
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    mirrors = {"psolve_desc": ps.Desc, "psolve_stats": ps.Stats, "psolve_schedule": ps.Schedule,
               "psolve_plan": ps.Plan}
    lines = ['#include <stdio.h>', '#include "psolve.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, py in mirrors.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def test_enum_values_match_the_header(tmp_path):
    """The binding's constants for the descriptor's choices have the
    header's values."""
    import shutil
    import subprocess
    import paper_2606_17636_gb300 as ps
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    names = {"PSOLVE_COARSEST_AUTO": ps.COARSEST_AUTO, "PSOLVE_COARSEST_SMALL": ps.COARSEST_SMALL,
             "PSOLVE_COARSEST_LARGE": ps.COARSEST_LARGE, "PSOLVE_DGF_AUTO": ps.DGF_AUTO,
             "PSOLVE_DGF_AUX": ps.DGF_AUX, "PSOLVE_DGF_EXTENDED": ps.DGF_EXTENDED,
             "PSOLVE_MIXED": ps.MIXED, "PSOLVE_FP64": ps.FP64}
    lines = ['#include <stdio.h>', '#include "psolve.h"', "int main(void) {"]
    lines += ['printf("%s %%d\\n", (int)%s);' % (n, n) for n in names]
    lines += ["return 0;", "}"]
    src = tmp_path / "enums.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "enums"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for n, v in names.items():
        assert int(got[n]) == v, n


def test_schedule_entry_points_reject_null_arguments(libpath):
    import paper_2606_17636_gb300 as ps
    L = ps.lib()
    s = ps.Schedule(nu_pre=2, nu_post=2, n_sor=2, lines_r=8)
    assert L.psolve_set_schedule(None, ctypes.byref(s)) == ps.ERR_ARG
    assert L.psolve_get_schedule(None, ctypes.byref(s)) == ps.ERR_ARG
    assert L.psolve_autotune(None, None, None, 1e-8, None) == ps.ERR_ARG
    assert "null" in ps.last_error()
