"""Smoothing schedule, tile shapes and the autotuner (psolve_set_schedule,
psolve_autotune).

Tile shapes group lines into thread blocks differently but relax every line
with the same arithmetic, so every shape must give bitwise the same solve.
The schedule (Sec. 3.2: a few smoothing cycles per level, a few SOR sweeps
per line) changes the convergence rate, not the converged answer."""
import json
import os
import subprocess
import sys

import pytest

from gpu_helpers import clumps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("nu_pre", "nu_post", "n_sor", "lines_r", "cols_t", "nu_pre_fused", "nu_post_fused")


@pytest.fixture(scope="module")
def ps():
    import paper_2606_17636_gb300 as m
    m.lib()
    return m


def _spec(*a):
    from paper_2606_17636_gb300 import workloads
    return workloads.spec(*a)


def _wide_level_specs():
    """Grids whose finest level is smoothed by the level-wide passes (too
    large for the shared-memory V-cycle)."""
    from paper_2606_17636_gb300 import workloads as wl
    return {"sph_log": _spec(wl.SPHERICAL, 256, 64, 8, wl.LOG, 0.1, 10.0),
            "cyl_cavity": _spec(wl.CYLINDRICAL, 128, 128, 8, wl.UNIFORM, 0.2, 1.0, -0.4, 0.4)}


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("key", ["sph_log", "cyl_cavity"])
@pytest.mark.parametrize("precision", [0, 1])
def test_tile_shapes_give_bitwise_equal_solves(ps, key, precision):
    sp = _wide_level_specs()[key]
    rho = torch.from_numpy(clumps(sp, 41)).cuda()
    s = ps.Solver.from_spec(sp, precision=precision)
    assert s.fused_level() >= 1
    ref = s.solve(rho, tol=1e-10)[0].clone()
    for lines in (4, 8):
        for cols in (8, 16, 32):
            s.set_schedule(2, 2, 2, lines_r=lines, cols_t=cols)
            assert s.schedule()["lines_r"] == lines and s.schedule()["cols_t"] == cols
            phi = s.solve(rho, tol=1e-10)[0]
            assert torch.equal(phi, ref), (lines, cols)
    s.close()


def test_schedule_changes_cycles_not_the_answer(ps):
    sp = _wide_level_specs()["sph_log"]
    rho = torch.from_numpy(clumps(sp, 42)).cuda()
    s = ps.Solver.from_spec(sp, precision=ps.FP64)
    ref = s.solve(rho, tol=1e-11)[0].clone()
    counts = {}
    cases = {"light": dict(nu_pre=1, nu_post=1, n_sor=1), "heavy": dict(nu_pre=3, nu_post=3, n_sor=3),
             "light fused levels": dict(nu_pre=2, nu_post=2, n_sor=2, nu_pre_fused=1, nu_post_fused=1),
             "heavy fused levels": dict(nu_pre=2, nu_post=2, n_sor=2, nu_pre_fused=3, nu_post_fused=3)}
    for name, kw in cases.items():
        s.set_schedule(**kw)
        assert {k: s.schedule()[k] for k in kw} == kw
        phi = s.solve(rho, tol=1e-11)[0]
        counts[name] = s.stats()["iterations_psi"]
        assert _rel(phi, ref) <= 1e-9, name
    assert counts["light"] > counts["heavy"]
    assert counts["light fused levels"] >= counts["heavy fused levels"]
    s.close()


def test_set_schedule_rejects_out_of_range_fields(ps):
    sp = _wide_level_specs()["sph_log"]
    s = ps.Solver.from_spec(sp, precision=ps.MIXED)
    before = s.schedule()
    for bad in [dict(nu_pre=0, nu_post=2, n_sor=2), dict(nu_pre=2, nu_post=9, n_sor=2),
                dict(nu_pre=2, nu_post=2, n_sor=0), dict(nu_pre=2, nu_post=2, n_sor=2, lines_r=6),
                dict(nu_pre=2, nu_post=2, n_sor=2, cols_t=12),
                dict(nu_pre=2, nu_post=2, n_sor=2, nu_pre_fused=9), dict(nu_pre=2, nu_post=2, n_sor=2, nu_post_fused=-1)]:
        with pytest.raises(ps.PSolveError) as e:
            s.set_schedule(**bad)
        assert e.value.code == ps.ERR_ARG
        assert s.schedule() == before
    s.close()


def test_autotune_picks_a_candidate_and_keeps_the_answer(ps):
    sp = _wide_level_specs()["sph_log"]
    rho = torch.from_numpy(clumps(sp, 43)).cuda()
    ref64 = ps.Solver.from_spec(sp, precision=ps.FP64)
    tight = ref64.solve(rho, tol=1e-11)[0].clone()
    ref64.close()
    s = ps.Solver.from_spec(sp, precision=ps.MIXED)
    default = s.solve(rho, tol=1e-8)[0].clone()
    ch = s.autotune(rho, tol=1e-8)
    assert ch["cached"] == 0 and ch["candidates"] >= 18 and ch["ms"] > 0
    assert 1 <= ch["nu_post"] <= ch["nu_pre"] <= 3 and 1 <= ch["n_sor"] <= 3
    assert ch["lines_r"] in (4, 8) and ch["cols_t"] in (0, 8, 16, 32)
    assert 0 <= ch["nu_post_fused"] <= 3 and 0 <= ch["nu_pre_fused"] <= 3
    now = s.schedule()
    assert all(now[k] == ch[k] for k in KEYS)
    phi = s.solve(rho, tol=1e-8)[0]
    st = s.stats()
    assert st["rel_residual_psi"] <= 1e-8 and st["rel_residual_phi"] <= 1e-8
    assert _rel(phi, tight) <= 1e-7
    assert _rel(default, tight) <= 1e-7
    # the same key in this process: installed from the cache, nothing timed
    s2 = ps.Solver.from_spec(sp, precision=ps.MIXED)
    ch2 = s2.autotune(rho, tol=1e-8)
    assert ch2["cached"] == 1 and ch2["candidates"] == 0
    assert all(ch2[k] == ch[k] for k in KEYS)
    s.close()
    s2.close()


def test_autotune_file_cache(ps, tmp_path, monkeypatch):
    sp = _wide_level_specs()["cyl_cavity"]
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("PSOLVE_TUNE_CACHE", str(path))
    rho = torch.from_numpy(clumps(sp, 44)).cuda()
    s = ps.Solver.from_spec(sp, precision=ps.MIXED)
    ch = s.autotune(rho, tol=1e-8)
    s.close()
    assert ch["cached"] == 0
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    f = lines[0].split()
    assert [int(x) for x in f[1:8]] == [ch[k] for k in KEYS]
    # another process reads the file: rewrite the entry and check it is used
    assert len(f) == 10 and int(f[9]) == ch["tail_planes"]
    path.write_text("%s 3 1 1 4 8 2 1 1.0 0\n" % f[0])
    code = ("import json, sys, torch; sys.path.insert(0, %r)\n"
            "import paper_2606_17636_gb300 as ps\n"
            "s = ps.Solver.from_spec(json.loads(%r), precision=ps.MIXED)\n"
            "rho = torch.zeros(s.shape, dtype=torch.float64, device='cuda')\n"
            "print(json.dumps(s.autotune(rho, tol=1e-8)))\n") % (ROOT, json.dumps(sp))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, PSOLVE_TUNE_CACHE=str(path)))
    assert out.returncode == 0, out.stderr[-2000:]
    got = json.loads(out.stdout.strip().splitlines()[-1])
    assert got["cached"] == 1 and got["candidates"] == 0
    assert [got[k] for k in KEYS] == [3, 1, 1, 4, 8, 2, 1] and got["tail_planes"] == 0


def test_autotune_reports_a_failing_solve_and_keeps_the_schedule(ps):
    """A handle whose solves cannot converge (two V-cycles at most): the
    tuner returns the solve's error and leaves the handle's schedule as it
    was.  FP64 on this grid is a key no other test tunes, so the process
    cache cannot answer."""
    sp = _wide_level_specs()["cyl_cavity"]
    rho = torch.from_numpy(clumps(sp, 45)).cuda()
    s = ps.Solver.from_spec(sp, precision=ps.FP64, max_cycles=2)
    s.set_schedule(2, 1, 2, lines_r=8, cols_t=32)
    before = s.schedule()
    with pytest.raises(ps.PSolveError) as e:
        s.autotune(rho, tol=1e-10)
    assert e.value.code == ps.ERR_NOT_CONVERGED
    assert s.schedule() == before
    s.close()
