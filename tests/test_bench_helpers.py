"""The bench's own arithmetic, checked on the CPU: the volume weights of its
accuracy figure, the FP32 work per cell it divides by for the fused
V-cycle's roofline, and its count of kernel launches per solve."""
import importlib.util
import os

import numpy as np
import pytest

from gpu_helpers import SMALL, oracle_plane

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("key", list(SMALL))
def test_cell_volumes_are_the_oracles_volume_weights(bench, key):
    a = bench.cell_volumes(SMALL[key])
    b = oracle_plane(SMALL[key]).volume_weights()
    ratio = a / b
    # the same weights up to the constant azimuthal factor
    assert np.allclose(ratio, ratio.flat[0], rtol=1e-12, atol=0)


def test_vcycle_flops_per_cell(bench):
    base = dict(nu_pre=2, nu_post=2, n_sor=2, nu_pre_fused=0, nu_post_fused=0)
    # two passes per cycle, (16 + 16 N_SOR) per pass, 40 for the transfers
    assert bench.vcycle_flops_per_cell(base) == 4 * 2 * 48 + 40 == 424
    assert bench.vcycle_flops_per_cell(dict(base, n_sor=1)) == 4 * 2 * 32 + 40
    # the fused levels' own counts replace the level-wide ones
    assert bench.vcycle_flops_per_cell(dict(base, nu_pre_fused=3, nu_post_fused=3)) == 6 * 2 * 48 + 40


class _FakeSolver:
    def __init__(self, sched, first, tail=0):
        self._s, self._f, self._t = sched, first, tail

    def schedule(self):
        return self._s

    def fused_level(self):
        return self._f

    def tail(self):
        return (self._t, 16 if self._t else 0)


def test_launches_per_solve_counts_the_loop_body(bench):
    """One iteration at the benchmark's shape (fused from level 1, nu = (2, 2)):
    residual, 2 x 2 smoothing passes, restriction, fused V-cycle,
    prolongation, 2 x 2 passes (the last does the update) = 12 launches; a
    loop of I iterations runs I + 1 residuals and I V-cycles; a solve adds 8
    fixed launches.  Without post-smoothing the update is a launch of its
    own.  With the tail kernel (P planes) a loop hands over after the first
    iteration that leaves at most P planes active."""
    cyc_psi = [21, 9, 5] + [1] * 126
    cyc_phi = [16, 7, 3] + [1] * 126
    st = {"cycles_psi": cyc_psi, "cycles_phi": cyc_phi}
    s = _FakeSolver(dict(nu_pre=2, nu_post=2, n_sor=1), 1)
    assert bench.launches_per_solve(s, st) == 8 + (22 + 21 * 11) + (17 + 16 * 11)
    s = _FakeSolver(dict(nu_pre=3, nu_post=1, n_sor=2), 2)
    # two level-wide levels: each 2 x 3 + 1 + 1 + 2 x 1 = 10 launches
    v = 2 * 10 + 1
    assert bench.launches_per_solve(s, st) == 8 + (22 + 21 * v) + (17 + 16 * v)
    s = _FakeSolver(dict(nu_pre=2, nu_post=0, n_sor=1), 1)
    # 2 x 2 + 1, fused V-cycle, prolongation, update
    v = 4 + 1 + 1 + 1 + 1
    assert bench.launches_per_solve(s, st) == 8 + (22 + 21 * v) + (17 + 16 * v)
    # tail of 2 planes: Psi hands over after iteration 5 (planes with more
    # than 5 cycles: 21 and 9), Phi after iteration 3 (16 and 7)
    s = _FakeSolver(dict(nu_pre=2, nu_post=2, n_sor=1), 1, tail=2)
    assert bench.launches_per_solve(s, st) == 8 + (6 * 12 + 1) + (4 * 12 + 1)


def test_oracle_timings_runs_the_full_oracle_solve(bench):
    """The CPU baseline times whole oracle solves (every mode, real DGF
    tables) in a spawned pool and in one process."""
    from gpu_helpers import clumps
    sp = SMALL["cyl_cavity"]
    tm = bench.oracle_timings(clumps(sp, 1), sp, warmup=1, steps=2, procs=2, single_thread_repeats=1)
    assert tm["procs"] == 2 and tm["dgf_setup_s"] > 0
    assert len(tm["solve_s"]) == 2 and all(t > 0 for t in tm["solve_s"])
    assert len(tm["solve_1thread_s"]) == 1 and tm["solve_1thread_s"][0] > 0


def test_solve_algorithmic_bytes_follow_the_per_unknown_model(bench):
    """Per real unknown: 152 B per V-cycle and 40 B per refinement step
    (cycles + 1 residual evaluations per mode and solve), plus 32 B per cell
    for the two transforms and one read of the DGF tables."""
    sp = dict(n_r=256, n_tz=128, n_phi=256)
    st = {"cycles_psi": [19] + [3] * 128, "cycles_phi": [15] + [1] * 128}
    cyc = 19 + 3 * 128 + 15 + 128
    want = 2 * 256 * 128 * (152 * cyc + 40 * (cyc + 2 * 129)) + 32 * 256 * 128 * 256 + 8 * 129 * 256 * 256
    assert bench.solve_algorithmic_bytes(sp, st, 256) == want
