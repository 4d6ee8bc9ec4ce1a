"""The multigrid plan (psolve_plan_inspect), computed on the host with no
GPU: the coarsening rules (small and large coarsest level), the form of the
direct coarsest solve (Sec. 3.3 allows a direct solver) and its factor
sizes, and argument checks."""
import numpy as np
import pytest

from paper_2606_17636_gb300 import workloads as wl


@pytest.fixture(scope="module")
def ps():
    import os
    import paper_2606_17636_gb300 as m
    if not os.path.exists(m.LIB_PATH):
        from paper_2606_17636_gb300 import build
        build.build()
    return m


def _coarsen(nr, nt, side=16, cells=1024):
    """The coarsening rule: halve both sides while the short side exceeds
    `side`, or exceeds 4 with more than `cells` cells (small rule 16 / 1024,
    large rule 32 / 2048)."""
    out = [(nr, nt)]
    while True:
        mn = min(nr, nt)
        if not (mn > side or (mn > 4 and nr * nt > cells)):
            return out
        nr, nt = nr // 2, nt // 2
        out.append((nr, nt))


def test_benchmark_grid_plan(ps):
    sp = wl.spec(wl.SPHERICAL, 256, 128, 256, wl.LOG, 0.05, 20.0)
    # the mixed path's automatic choice: the large coarsest level (64 x 32)
    p = ps.plan_inspect(sp)
    assert p["n_modes"] == 129
    assert p["levels"] == [(256, 128), (128, 64), (64, 32)]
    # full theta range: the polar operator is mirror-symmetric about the equator
    assert p["coarsest"] == "separable, mirror-symmetric"
    nr, nt = p["levels"][-1]
    # half of V and of V^-1 (nt^2 in all), three Thomas factor tables nt x nr
    assert p["coarse_doubles_per_mode"] == nt * nt + 3 * nt * nr
    # the FP64 path, and the small rule on request: 32 x 16
    for q in (ps.plan_inspect(sp, precision=0), ps.plan_inspect(sp, coarsest_size=ps.COARSEST_SMALL)):
        assert q["levels"] == [(256, 128), (128, 64), (64, 32), (32, 16)]
        assert q["coarsest"] == "separable, mirror-symmetric"
    assert ps.plan_inspect(sp, precision=0, coarsest_size=ps.COARSEST_LARGE)["levels"] == p["levels"]


@pytest.mark.parametrize("nr,nt", [(8, 8), (16, 8), (32, 32), (64, 16), (128, 8), (256, 16), (8, 128),
                                   (512, 256), (1024, 64), (64, 1024)])
def test_levels_follow_the_coarsening_rule(ps, nr, nt):
    sp = wl.spec(wl.CYLINDRICAL, nr, nt, 8, wl.UNIFORM, 0.2, 1.0)
    small, large = _coarsen(nr, nt), _coarsen(nr, nt, 32, 2048)
    if max(nr, nt) <= 512:   # the FP64 path's line limit
        assert ps.plan_inspect(sp, precision=0)["levels"] == small
    assert ps.plan_inspect(sp, coarsest_size=ps.COARSEST_SMALL)["levels"] == small
    # the large rule when the coarsest level is separable (at most 64 polar
    # cells); the automatic choice takes it only with two levels or more
    sep = large[-1][1] <= 64
    assert ps.plan_inspect(sp, coarsest_size=ps.COARSEST_LARGE)["levels"] == (large if sep else small)
    auto = large if sep and len(large) >= 2 else small
    assert ps.plan_inspect(sp)["levels"] == auto


def test_coarsest_size_is_checked(ps):
    sp = wl.spec(wl.SPHERICAL, 32, 32, 8, wl.UNIFORM, 0.5, 2.0)
    for bad in (-1, 3):
        with pytest.raises(ps.PSolveError) as e:
            ps.plan_inspect(sp, coarsest_size=bad)
        assert e.value.code == ps.ERR_ARG and "coarsest_size" in str(e.value)


def test_off_centre_polar_range_takes_the_general_separable_form(ps):
    p = ps.plan_inspect(wl.spec(wl.SPHERICAL, 32, 32, 8, wl.UNIFORM, 1.0, 2.0, 0.3 * np.pi, 0.65 * np.pi))
    assert p["coarsest"] == "separable"
    nr, nt = p["levels"][-1]
    assert p["coarse_doubles_per_mode"] == (2 * nt * nt + 3 * nt * nr + 1) // 2 * 2


@pytest.mark.parametrize("sp", [
    wl.spec(wl.SPHERICAL, 64, 32, 16, wl.LOG, 0.1, 10.0),                          # full theta
    wl.spec(wl.SPHERICAL, 32, 32, 8, wl.UNIFORM, 1.0, 2.0, 0.25 * np.pi, 0.75 * np.pi),  # centred range
    wl.spec(wl.CYLINDRICAL, 32, 64, 8, wl.UNIFORM, 0.2, 1.0, -0.3, 0.5),          # uniform z, any range
])
def test_mirror_symmetric_polar_operators(ps, sp):
    assert ps.plan_inspect(sp)["coarsest"] == "separable, mirror-symmetric"


def test_many_polar_cells_on_the_coarsest_level_take_block_factors(ps):
    # 8 x 128 is not coarsened (short side 8, 1024 cells); 128 polar cells
    # exceed the separable form's 64, so the polar rows become 8 x 8 blocks
    p = ps.plan_inspect(wl.spec(wl.CYLINDRICAL, 8, 128, 8, wl.UNIFORM, 0.2, 1.0))
    assert p["levels"] == [(8, 128)]
    assert p["coarsest"] == "block-tridiagonal"
    assert p["coarse_doubles_per_mode"] == 128 * 8 * (8 + 2)


@pytest.mark.parametrize("bad,word", [
    (dict(n_r=24), "power"),
    (dict(spacing=wl.LOG, r_in=0.0), "r_in"),
    (dict(n_r=512, n_tz=8), "16"),
    (dict(t_min=-0.5, t_max=1.0), "theta"),
])
def test_invalid_descriptors_are_rejected(ps, bad, word):
    sp = dict(wl.spec(wl.SPHERICAL, 32, 32, 8, wl.UNIFORM, 0.5, 2.0))
    sp.update(bad)
    with pytest.raises(ps.PSolveError) as e:
        ps.plan_inspect(sp)
    assert e.value.code == ps.ERR_ARG
    assert word in str(e.value)


@pytest.mark.parametrize("sp,bound", [
    # full theta: the poles make the polar weights span a wide range, and the
    # factors' residual sits near 1e-12 in either separable form
    (wl.spec(wl.SPHERICAL, 256, 128, 16, wl.LOG, 0.05, 20.0), 1e-11),
    (wl.spec(wl.SPHERICAL, 128, 64, 16, wl.LOG, 0.1, 10.0), 1e-12),
    # away from the poles both forms reach rounding level (64 x 32 coarsest
    # level for the mixed path's large rule here)
    (wl.spec(wl.SPHERICAL, 256, 128, 16, wl.LOG, 0.05, 20.0, 0.3 * np.pi, 0.7 * np.pi), 2e-13),
    (wl.spec(wl.SPHERICAL, 32, 32, 8, wl.UNIFORM, 1.0, 2.0, 0.3 * np.pi, 0.65 * np.pi), 1e-13),
    (wl.spec(wl.CYLINDRICAL, 64, 64, 16, wl.UNIFORM, 0.0, 1.0), 1e-13),
    (wl.spec(wl.CYLINDRICAL, 512, 256, 16, wl.UNIFORM, 0.2, 4.0, -1.0, 1.0), 1e-13),
])
def test_coarsest_factors_solve_the_coarsest_operator(ps, sp, bound):
    """The separable factors applied to a fixed vector, in the kernel's order
    of operations, against the coarsest operator applied to the result: the
    largest relative residual over all modes."""
    p = ps.plan_inspect(sp)
    assert p["coarsest"].startswith("separable")
    assert 0.0 <= p["coarse_check"] <= bound, p


def test_block_factors_report_no_separable_check(ps):
    p = ps.plan_inspect(wl.spec(wl.CYLINDRICAL, 8, 128, 8, wl.UNIFORM, 0.2, 1.0))
    assert p["coarsest"] == "block-tridiagonal" and p["coarse_check"] == -1.0


def test_tail_layout_of_the_benchmark_grid():
    """The cluster-resident tail's shared-memory layout (16 CTAs per plane,
    row slabs of 8/4/2/1 rows on the 256 x 128 .. 32 x 16 levels) fits one
    SM for the smoothing sweeps the autotuner picks (halo depth 2 n_sor, up
    to three sweeps); four need too deep a halo, and the FP64 path keeps the
    batched loop."""
    import paper_2606_17636_gb300 as ps
    from paper_2606_17636_gb300 import workloads
    w3 = workloads.spec(workloads.SPHERICAL, 256, 128, 256, workloads.LOG, 0.05, 20.0)
    small = dict(coarsest_size=ps.COARSEST_SMALL)
    for n_sor in (1, 2, 3):
        p = ps.plan_inspect(w3, n_sor=n_sor, **small)
        assert p["tail_cluster_ctas"] == 16
        assert 0 < p["tail_smem_bytes"] <= 224 * 1024
    assert (ps.plan_inspect(w3, n_sor=1, **small)["tail_smem_bytes"]
            < ps.plan_inspect(w3, n_sor=2, **small)["tail_smem_bytes"])
    assert ps.plan_inspect(w3, n_sor=4, **small)["tail_cluster_ctas"] == 0
    assert ps.plan_inspect(w3, precision=0)["tail_cluster_ctas"] == 0
    # the tail kernel takes the small coarsest level only
    assert ps.plan_inspect(w3)["tail_cluster_ctas"] == 0
    # radial lines of 512 cells are beyond the tail kernel's line relaxation
    w4 = workloads.spec(workloads.CYLINDRICAL, 512, 256, 512, workloads.UNIFORM, 0.2, 4.0, -1.0, 1.0)
    assert ps.plan_inspect(w4)["tail_cluster_ctas"] == 0
