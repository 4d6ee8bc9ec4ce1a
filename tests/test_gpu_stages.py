"""Stage-by-stage parity of the CUDA path with the FP64 oracle (through the
C ABI stage entry points)."""
import numpy as np
import pytest

from gpu_helpers import SMALL, clumps, oracle_plane, rel_l2, to_gpu, to_oracle
from paper_2606_17636_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import paper_2606_17636_gb300 as m
    m.lib()
    return m


def _solver(ps, key, precision):
    return ps.Solver.from_spec(SMALL[key], precision=precision, use_graph=False)


@pytest.mark.parametrize("key", list(SMALL))
def test_forward_and_inverse_transforms(ps, key):
    from oracle import dft
    sp = SMALL[key]
    s = _solver(ps, key, ps.FP64)
    rho = np.random.default_rng(1).standard_normal((sp["n_r"], sp["n_tz"], sp["n_phi"]))
    f = s.stage_forward(torch.from_numpy(rho).cuda()).cpu().numpy()
    ref = 4 * np.pi * dft.forward(rho)
    assert np.abs(to_oracle(f) - ref).max() <= 1e-13 * np.abs(ref).max()
    spec = np.random.default_rng(2).standard_normal(ref.shape) + 1j * np.random.default_rng(3).standard_normal(ref.shape)
    back = s.stage_inverse(torch.from_numpy(to_gpu(spec)).cuda()).cpu().numpy()
    ref2 = dft.inverse(spec, sp["n_phi"])
    assert np.abs(back - ref2).max() <= 1e-13 * np.abs(ref2).max()
    s.close()


def _rand_planes(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("key", list(SMALL))
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
@pytest.mark.parametrize("level", [0, 1])
def test_smooth_restrict_prolong(ps, key, precision, tol, level):
    from oracle import mg
    sp = SMALL[key]
    s = _solver(ps, key, precision)
    p = oracle_plane(sp)
    H = mg.Hierarchy(p)
    nr, nt, M = sp["n_r"] >> level, sp["n_tz"] >> level, s.n_modes
    cdt = torch.complex128 if precision == 0 else torch.complex64
    e0 = _rand_planes((M, nt, nr), 10 + level)
    f0 = _rand_planes((M, nt, nr), 20 + level)
    # smoothing: one cycle of Algorithm 1
    e = torch.from_numpy(e0).to(cdt).cuda()
    f = torch.from_numpy(f0).to(cdt).cuda()
    got = s.stage_smooth(level, e.clone(), f, 1).cpu().numpy().astype(np.complex128)
    ref = np.zeros_like(got)
    for m in range(M):
        u = np.zeros((nr + 2, nt + 2), complex)
        u[1:-1, 1:-1] = e.cpu().numpy()[m].T
        H.smooth(level, m, u, f.cpu().numpy()[m].T.astype(complex), 1)
        ref[m] = u[1:-1, 1:-1].T
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    if level + 1 >= len(H.levels):   # the coarsest level has no transfers
        s.close()
        return
    # defect restriction; the defect cancels terms of size |L e|, so the
    # rounding bound scales with the restricted |f| + |L e|
    from oracle import operator
    gotc = s.stage_restrict(level, e, f).cpu().numpy().astype(np.complex128)
    for m in range(M):
        u = np.zeros((nr + 2, nt + 2), complex)
        u[1:-1, 1:-1] = e.cpu().numpy()[m].T
        fm = f.cpu().numpy()[m].T.astype(complex)
        r = H.residual(level, m, u, fm)
        refc = H.restrict(level, r).T
        absLu = operator.from_vec(abs(operator.matrix(H.levels[level].plane, m)) @ operator.to_vec(np.abs(u[1:-1, 1:-1])), nr, nt)
        scale = H.restrict(level, np.abs(fm) + absLu).real.max()
        assert np.abs(gotc[m] - refc).max() <= tol * scale
    # prolongation + correction
    ec = torch.from_numpy(_rand_planes(gotc.shape, 30)).to(cdt).cuda()
    gotp = s.stage_prolong(level, e.clone(), ec).cpu().numpy().astype(np.complex128)
    for m in range(M):
        refp = e.cpu().numpy()[m].astype(complex) + H.prolong(level, m, ec.cpu().numpy()[m].T.astype(complex)).T
        assert np.abs(gotp[m] - refp).max() <= tol * np.abs(refp).max()
    s.close()


@pytest.mark.parametrize("key", list(SMALL))
@pytest.mark.parametrize("precision", [0, 1])
def test_fp64_residual_stage(ps, key, precision):
    """The refinement's defect (FP64 arithmetic, stored in the buffer
    precision) against the oracle's residual on the finest level."""
    from oracle import mg, operator
    sp = SMALL[key]
    s = _solver(ps, key, precision)
    p = oracle_plane(sp)
    H = mg.Hierarchy(p)
    nr, nt, M = sp["n_r"], sp["n_tz"], s.n_modes
    u = _rand_planes((M, nt, nr), 40)
    f = _rand_planes((M, nt, nr), 41)
    got = s.stage_residual(torch.from_numpy(f).cuda(), torch.from_numpy(u).cuda())
    assert got.dtype == (torch.complex64 if precision else torch.complex128)
    got = got.cpu().numpy().astype(np.complex128)
    for m in range(M):
        uu = np.zeros((nr + 2, nt + 2), complex)
        uu[1:-1, 1:-1] = u[m].T
        ref = H.residual(0, m, uu, f[m].T).T
        absLu = operator.from_vec(abs(operator.matrix(p, m)) @ operator.to_vec(np.abs(u[m].T)), nr, nt).T
        scale = np.abs(f[m]) + absLu
        # elementwise against |f| + |L_m| |u|: the plan's FP64 coefficient
        # tables agree with the oracle's to about 1e-12 relative (products of
        # face areas, spacings, metric factors and the mode's s_m^2 formed in
        # another order); then (mixed) one rounding to FP32
        bound = 1e-11 * scale + (2.0 ** -24 * np.abs(ref) if precision else 0.0)
        assert np.all(np.abs(got[m] - ref) <= bound), m
    with pytest.raises(ps.PSolveError):
        bad = torch.zeros(1, dtype=torch.complex128, device="cuda")
        from paper_2606_17636_gb300 import lib, check
        check(lib().psolve_stage_residual(s.h, 1 - precision, bad.data_ptr(), bad.data_ptr(),
                                          bad.data_ptr()), "psolve_stage_residual")
    s.close()


def _crafted_doubles(n, seed):
    """FP64 values whose FP32 rounding exercises every branch: normal values
    over the whole FP32 range, exact ties (the 29 dropped fraction bits equal
    to half a unit) with even and odd kept parts, one bit either side of a
    tie, values that round up to the largest FP32 number or overflow to
    infinity, results in the FP32 subnormal range, FP64 subnormals, zeros,
    infinities and NaN."""
    rng = np.random.default_rng(seed)
    out = [rng.standard_normal(n // 2) * 10.0 ** rng.uniform(-37, 38, n // 2)]
    bits = []
    for _ in range(64):
        e = int(rng.integers(1023 - 126, 1023 + 127))
        kept = int(rng.integers(0, 1 << 23))
        for rest in (1 << 28, (1 << 28) - 1, (1 << 28) + 1, 0, (1 << 29) - 1):
            for sign in (0, 1):
                bits.append((sign << 63) | (e << 52) | (kept << 29) | rest)
    out.append(np.array(bits, dtype=np.uint64).view(np.float64))
    fmax = float(np.finfo(np.float32).max)
    out.append(np.array([fmax, np.nextafter(fmax, np.inf), fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24),
                         -fmax * (1 + 2.0 ** -24), 1e39, 1e-39, 1e-45, 7e-46, 1e-310, -1e-310,
                         1.1754943508222875e-38, 1.1754942e-38, 0.0, -0.0, np.inf, -np.inf, np.nan]))
    v = np.concatenate(out)
    return np.resize(v, n)


def test_residual_rounds_to_fp32_as_ieee(ps):
    """The mixed path stores the FP64 defect in FP32 with its own
    integer-pipe conversion: with u = 0 the defect is f itself, so every
    stored value must be f rounded to nearest even, as numpy's binary64 to
    binary32 conversion gives it (zeros compared by value)."""
    sp = SMALL["sph_log"]
    s = _solver(ps, "sph_log", ps.MIXED)
    M, nt, nr = s.n_modes, sp["n_tz"], sp["n_r"]
    n = M * nt * nr
    f = (_crafted_doubles(n, 60) + 1j * _crafted_doubles(n, 61)[::-1]).reshape(M, nt, nr)
    r = s.stage_residual(torch.from_numpy(f).cuda(), torch.zeros((M, nt, nr), dtype=torch.complex128,
                                                                 device="cuda"))
    got = torch.view_as_real(r).cpu().numpy().reshape(-1)
    want = np.stack([f.real, f.imag], axis=-1).reshape(-1).astype(np.float32)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    same = got[~nan].view(np.uint32) == want[~nan].view(np.uint32)
    assert np.all(same | (got[~nan] == want[~nan])), got[~nan][~same][:8]
    s.close()


@pytest.mark.parametrize("key", list(SMALL))
def test_mg_solve_reaches_direct_solution_and_counts_cycles(ps, key):
    import scipy.sparse.linalg as spla

    from oracle import mg, operator
    sp = SMALL[key]
    s = _solver(ps, key, ps.FP64)
    p = oracle_plane(sp)
    M = s.n_modes
    f = _rand_planes((M, sp["n_tz"], sp["n_r"]), 7)
    u, cyc, rc = s.stage_mg_solve(torch.from_numpy(f).cuda(), tol=1e-12)
    assert rc == 0
    u = u.cpu().numpy()
    H = mg.Hierarchy(p)
    for m in range(M):
        A = operator.matrix(p, m).tocsc()
        b = f[m].T
        x = spla.spsolve(A, operator.to_vec(b.real)) + 1j * spla.spsolve(A, operator.to_vec(b.imag))
        ref = operator.from_vec(x, sp["n_r"], sp["n_tz"]).T
        assert np.abs(u[m] - ref).max() <= 1e-10 * np.abs(ref).max()
        if m in (0, 1, M - 1):
            _, c_or, _ = H.solve(m, b, 1e-12)
            assert abs(cyc[m] - c_or) <= 1, (m, cyc[m], c_or)
    s.close()


@pytest.mark.parametrize("key", list(SMALL))
def test_screening_boundary_and_dgf(ps, key):
    from oracle import dgf, james
    sp = SMALL[key]
    s = _solver(ps, key, ps.FP64)
    p = oracle_plane(sp)
    gt = dgf.dgf(p)
    got_gt = s.dgf().cpu().numpy()
    assert got_gt.shape == gt.shape
    assert np.abs(got_gt - gt).max() <= 1e-9 * np.abs(gt).max()
    psi = _rand_planes((s.n_modes, sp["n_tz"], sp["n_r"]), 5)
    sig = s.stage_screening(torch.from_numpy(psi).cuda()).cpu().numpy()
    ref_sig = np.stack([james.screening_mass(p, psi[m].T) for m in range(s.n_modes)])
    assert np.abs(sig - ref_sig).max() <= 1e-13 * np.abs(ref_sig).max()
    th = s.stage_boundary(torch.from_numpy(ref_sig).cuda()).cpu().numpy()
    ref_th = np.einsum("mts,ms->mt", got_gt, ref_sig)
    assert np.abs(th - ref_th).max() <= 1e-13 * np.abs(ref_th).max()
    s.close()


@pytest.mark.parametrize("key", list(SMALL))
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-4)])
def test_fused_vcycle_matches_oracle_vcycle(ps, key, precision, tol):
    """The fused coarse V-cycle (Sec. 3) from the fused level down, zero
    initial guess, against the oracle's recursive V-cycle on the same level.
    FP32: the cycle chains ~400 single-precision operations per cell and
    level plus the exact coarsest solve, hence 1e-4 of the largest value."""
    from oracle import mg
    sp = SMALL[key]
    s = _solver(ps, key, precision)
    lev = s.fused_level()
    H = mg.Hierarchy(oracle_plane(sp))
    nr, nt, M = sp["n_r"] >> lev, sp["n_tz"] >> lev, s.n_modes
    cdt = torch.complex128 if precision == 0 else torch.complex64
    f = torch.from_numpy(_rand_planes((M, nt, nr), 40 + lev)).to(cdt).cuda()
    got = s.stage_vcycle(f).cpu().numpy().astype(np.complex128)
    fh = f.cpu().numpy().astype(np.complex128)
    ref = np.zeros_like(got)
    for m in range(M):
        u = np.zeros((nr + 2, nt + 2), complex)
        H.vcycle(lev, m, u, fh[m].T)
        ref[m] = u[1:-1, 1:-1].T
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= tol, err
    s.close()


# grids whose large-rule coarsest level differs from the small rule's:
# 64 x 32 under a fused 128 x 64 level (full theta: the mirror-symmetric
# form), 32 x 32 under 64 x 64 (cylinder with the axis), and 64 x 32 with an
# off-centre polar range (the general separable form)
LARGE = {
    "sph_log_128x64": workloads.spec(workloads.SPHERICAL, 128, 64, 8, workloads.LOG, 0.05, 20.0),
    "cyl_axis_128x128": workloads.spec(workloads.CYLINDRICAL, 128, 128, 8, workloads.UNIFORM, 0.0, 1.0,
                                       -0.5, 0.5),
    "sph_band_128x64": workloads.spec(workloads.SPHERICAL, 128, 64, 8, workloads.UNIFORM, 1.0, 2.0,
                                      0.3 * np.pi, 0.65 * np.pi),
}


@pytest.mark.parametrize("key", list(LARGE))
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-4)])
def test_fused_vcycle_with_the_large_coarsest_level(ps, key, precision, tol):
    """The fused V-cycle on the large coarsest-level rule (short side up to
    32, up to 2048 cells; Sec. 3.3 leaves the size open), against the
    oracle's V-cycle on the same levels.  The mixed path solves that level
    with FP32 polar transforms around FP64 radial sweeps: its error stays
    within the FP32 V-cycle's 1e-4."""
    from oracle import mg
    sp = LARGE[key]
    s = ps.Solver.from_spec(sp, precision=precision, use_graph=False, coarsest_size=ps.COARSEST_LARGE)
    plan = ps.plan_inspect(sp, precision=precision, coarsest_size=ps.COARSEST_LARGE)
    H = mg.Hierarchy(oracle_plane(sp), min_cells=32, max_coarse=2048)
    assert [(l.plane.n_r, l.plane.n_t) for l in H.levels] == plan["levels"]
    assert s.n_levels == len(plan["levels"]) >= 2
    lev = s.fused_level()
    nr, nt, M = sp["n_r"] >> lev, sp["n_tz"] >> lev, s.n_modes
    cdt = torch.complex128 if precision == 0 else torch.complex64
    f = torch.from_numpy(_rand_planes((M, nt, nr), 60 + lev)).to(cdt).cuda()
    got = s.stage_vcycle(f).cpu().numpy().astype(np.complex128)
    fh = f.cpu().numpy().astype(np.complex128)
    for m in range(M):
        u = np.zeros((nr + 2, nt + 2), complex)
        H.vcycle(lev, m, u, fh[m].T)
        ref = u[1:-1, 1:-1].T
        err = np.abs(got[m] - ref).max() / np.abs(ref).max()
        assert err <= tol, (m, err)
    s.close()


@pytest.mark.parametrize("key", ["sph_log_128x64", "cyl_axis_128x128"])
@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-11, 1e-9), (1, 1e-9, 1e-7)])
def test_solve_with_the_large_coarsest_level(ps, key, precision, tol, bound):
    """Whole solves (captured graph) on the large coarsest-level rule against
    the oracle's solve, every mode solved directly: the coarsest size changes
    the V-cycle, not the solution.  FP64 path at tol 1e-11, mixed path at
    1e-9."""
    from oracle import dgf, james
    sp = LARGE[key]
    s = ps.Solver.from_spec(sp, precision=precision, use_graph=True, coarsest_size=ps.COARSEST_LARGE)
    assert s.n_levels == len(ps.plan_inspect(sp, precision=precision, coarsest_size=ps.COARSEST_LARGE)["levels"])
    p = oracle_plane(sp)
    rho = clumps(sp, 43)
    ref = james.solve(p, rho, dgf.dgf(p))
    phi, rc = s.solve(torch.from_numpy(rho).cuda(), tol=tol)
    assert rc == ps.OK
    err = rel_l2(p, phi.cpu().numpy(), ref)
    assert err <= bound, err
    s.close()
