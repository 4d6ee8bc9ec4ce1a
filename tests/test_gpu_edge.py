"""Edge cases of the CUDA path against the oracle: zero density, a density
with a single azimuthal mode, the smallest grid (one multigrid level), the
largest azimuthal resolution, and elongated grids (largest coarse blocks,
dense coarse solve inside the DGF construction)."""
import numpy as np
import pytest

from gpu_helpers import clumps, oracle_plane, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import paper_2606_17636_gb300 as m
    m.lib()
    return m


def _spec(*a, **k):
    from paper_2606_17636_gb300 import workloads
    return workloads.spec(*a, **k)


def _oracle(spec, rho):
    from oracle import dgf, james
    p = oracle_plane(spec)
    return p, james.solve(p, rho, dgf.dgf(p))


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_density_gives_zero_potential(ps, precision):
    from paper_2606_17636_gb300 import workloads as wl
    sp = _spec(wl.CYLINDRICAL, 32, 32, 16, wl.UNIFORM, 0.0, 1.0, -0.5, 0.5)
    s = ps.Solver.from_spec(sp, precision=precision)
    phi, rc = s.solve(torch.zeros((32, 32, 16), dtype=torch.float64, device="cuda"), tol=1e-8)
    assert rc == ps.OK
    assert torch.count_nonzero(phi).item() == 0
    st = s.stats()
    assert all(v == 0 for v in st["status"])
    s.close()


def test_single_mode_density_excites_one_mode(ps):
    from oracle import dft, dgf, james
    from paper_2606_17636_gb300 import workloads as wl
    sp = _spec(wl.SPHERICAL, 64, 32, 16, wl.LOG, 0.1, 10.0)
    r, t, ph = wl.midpoints(sp)
    g = np.exp(-(np.log(r[:, None] / 1.0)) ** 2) * np.sin(t[None, :]) ** 3
    rho = g[:, :, None] * np.cos(3 * ph[None, None, :])
    s = ps.Solver.from_spec(sp, precision=ps.FP64)
    phi, rc = s.solve(torch.from_numpy(rho).cuda(), tol=1e-12)
    s.close()
    modes = dft.forward(phi.cpu().numpy())
    p = oracle_plane(sp)
    f = 4.0 * np.pi * p.G * dft.forward(rho)
    ref = james.solve_mode(p, 3, f[:, :, 3], dgf.dgf(p, modes=[3])[0])[3]
    scale = np.abs(ref).max()
    for m in range(modes.shape[2]):
        if m != 3:
            assert np.abs(modes[:, :, m]).max() <= 1e-12 * scale, m
    assert np.abs(modes[:, :, 3] - ref).max() <= 1e-10 * scale


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-10), (1, 1e-10, 1e-7)])
def test_smallest_grid_single_level(ps, precision, tol, bound):
    from paper_2606_17636_gb300 import workloads as wl
    sp = _spec(wl.CYLINDRICAL, 8, 8, 4, wl.UNIFORM, 0.2, 1.0)
    rho = clumps(sp, 21)
    s = ps.Solver.from_spec(sp, precision=precision)
    assert s.n_levels == 1
    phi, rc = s.solve(torch.from_numpy(rho).cuda(), tol=tol)
    s.close()
    p, ref = _oracle(sp, rho)
    assert rel_l2(p, phi.cpu().numpy(), ref) <= bound


def test_largest_azimuthal_resolution(ps):
    from oracle import dft, dgf, james
    from paper_2606_17636_gb300 import workloads as wl
    sp = _spec(wl.CYLINDRICAL, 16, 16, 1024, wl.UNIFORM, 0.25, 1.25)
    # clumps plus seeded white noise, so that the highest modes carry signal
    rho = clumps(sp, 22) + 0.1 * np.random.default_rng(22).standard_normal((16, 16, 1024))
    s = ps.Solver.from_spec(sp, precision=ps.FP64)
    phi, rc = s.solve(torch.from_numpy(rho).cuda(), tol=1e-12)
    s.close()
    modes = dft.forward(phi.cpu().numpy())
    p = oracle_plane(sp)
    f = 4.0 * np.pi * p.G * dft.forward(rho)
    sampled = (0, 1, 255, 511, 512)
    gt = dgf.dgf(p, modes=sampled)
    refs = [james.solve_mode(p, m, f[:, :, m], gt[k])[3] for k, m in enumerate(sampled)]
    scale0 = np.abs(refs[0]).max()
    for m, ref in zip(sampled, refs):
        # relative to the mode itself, or at rounding level of the whole
        # potential for modes the smooth density barely excites
        err = np.abs(modes[:, :, m] - ref).max()
        assert err <= 1e-10 * np.abs(ref).max() + 1e-13 * scale0, (m, err, np.abs(ref).max())


@pytest.mark.parametrize("geometry", ["cyl", "sph"])
def test_elongated_grids(ps, geometry):
    """Aspect ratio 16, the largest accepted: the cylinder's coarsest level
    is 64 x 4 (the largest block of the block-tridiagonal coarse solve); the
    logarithmic sphere's DGF uses the extended domain, 512 x 16, whose
    coarsest level (128 x 4) takes the dense coarse solve."""
    from paper_2606_17636_gb300 import workloads as wl
    if geometry == "cyl":
        sp = _spec(wl.CYLINDRICAL, 256, 16, 8, wl.UNIFORM, 0.125, 4.125, -0.5, 0.5)
    else:
        sp = _spec(wl.SPHERICAL, 256, 16, 8, wl.LOG, 0.1, 100.0)
    rho = clumps(sp, 23)
    s = ps.Solver.from_spec(sp, precision=ps.FP64)
    phi, rc = s.solve(torch.from_numpy(rho).cuda(), tol=1e-11)
    s.close()
    p, ref = _oracle(sp, rho)
    assert rel_l2(p, phi.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("geometry", ["cyl_radial", "sph_polar"])
def test_largest_radial_and_polar_sizes(ps, geometry):
    """The largest accepted line lengths at the largest accepted aspect
    ratio: 1024 radial cells (a cylindrical shell whose cells are square in
    (R, z)) and 1024 polar cells (uniform spherical shell), on the mixed
    path against the oracle.  The FP64 path holds lines of at most 512
    cells and refuses these grids at create.  (Cells far from square along
    1024-cell lines, e.g. a logarithmic sphere with 1024 radial and 64 polar
    cells, defeat the single-sweep SOR line relaxation: the low modes then
    stop at the cycle cap and report it.)"""
    from paper_2606_17636_gb300 import workloads as wl
    if geometry == "cyl_radial":
        sp = _spec(wl.CYLINDRICAL, 1024, 64, 4, wl.UNIFORM, 0.5, 1.5, -1.0 / 32, 1.0 / 32)
    else:
        sp = _spec(wl.SPHERICAL, 64, 1024, 4, wl.UNIFORM, 1.0, 2.0)
    with pytest.raises(ps.PSolveError) as ei:
        ps.Solver.from_spec(sp, precision=ps.FP64)
    assert ei.value.code == ps.ERR_ARG and "512" in str(ei.value)
    rho = clumps(sp, 24)
    p, ref = _oracle(sp, rho)
    s = ps.Solver.from_spec(sp, precision=ps.MIXED)
    phi, rc = s.solve(torch.from_numpy(rho).cuda(), tol=1e-10)
    assert rc == ps.OK
    s.close()
    err = rel_l2(p, phi.cpu().numpy(), ref)
    assert err <= 1e-7, err


def test_extended_domain_size_limit(ps):
    """The extended-domain DGF doubles n_r, so a logarithmic grid with
    r_out / r_in >= 100 and 1024 radial cells is refused with a message
    that names the auxiliary-window alternative, which it accepts."""
    from paper_2606_17636_gb300 import workloads as wl
    sp = _spec(wl.SPHERICAL, 1024, 64, 4, wl.LOG, 0.1, 10.0)
    with pytest.raises(ps.PSolveError) as ei:
        ps.Solver.from_spec(sp, precision=ps.MIXED)
    assert ei.value.code == ps.ERR_ARG and "PSOLVE_DGF_AUX" in str(ei.value)
    s = ps.Solver.from_spec(sp, precision=ps.MIXED, dgf_construction=ps.DGF_AUX)
    phi, rc = s.solve(torch.from_numpy(clumps(sp, 25)).cuda(), tol=1e-9)
    assert rc == ps.OK and torch.isfinite(phi).all()
    s.close()
