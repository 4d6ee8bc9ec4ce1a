"""Pins of the oracle's geometry (Sec. 2.1.1, 2.1.2) against quadrature and
analytic volumes, and of its operator against the general finite-volume
formula (Eq. poisson_discrete) and against closed-form 1-D solutions (App. A).
"""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.sparse.linalg as spla

from oracle import closed_forms as cf
from oracle import operator
from oracle.geometry import CYLINDRICAL, LOG, SPHERICAL, UNIFORM, Axis, Plane

GRIDS = [
    (SPHERICAL, LOG, 0.1, 10.0, {}),
    (SPHERICAL, UNIFORM, 0.0, 2.0, {}),
    (SPHERICAL, UNIFORM, 1.0, 3.0, dict(t_min=0.3 * np.pi, t_max=0.7 * np.pi)),
    (CYLINDRICAL, UNIFORM, 0.0, 1.0, {}),
    (CYLINDRICAL, LOG, 0.05, 4.0, dict(t_min=-1.0, t_max=2.0)),
]


@pytest.mark.parametrize("g,sp,ri,ro,kw", GRIDS)
def test_volumes_sum_to_analytic_volume(g, sp, ri, ro, kw):
    p = Plane.make(g, 16, 8, 12, sp, ri, ro, **kw)
    total = p.volume_weights().sum() * p.n_phi
    if g == SPHERICAL:
        t0, t1 = kw.get("t_min", 0.0), kw.get("t_max", np.pi)
        exact = 2.0 * np.pi / 3.0 * (ro**3 - ri**3) * (np.cos(t0) - np.cos(t1))
    else:
        z0, z1 = kw.get("t_min", -(ro - ri) / 2), kw.get("t_max", (ro - ri) / 2)
        exact = np.pi * (ro**2 - ri**2) * (z1 - z0)
    assert abs(total - exact) <= 1e-13 * exact


@pytest.mark.parametrize("kind,lo,hi,sp", [("r_sph", 0.1, 10.0, LOG), ("r_sph", 0.0, 1.0, UNIFORM),
                                            ("r_cyl", 0.2, 4.0, UNIFORM), ("r_cyl", 0.01, 1.0, LOG),
                                            ("theta", 0.0, np.pi, UNIFORM)])
def test_centroids_match_quadrature(kind, lo, hi, sp):
    ax = Axis.make(kind, 8, lo, hi, sp)
    wt = {"r_sph": lambda s: s * s, "r_cyl": lambda s: s, "theta": np.sin}[kind]
    for c in range(1, ax.n + 1):
        a, b = ax.F[c], ax.F[c + 1]
        num = si.quad(lambda s: s * wt(s), a, b, epsabs=0, epsrel=1e-13)[0]
        den = si.quad(wt, a, b, epsabs=0, epsrel=1e-13)[0]
        assert abs(ax.x[c] - num / den) <= 1e-12 * max(1.0, abs(ax.x[c]))


def test_ghost_centres_mirror_across_axis_and_pole():
    r = Axis.make("r_cyl", 8, 0.0, 1.0)
    assert abs(r.x[0] + r.x[1]) < 1e-15
    t = Axis.make("theta", 8, 0.0, np.pi)
    assert abs(t.x[0] + t.x[1]) < 1e-14
    assert abs(t.x[9] - (2 * np.pi - t.x[8])) < 1e-13


def test_zero_area_faces_have_zero_coefficients():
    p = Plane.make(SPHERICAL, 8, 8, 8, UNIFORM, 0.0, 1.0)
    assert p.aW[1] == 0.0 and p.aS[1] == 0.0 and p.aN[8] == 0.0
    assert not p.has_inner() and not p.has_lower() and not p.has_upper()
    q = Plane.make(CYLINDRICAL, 8, 8, 8, UNIFORM, 0.0, 1.0)
    assert q.aW[1] == 0.0 and q.has_lower() and q.has_upper()


def _fv3d(p, U, m):
    """Eq. poisson_discrete assembled from face areas (Eqs. surface_sph,
    surface_cyl), projected distances and volumes (Eqs. vol_sph, vol_cyl),
    applied to u_ijk = U_ij exp(2 pi i m k / N) and returned at k = 0."""
    N, dphi = p.n_phi, p.dphi
    Fr, Ft, xr, xt = p.r.F, p.t.F, p.r.x, p.t.x
    nr, nt = p.n_r, p.n_t
    ph = lambda k: np.exp(2j * np.pi * m * k / N)
    out = np.zeros((nr, nt), dtype=complex)
    for i in range(1, nr + 1):
        for j in range(1, nt + 1):
            ri0, ri1, tj0, tj1 = Fr[i], Fr[i + 1], Ft[j], Ft[j + 1]
            if p.geometry == SPHERICAL:
                dV = (ri1**3 - ri0**3) / 3 * (np.cos(tj0) - np.cos(tj1)) * dphi
                faces = [
                    (ri1**2 * (np.cos(tj0) - np.cos(tj1)) * dphi, xr[i + 1] - xr[i], U[i + 1, j]),
                    (ri0**2 * (np.cos(tj0) - np.cos(tj1)) * dphi, xr[i] - xr[i - 1], U[i - 1, j]),
                    (0.5 * (ri1**2 - ri0**2) * abs(np.sin(tj1)) * dphi * (tj1 < np.pi - 1e-12),
                     xr[i] * (xt[j + 1] - xt[j]), U[i, j + 1]),
                    (0.5 * (ri1**2 - ri0**2) * abs(np.sin(tj0)) * dphi * (tj0 > 1e-12),
                     xr[i] * (xt[j] - xt[j - 1]), U[i, j - 1]),
                ]
                aphi = 0.5 * (ri1**2 - ri0**2) * (tj1 - tj0)
                dph = xr[i] * np.sin(xt[j]) * dphi
            else:
                dz = tj1 - tj0
                dV = 0.5 * (ri1**2 - ri0**2) * dphi * dz
                faces = [
                    (ri1 * dphi * dz, xr[i + 1] - xr[i], U[i + 1, j]),
                    (ri0 * dphi * dz, xr[i] - xr[i - 1], U[i - 1, j]),
                    (0.5 * (ri1**2 - ri0**2) * dphi, xt[j + 1] - xt[j], U[i, j + 1]),
                    (0.5 * (ri1**2 - ri0**2) * dphi, xt[j] - xt[j - 1], U[i, j - 1]),
                ]
                aphi = (ri1 - ri0) * dz
                dph = xr[i] * dphi
            s = sum(A * (un - U[i, j]) / d for A, d, un in faces)
            s += aphi * (U[i, j] * ph(1) - U[i, j]) / dph + aphi * (U[i, j] * ph(-1) - U[i, j]) / dph
            out[i - 1, j - 1] = s / dV
    return out


@pytest.mark.parametrize("g,sp,ri,ro,kw", GRIDS)
@pytest.mark.parametrize("m", [0, 1, 3, 6])
def test_mode_operator_equals_3d_finite_volume_operator(g, sp, ri, ro, kw, m):
    p = Plane.make(g, 6, 5, 12, sp, ri, ro, **kw)
    rng = np.random.default_rng(m)
    U = np.zeros((p.n_r + 2, p.n_t + 2), dtype=complex)
    U[1:-1, 1:-1] = rng.standard_normal((p.n_r, p.n_t)) + 1j * rng.standard_normal((p.n_r, p.n_t))
    ref = _fv3d(p, U, m)
    got = operator.apply(p, m, U)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("g,sp,ri,ro,kw", GRIDS)
@pytest.mark.parametrize("m", [0, 2, 5])
def test_operator_is_volume_symmetric_and_negative_definite(g, sp, ri, ro, kw, m):
    p = Plane.make(g, 8, 6, 12, sp, ri, ro, **kw)
    A = operator.matrix(p, m).toarray()
    w = operator.to_vec(p.volume_weights())
    B = w[:, None] * A
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    ev = np.linalg.eigvalsh(0.5 * (B + B.T))
    assert ev.max() < 0.0


def _dirichlet_solve(p, m, f, exact_fn):
    """Solve L_m u = f with Dirichlet ghosts = exact values at ghost centres."""
    g = np.zeros((p.n_r + 2, p.n_t + 2))
    R, T = np.meshgrid(p.r.x, p.t.x, indexing="ij")
    ex = exact_fn(R, T)
    g[0, :], g[-1, :], g[:, 0], g[:, -1] = ex[0, :], ex[-1, :], ex[:, 0], ex[:, -1]
    b = f - operator.ghost_rhs(p, g)
    u = spla.spsolve(operator.matrix(p, m).tocsc(), operator.to_vec(b))
    return operator.from_vec(u, p.n_r, p.n_t), ex[1:-1, 1:-1]


@pytest.mark.parametrize("sp", [LOG, UNIFORM])
def test_radial_operator_second_order_on_smooth_radial_potential(sp):
    """Radial part (nabla^2_r, Eq. discrete_poisson_sph) against the potential
    of a smooth sphere centred at the origin; full theta so only the radial
    operator acts at m = 0."""
    errs = []
    for n in (16, 32, 64):
        p = Plane.make(SPHERICAL, n, 4, 4, sp, 0.1, 1.0)
        R, _ = np.meshgrid(p.r.x[1:-1], p.t.x[1:-1], indexing="ij")
        f = 4 * np.pi * cf.smooth_sphere_density(R, 0.8)
        u, ex = _dirichlet_solve(p, 0, f, lambda r, t: cf.smooth_sphere_potential(r, 0.8))
        errs.append(np.abs(u - ex).max() / np.abs(ex).max())
    assert errs[1] / errs[2] > 3.5 and errs[0] / errs[1] > 3.5


def test_radial_shell_of_appendix_a():
    """App. A radial problem: discontinuous shell density; the FV solution
    converges to the printed closed form (unevenly: the shell edges do not
    sit on cell faces, so the represented mass jitters with resolution)."""
    errs = []
    for n in (32, 128, 256):
        p = Plane.make(SPHERICAL, n, 4, 4, LOG, 1e-3, 1.0)
        R, _ = np.meshgrid(p.r.x[1:-1], p.t.x[1:-1], indexing="ij")
        f = 4 * np.pi * ((R >= 0.2) & (R <= 0.5)).astype(float)
        u, ex = _dirichlet_solve(p, 0, f, lambda r, t: cf.radial_shell_potential(r, 0.2, 0.5))
        errs.append(np.abs(u - ex).max() / np.abs(ex).max())
    assert max(errs[1:]) < 0.02 and errs[0] > 5 * max(errs[1:])


def test_polar_operator_second_order_on_sin2theta():
    """App. A polar problem: (1/sin) d/dth (sin du/dth) = f with u = sin 2 th
    on [pi/6, 5 pi/6], using the polar coefficients of nabla^2_theta."""
    errs = []
    for n in (16, 32, 64):
        ax = Axis.make("theta", n, np.pi / 6, 5 * np.pi / 6)
        p = Plane(SPHERICAL, Axis.make("r_sph", 2, 1.0, 1.1), ax, 4)
        a, c = p.aS[1:n + 1], p.aN[1:n + 1]
        A = np.diag(-(a + c)) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        x = ax.x
        b = cf.polar_source(x[1:n + 1])
        b[0] -= a[0] * np.sin(2 * x[0])
        b[-1] -= c[-1] * np.sin(2 * x[n + 1])
        u = np.linalg.solve(A, b)
        errs.append(np.abs(u - np.sin(2 * x[1:n + 1])).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
