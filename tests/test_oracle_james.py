"""Pins of the oracle's vacuum boundary treatment (Sec. 4) and of the whole
seven-step solve (Sec. 5.1) against closed forms, conservation and brute force.
"""
import json
import os

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import dft, dgf, james
from oracle.geometry import CYLINDRICAL, LOG, SPHERICAL, UNIFORM, Plane

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def cart_centres(p):
    N = p.n_phi
    ph = (np.arange(N) + 0.5) * 2 * np.pi / N
    a = p.r.x[1:-1][:, None, None]
    b = p.t.x[1:-1][None, :, None]
    c = ph[None, None, :]
    if p.geometry == SPHERICAL:
        return np.broadcast_arrays(*cf.sph_to_cart(a, b, c))
    return np.broadcast_arrays(*cf.cyl_to_cart(a, c, b))


def sphere_distance(p, centre):
    x, y, z = cart_centres(p)
    if p.geometry == SPHERICAL:
        cx, cy, cz = cf.sph_to_cart(*centre)
    else:
        cx, cy, cz = cf.cyl_to_cart(*centre)
    return np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)


def rel_l2(p, a, ref):
    w = np.broadcast_to(p.volume_weights()[:, :, None], a.shape)
    return np.sqrt((w * (a - ref) ** 2).sum() / (w * ref**2).sum())


def test_screening_mass_of_mode_zero_cancels_the_interior_mass():
    """sigma is the finite-volume Laplacian of Psi at the ghost cells (Eqs.
    charge_sph, charge_cyl, screen_mass): the discrete divergence theorem makes
    sum_ghosts sigma^0 dV = - sum_cells rho^0 dV exactly."""
    for p in (Plane.make(CYLINDRICAL, 16, 16, 8, UNIFORM, 0.2, 1.0),
              Plane.make(SPHERICAL, 16, 8, 8, LOG, 0.1, 2.0),
              Plane.make(SPHERICAL, 16, 8, 8, UNIFORM, 1.0, 2.0, t_min=0.5, t_max=2.5)):
        rho = np.random.default_rng(0).random((p.n_r, p.n_t, p.n_phi))
        gt = np.zeros((p.n_modes, len(james.boundary_points(p)), len(james.boundary_points(p))))
        _, parts = james.solve(p, rho, gt, return_parts=True)
        dv_g = np.array([p.dV[i, j] for _, i, j in james.boundary_points(p)])
        lhs = (parts["sigma"][:, 0] * dv_g).sum()
        rhs = -(parts["rho_hat"][:, :, 0] * p.volume_weights()).sum()
        assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


CASES = [
    ("cyl_axis_aux", CYLINDRICAL, UNIFORM, 0.0, 1.0, (0.4, 0.0, 0.0), 0.3, (16, 32)),
    ("cyl_cavity_aux", CYLINDRICAL, UNIFORM, 0.2, 1.0, (0.6, 0.5, 0.0), 0.3, (16, 32)),
    ("sph_log_ext", SPHERICAL, LOG, 0.1, 10.0, (2.0, 1.2, 0.5), 1.5, (32, 64)),
]


@pytest.mark.parametrize("name,g,sp,ri,ro,centre,a,ns", CASES)
def test_smooth_sphere_second_order(name, g, sp, ri, ro, centre, a, ns):
    """Whole solve against the closed-form potential of a smooth sphere: the
    error falls at second order (Sec. 6.1.3), which fails for any O(1)
    boundary error (a wrong screening-mass factor, DGF normalisation or sign)."""
    errs = []
    for n in ns:
        p = Plane.make(g, n, n, n, sp, ri, ro)
        d = sphere_distance(p, centre)
        phi = james.solve(p, cf.smooth_sphere_density(d, a), dgf.dgf(p))
        errs.append(rel_l2(p, phi, cf.smooth_sphere_potential(d, a)))
    assert errs[0] / errs[1] > 3.3, errs
    assert errs[1] < 1e-2


@pytest.mark.parametrize("geom", [SPHERICAL, CYLINDRICAL])
def test_double_sphere_matches_closed_form(geom):
    """Sec. 6.1.1 double sphere (paper: max error < 0.1% at N = 256 on N x N x 2N
    grids); here N = 32 on the paper's domains, where the mass representation
    of the spheres limits the error to the percent level."""
    ds = GOLD["double_sphere"]
    N = 32
    if geom == SPHERICAL:
        p = Plane.make(SPHERICAL, N, N, 2 * N, LOG, *ds["sph_domain"]["r"])
        c1 = (ds["sphere1"]["r"], np.pi / 2, ds["sphere1"]["phi"])
        c2 = (ds["sphere2"]["r"], np.pi / 2, np.pi)
    else:
        p = Plane.make(CYLINDRICAL, N, N, 2 * N, LOG, *ds["cyl_domain"]["R"],
                       t_min=ds["cyl_domain"]["z"][0], t_max=ds["cyl_domain"]["z"][1])
        c1 = (ds["cyl_sphere1"]["R"], 0.0, 0.0)
        c2 = (ds["cyl_sphere2_reading"]["R"], np.pi, 0.0)
    d1, d2 = sphere_distance(p, c1), sphere_distance(p, c2)
    a1, a2 = ds["sphere1"]["a"], ds["sphere2"]["a"]
    rho = ((d1 < a1) | (d2 < a2)).astype(float)
    phi = james.solve(p, rho, dgf.dgf(p))
    ref = cf.uniform_sphere_potential(d1, a1) + cf.uniform_sphere_potential(d2, a2)
    assert np.abs((phi - ref) / ref).max() < 0.05
    assert rel_l2(p, phi, ref) < 0.01


def test_boundary_potential_matches_brute_force_green_sum():
    """-Theta at the ghost cells is the potential of the interior mass there
    (Sec. 4, James step 4); compare with the direct sum -G sum rho dV / |x-x'|
    over the cells, whose difference falls with resolution."""
    errs = []
    for n in (16, 32):
        p = Plane.make(CYLINDRICAL, n, n, n, UNIFORM, 0.2, 1.0)
        d = sphere_distance(p, (0.6, 0.5, 0.0))
        rho = cf.smooth_sphere_density(d, 0.3)
        _, parts = james.solve(p, rho, dgf.dgf(p), return_parts=True)
        theta = dft.inverse(parts["theta"], p.n_phi)          # [t, k]
        x, y, z = cart_centres(p)
        m = (rho * p.volume_weights()[:, :, None]).ravel()
        ph = (np.arange(p.n_phi) + 0.5) * 2 * np.pi / p.n_phi
        brute = []
        for side, i, j in james.boundary_points(p):
            gx, gy, gz = cf.cyl_to_cart(p.r.x[i], ph, np.full_like(ph, p.t.x[j]))
            dd = np.sqrt((gx[:, None] - x.ravel()) ** 2 + (gy[:, None] - y.ravel()) ** 2
                         + (gz[:, None] - z.ravel()) ** 2)
            brute.append(-(m / dd).sum(axis=1))
        brute = np.array(brute)
        errs.append(np.abs(-theta - brute).max() / np.abs(brute).max())
    assert errs[1] < 0.02 and errs[0] / errs[1] > 2.5, errs


@pytest.mark.parametrize("p", [Plane.make(CYLINDRICAL, 16, 16, 8, UNIFORM, 0.2, 1.0),
                               Plane.make(SPHERICAL, 32, 16, 8, LOG, 0.1, 10.0)])
def test_dgf_is_nearly_reciprocal(p):
    """Green's reciprocity G^m(t, s) = G^m(s, t): Gt_ts / dV_s is symmetric up
    to the accuracy of the boundary data of the constructions."""
    gt = dgf.dgf(p)
    dV = np.array([p.dV[i, j] for _, i, j in james.boundary_points(p)])
    G = gt / dV[None, None, :]
    asym = np.abs(G - G.transpose(0, 2, 1)).max(axis=(1, 2)) / np.abs(G).max(axis=(1, 2))
    assert asym.max() < 2e-2


def test_domain_enlargement_leaves_potential_unchanged():
    """Vacuum boundary conditions: the same density in a larger box (same
    cells inside) gives the same potential on the common cells."""
    rho_fn = lambda p: cf.smooth_sphere_density(sphere_distance(p, (0.5, 0.3, 0.0)), 0.25)
    small = Plane.make(CYLINDRICAL, 16, 16, 16, UNIFORM, 0.0, 1.0, t_min=-0.5, t_max=0.5)
    big = Plane.make(CYLINDRICAL, 24, 24, 16, UNIFORM, 0.0, 1.5, t_min=-0.75, t_max=0.75)
    ps = james.solve(small, rho_fn(small), dgf.dgf(small))
    pb = james.solve(big, rho_fn(big), dgf.dgf(big))[:16, 4:20, :]
    assert np.abs(ps - pb).max() / np.abs(pb).max() < 5e-3


def test_solution_of_real_density_is_real_and_hermitian():
    p = Plane.make(SPHERICAL, 32, 16, 16, LOG, 0.1, 10.0)
    rho = np.random.default_rng(2).random((32, 16, 16))
    _, parts = james.solve(p, rho, dgf.dgf(p), return_parts=True)
    for key in ("psi", "phi_hat"):
        assert np.abs(parts[key][:, :, 0].imag).max() <= 1e-12 * np.abs(parts[key]).max()
        assert np.abs(parts[key][:, :, -1].imag).max() <= 1e-12 * np.abs(parts[key]).max()
