"""Direct pins of the azimuthal Green's-function mode sums (Sec. 4.2, Eqs.
DGF_bc_sph and DGF_bc_cyl, and the radial derivative the extended-domain
construction imposes on its inner face) and of the spherical extended-domain
DGF (Sec. 4.2, logarithmic grids with a large radial extent ratio).

The mode sums are checked against the same sums written in Cartesian form:
every field point is placed at its azimuth 2 pi k / N explicitly and its
distance to the source taken from Cartesian coordinates, so that an error in
the A - B cos and C - D cos forms (a dropped term, a sign, a swapped
argument) shows.  The derivative is checked against a centred difference in
r of that Cartesian sum.
"""
import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import dft, dgf, green, james
from oracle.geometry import CYLINDRICAL, LOG, SPHERICAL, Plane


def _cartesian_mode_sum(geometry, N, G, xt, yt, xs, ys):
    """sum_k cos(2 pi m k / N) (-G / |x_t(phi_k) - x_s(0)|), m = 0..N/2,
    for scalar field point (xt, yt) and source (xs, ys)."""
    ph = 2.0 * np.pi * np.arange(N) / N
    if geometry == SPHERICAL:
        tx, ty, tz = cf.sph_to_cart(xt, yt, ph)
        sx, sy, sz = cf.sph_to_cart(xs, ys, 0.0)
    else:
        tx, ty, tz = cf.cyl_to_cart(xt, ph, yt)
        sx, sy, sz = cf.cyl_to_cart(xs, 0.0, ys)
    d = np.sqrt((tx - sx) ** 2 + (ty - sy) ** 2 + (tz - sz) ** 2)
    m = np.arange(N // 2 + 1)[:, None]
    return (np.cos(m * ph[None, :]) * (-G / d)[None, :]).sum(axis=1)


POINTS = {
    SPHERICAL: [((2.0, 1.1), (0.7, 0.4)), ((0.15, 2.8), (3.0, 1.9)), ((5.0, 0.3), (4.5, 0.35))],
    CYLINDRICAL: [((1.0, 0.2), (0.4, -0.3)), ((0.3, -1.0), (2.0, 0.5)), ((1.5, 0.0), (1.45, 0.05))],
}


@pytest.mark.parametrize("geometry", [SPHERICAL, CYLINDRICAL])
@pytest.mark.parametrize("N", [8, 64])
def test_mode_sum_equals_cartesian_sum(geometry, N):
    G = 1.3
    for (xt, yt), (xs, ys) in POINTS[geometry]:
        got = green.mode_sum(geometry, N, G, xt, yt, xs, ys)
        ref = _cartesian_mode_sum(geometry, N, G, xt, yt, xs, ys)
        assert got.shape == (N // 2 + 1,)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (got, ref)


@pytest.mark.parametrize("geometry", [SPHERICAL, CYLINDRICAL])
def test_mode_sum_broadcasts_over_points(geometry):
    """Arrays of field points against one source give the scalar results."""
    N, G = 16, 1.0
    pts = POINTS[geometry]
    xt = np.array([p[0][0] for p in pts])
    yt = np.array([p[0][1] for p in pts])
    xs, ys = pts[0][1]
    got = green.mode_sum(geometry, N, G, xt, yt, xs, ys)
    for q in range(len(pts)):
        ref = _cartesian_mode_sum(geometry, N, G, xt[q], yt[q], xs, ys)
        assert np.abs(got[q] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("geometry", [SPHERICAL, CYLINDRICAL])
@pytest.mark.parametrize("N", [8, 64])
def test_mode_sum_dr_equals_centred_difference(geometry, N):
    """d/dr of the field point's radius, at fixed polar angle (spherical) or
    height (cylindrical): the fourth-order centred difference of the
    Cartesian sum with step h = 1e-3 r has error O((h/d)^4), below 1e-8
    relative even for the closest pair (d = 0.07)."""
    G = 0.7
    for (xt, yt), (xs, ys) in POINTS[geometry]:
        h = 1e-3 * xt
        S = lambda r: _cartesian_mode_sum(geometry, N, G, r, yt, xs, ys)
        fd = (8.0 * (S(xt + h) - S(xt - h)) - (S(xt + 2 * h) - S(xt - 2 * h))) / (12.0 * h)
        got = green.mode_sum_dr(geometry, N, G, xt, yt, xs, ys)
        assert np.abs(got - fd).max() <= 1e-6 * np.abs(fd).max(), (got, fd)


def test_mode_sum_dr_sign_for_an_outward_field_point():
    """Moving the field point away from a source raises -G/d (less negative):
    the m = 0 derivative is positive when the point lies outside the source's
    radius on the same ray."""
    for geometry, (xt, yt), (xs, ys) in ((SPHERICAL, (3.0, 1.0), (1.0, 1.0)),
                                          (CYLINDRICAL, (3.0, 0.0), (1.0, 0.0))):
        assert green.mode_sum_dr(geometry, 32, 1.0, xt, yt, xs, ys)[0] > 0.0


def _sph_cart_centres(p):
    N = p.n_phi
    ph = (np.arange(N) + 0.5) * 2 * np.pi / N
    return np.broadcast_arrays(*cf.sph_to_cart(p.r.x[1:-1][:, None, None],
                                               p.t.x[1:-1][None, :, None], ph[None, None, :]))


def test_spherical_extended_domain_boundary_potential_matches_brute_force():
    """The extended-domain construction of a full-theta logarithmic sphere
    (r_out / r_in = 100, n_r >= 32): -Theta at every boundary ghost cell
    (inner and outer radial) is the potential of the interior mass there.
    Compare with the direct sum -G sum rho dV / |x - x'| over all cells; the
    difference falls at second order when all three directions are refined
    (with N_phi fixed, the azimuthal discretisation error of the discrete
    operator would stay)."""
    errs = []
    for n in (32, 64):
        p = Plane.make(SPHERICAL, n, n // 2, n // 2, LOG, 0.1, 10.0)
        assert dgf.uses_extended_domain(p)
        x, y, z = _sph_cart_centres(p)
        cx, cy, cz = cf.sph_to_cart(2.0, 1.2, 0.5)
        d = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
        rho = cf.smooth_sphere_density(d, 1.5)
        _, parts = james.solve(p, rho, dgf.dgf(p), return_parts=True)
        theta = dft.inverse(parts["theta"], p.n_phi)           # [ghost, k]
        mass = (rho * p.volume_weights()[:, :, None]).ravel()
        ph = (np.arange(p.n_phi) + 0.5) * 2 * np.pi / p.n_phi
        brute = []
        for side, i, j in james.boundary_points(p):
            gx, gy, gz = np.broadcast_arrays(*cf.sph_to_cart(p.r.x[i], p.t.x[j], ph))
            dd = np.sqrt((gx[:, None] - x.ravel()) ** 2 + (gy[:, None] - y.ravel()) ** 2
                         + (gz[:, None] - z.ravel()) ** 2)
            brute.append(-(mass / dd).sum(axis=1))
        brute = np.array(brute)
        errs.append(np.abs(-theta - brute).max() / np.abs(brute).max())
    assert errs[1] < 5e-3 and errs[0] / errs[1] > 3.0, errs
