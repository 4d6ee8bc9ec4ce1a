"""Discrete Green's function tables Gt^m_{t s} = G^m(t; s) DeltaV_s (Sec. 4.2).

G^m(.; s) solves (nabla^2 + lambda^m) G^m = 4 pi G delta_s / DeltaV_s
(Eqs. DGF_fft_sph, DGF_fft_cyl) with DeltaV_s the 3-D volume of the source
cell.  Sources and targets are the boundary ghost cells of the domain
(``james.boundary_points``).  Two constructions, as the paper describes:

* Auxiliary grid (Moon et al. construction, n_pad = 16): a window of
  (2 n_pad + 1)^2 cells of the same grid law centred on the source, Dirichlet
  data from Eq. DGF_bc_sph / DGF_bc_cyl on the ring of ghost cells around the
  window, solved exactly.  Targets inside the window take the solved value;
  all other targets take the closed-form mode sum.  The window is clipped at
  a face of zero area (r = 0 or a pole), where no boundary data is needed.
* Extended domain (logarithmic radial grids with r_out / r_in >= 100): the
  domain grows by n_r - 16 radial cells inwards and 16 outwards; a bounded
  theta or z direction grows by n_t / 2 cells on each side.  The outer, upper
  and lower ghosts carry the closed-form Dirichlet data, the inner radial face
  the closed-form radial derivative as a prescribed (Neumann) flux.  The system
  is solved exactly for every source.

Both solves are sparse direct factorisations: the table is the exact
solution of the discrete problem that each construction defines.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import green, operator
from .geometry import LOG, SPHERICAL, Plane
from .james import boundary_points

N_PAD = 16
EXTENDED_RATIO = 100.0
FACE_TOL = 1e-12


def uses_extended_domain(plane):
    lo, hi, n, spacing = plane.r.law
    return spacing == LOG and hi / lo >= EXTENDED_RATIO and plane.n_r >= 32


def dgf(plane, modes=None):
    """Gt[k, t, s] for the modes in ``modes`` (default: all)."""
    modes = list(range(plane.n_modes)) if modes is None else list(modes)
    if uses_extended_domain(plane):
        return extended_dgf(plane, modes)
    return aux_dgf(plane, modes)


def _solve_real(lu, b):
    return lu.solve(np.ascontiguousarray(b))


# ---------------------------------------------------------------------------
# extended domain
# ---------------------------------------------------------------------------
def extended_plane(plane):
    """The extended plane and the index offsets (o_r, o_t) that map an
    original cell (i, j) to the extended cell (i + o_r, j + o_t)."""
    n_r, n_t = plane.n_r, plane.n_t
    o_r = n_r - 16
    r_ext = plane.r.cells(1 - o_r, n_r + 16)
    bounded_t = plane.geometry != SPHERICAL or plane.has_lower() or plane.has_upper()
    if bounded_t:
        o_t = n_t // 2
        t_ext = plane.t.cells(1 - o_t, n_t + o_t)
    else:
        o_t = 0
        t_ext = plane.t.cells(1, n_t)
    return Plane(plane.geometry, r_ext, t_ext, plane.n_phi, plane.G), o_r, o_t


def inner_flux_coefficient(ext):
    """A_{1/2} / DeltaV_1 of the first extended cell (spherical 3 r^2/(r^3 - r^3),
    cylindrical 2 R/(R^2 - R^2))."""
    F = ext.r.F
    if ext.geometry == SPHERICAL:
        return 3.0 * F[1] ** 2 / (F[2] ** 3 - F[1] ** 3)
    return 2.0 * F[1] / (F[2] ** 2 - F[1] ** 2)


def extended_dgf(plane, modes):
    ext, o_r, o_t = extended_plane(plane)
    pts = boundary_points(plane)
    nb = len(pts)
    nre, nte = ext.n_r, ext.n_t
    N, G = plane.n_phi, plane.G
    xr, xt = ext.r.x, ext.t.x
    src = [(i + o_r, j + o_t) for _, i, j in pts]              # extended indices
    src_x = np.array([xr[i] for i, _ in src])
    src_y = np.array([xt[j] for _, j in src])
    dV = np.array([plane.dV[i, j] for _, i, j in pts])
    # Dirichlet ghosts of the extended plane (outer radial; bounded t edges)
    ghosts = [(nre + 1, j) for j in range(1, nte + 1)]
    if ext.has_lower():
        ghosts += [(i, 0) for i in range(1, nre + 1)]
    if ext.has_upper():
        ghosts += [(i, nte + 1) for i in range(1, nre + 1)]
    gx = np.array([xr[i] for i, _ in ghosts])
    gy = np.array([xt[j] for _, j in ghosts])
    # closed-form data, all modes: [ghost, source, m] and [row, source, m]
    gval = green.mode_sum(ext.geometry, N, G, gx[:, None], gy[:, None], src_x[None, :], src_y[None, :])
    rows = np.arange(1, nte + 1)
    dval = green.mode_sum_dr(ext.geometry, N, G, ext.r.F[1], xt[rows][:, None],
                             src_x[None, :], src_y[None, :])
    cN = inner_flux_coefficient(ext)
    aW1 = ext.aW[1]
    ext.aW[1] = 0.0                                             # Neumann inner face
    out = np.zeros((len(modes), nb, nb))
    for k, m in enumerate(modes):
        lu = spla.splu(operator.matrix(ext, m).tocsc())
        B = np.zeros((nre, nte, nb))
        for s, (i, j) in enumerate(src):
            B[i - 1, j - 1, s] += 4.0 * np.pi * G / dV[s]
        g = np.zeros((nre + 2, nte + 2, nb))
        for q, (i, j) in enumerate(ghosts):
            g[i, j] = gval[q, :, m]
        B -= operator.ghost_rhs(ext, g)
        B[0, :, :] += cN * dval[:, :, m]
        X = operator.from_vec(_solve_real(lu, operator.to_vec(B)), nre, nte)
        for t, (i, j) in enumerate(src):
            out[k, t, :] = X[i - 1, j - 1, :] * dV
    ext.aW[1] = aW1
    return out


# ---------------------------------------------------------------------------
# auxiliary grids
# ---------------------------------------------------------------------------
def _window(axis, c_src, n_dom):
    """Cells c_src-16..c_src+16 of the axis law, clipped at zero-area faces.
    Returns (c_lo, c_hi)."""
    c_lo, c_hi = c_src - N_PAD, c_src + N_PAD
    lo, hi, n, spacing = axis.law
    if axis.kind in ("r_sph", "r_cyl"):
        while True:
            f_in = axis.cells(c_lo, c_lo).F[1]
            if f_in >= -FACE_TOL:
                break
            c_lo += 1
        if c_lo > c_src - N_PAD and abs(axis.cells(c_lo, c_lo).F[1]) > FACE_TOL:
            raise ValueError("auxiliary window crosses r = 0 away from a cell face")
    elif axis.kind == "theta":
        while axis.cells(c_lo, c_lo).F[1] < -FACE_TOL:
            c_lo += 1
        while axis.cells(c_hi, c_hi).F[2] > np.pi + FACE_TOL:
            c_hi -= 1
        if (c_lo > c_src - N_PAD and abs(axis.cells(c_lo, c_lo).F[1]) > FACE_TOL) or \
           (c_hi < c_src + N_PAD and abs(axis.cells(c_hi, c_hi).F[2] - np.pi) > FACE_TOL):
            raise ValueError("auxiliary window crosses a pole away from a cell face")
    return c_lo, c_hi


def aux_dgf(plane, modes):
    pts = boundary_points(plane)
    nb = len(pts)
    N, G = plane.n_phi, plane.G
    M = len(modes)
    xr, xt = plane.r.x, plane.t.x
    px = np.array([xr[i] for _, i, _ in pts])
    py = np.array([xt[j] for _, _, j in pts])
    dV = np.array([plane.dV[i, j] for _, i, j in pts])
    out = np.zeros((M, nb, nb))
    # far field: closed form for every pair (overwritten inside windows)
    with np.errstate(divide="ignore", invalid="ignore"):
        for s in range(nb):       # self and near pairs are replaced below
            far = green.mode_sum(plane.geometry, N, G, px, py, px[s], py[s])
            out[:, :, s] = (far[:, modes] * dV[s]).T
    for s, (_, i_s, j_s) in enumerate(pts):
        i_lo, i_hi = _window(plane.r, i_s, plane.n_r)
        j_lo, j_hi = _window(plane.t, j_s, plane.n_t)
        win = Plane(plane.geometry, plane.r.cells(i_lo, i_hi), plane.t.cells(j_lo, j_hi),
                    N, G)
        nw_r, nw_t = win.n_r, win.n_t
        wx, wy = win.r.x, win.t.x
        ring = [(nw_r + 1, j) for j in range(1, nw_t + 1)]     # ring sides with area
        if win.has_inner():
            ring += [(0, j) for j in range(1, nw_t + 1)]
        if win.has_lower():
            ring += [(i, 0) for i in range(1, nw_r + 1)]
        if win.has_upper():
            ring += [(i, nw_t + 1) for i in range(1, nw_r + 1)]
        rx = np.array([wx[i] for i, _ in ring])
        ry = np.array([wy[j] for _, j in ring])
        gring = green.mode_sum(plane.geometry, N, G, rx, ry, px[s], py[s])
        inside = [t for t, (_, i, j) in enumerate(pts) if i_lo <= i <= i_hi and j_lo <= j <= j_hi]
        for k, m in enumerate(modes):
            g = np.zeros((nw_r + 2, nw_t + 2))
            for q, (i, j) in enumerate(ring):
                g[i, j] = gring[q, m]
            b = -operator.ghost_rhs(win, g)
            b[i_s - i_lo, j_s - j_lo] += 4.0 * np.pi * G / dV[s]
            x = spla.spsolve(operator.matrix(win, m).tocsc(), operator.to_vec(b))
            X = operator.from_vec(x, nw_r, nw_t)
            for t in inside:
                _, i, j = pts[t]
                out[k, t, s] = X[i - i_lo, j - j_lo] * dV[s]
    return out
