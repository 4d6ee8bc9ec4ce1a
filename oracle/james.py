"""James' screening-mass method per Fourier mode and the seven-step solve.

* Boundary points (Sec. 4.1): the ghost cells next to the domain, in the
  order L (i = 0), R (i = n_r+1), B (j = 0), T (j = n_t+1).  A side whose
  face has zero area (r_in = 0, or a polar face at theta = 0, pi) is not a
  boundary: the polar ghosts obey the parity condition of Eq. polar_bc and
  carry no flux.
* Screening mass (Eqs. charge_sph, charge_cyl): the finite-volume Laplacian
  evaluated at the ghost cell with Psi = 0 outside the domain, divided by
  4 pi G.  Only the neighbour in the first domain cell contributes, so
  sigma = coef * Psi_adjacent with coef the ghost cell's own coupling to that
  neighbour.  The 1/(4 pi G) that Eq. charge_cyl omits is applied in both
  geometries (Eq. screen_mass defines sigma that way).
* Boundary potential (Eqs. theta_left .. theta_top):
  Theta^m_t = sum_s Gt^m_{t s} sigma^m_s with Gt = G^m * DeltaV_s.
* Solve (Sec. 5.1 steps 2-7): forward DFT, L_m Psi = 4 pi G rho^m with zero
  ghosts, sigma, Theta, L_m Phi = 4 pi G rho^m with ghosts -Theta, inverse DFT.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import dft, operator
from .geometry import SPHERICAL


def boundary_points(plane):
    """List of (side, i_ghost, j_ghost) in L, R, B, T order."""
    nr, nt = plane.n_r, plane.n_t
    pts = []
    if plane.has_inner():
        pts += [("L", 0, j) for j in range(1, nt + 1)]
    pts += [("R", nr + 1, j) for j in range(1, nt + 1)]
    if plane.has_lower():
        pts += [("B", i, 0) for i in range(1, nr + 1)]
    if plane.has_upper():
        pts += [("T", i, nt + 1) for i in range(1, nr + 1)]
    return pts


def adjacent(side, i, j):
    """Domain cell next to a boundary ghost."""
    return {"L": (1, j), "R": (i - 1, j), "B": (i, 1), "T": (i, j - 1)}[side]


def screening_coefficients(plane):
    """Per boundary point: sigma = coef * Psi(adjacent) (Eqs. charge_sph/cyl)."""
    out = []
    for side, i, j in boundary_points(plane):
        if side == "L":
            c = plane.aE[0]                        # ghost cell 0 -> cell 1
        elif side == "R":
            c = plane.aW[plane.n_r + 1]            # ghost cell n_r+1 -> cell n_r
        elif side == "B":
            c = plane.P[i] * plane.aN[0]           # ghost row 0 -> row 1
        else:
            c = plane.P[i] * plane.aS[plane.n_t + 1]
        out.append(c / (4.0 * np.pi * plane.G))
    return np.array(out)


def ghost_couplings(plane):
    """Per boundary point: coefficient of the ghost value in L_m at the
    adjacent domain cell."""
    out = []
    for side, i, j in boundary_points(plane):
        if side == "L":
            c = plane.aW[1]
        elif side == "R":
            c = plane.aE[plane.n_r]
        elif side == "B":
            c = plane.P[i] * plane.aS[1]
        else:
            c = plane.P[i] * plane.aN[plane.n_t]
        out.append(c)
    return np.array(out)


def screening_mass(plane, psi):
    """psi (n_r, n_t, ...) complex per mode -> sigma (nb, ...)."""
    coef = screening_coefficients(plane)
    vals = []
    for (side, i, j), c in zip(boundary_points(plane), coef):
        ia, ja = adjacent(side, i, j)
        vals.append(c * psi[ia - 1, ja - 1])
    return np.array(vals)


def boundary_potential(gt, sigma):
    """Theta[m, t] = sum_s gt[m, t, s] sigma[m, s]."""
    return np.einsum("mts,ms->mt", gt, sigma)


def ghost_values(plane, values):
    """Full ghost-ring array with ``values`` (nb, ...) at the boundary points."""
    g = np.zeros((plane.n_r + 2, plane.n_t + 2) + values.shape[1:], dtype=values.dtype)
    for (side, i, j), v in zip(boundary_points(plane), values):
        g[i, j] = v
    return g


def solve_mode(plane, m, f_m, gt_m):
    """Steps 3-6 of Sec. 5.1 for one azimuthal mode: f_m (n_r, n_t) complex
    right-hand side 4 pi G rho^m, gt_m the mode's DGF table [t, s].  Returns
    (psi^m, sigma^m, theta^m, phi^m)."""
    nr, nt = plane.n_r, plane.n_t
    lu = spla.splu(operator.matrix(plane, m).tocsc())
    b = operator.to_vec(f_m)
    x = lu.solve(np.ascontiguousarray(b.real)) + 1j * lu.solve(np.ascontiguousarray(b.imag))
    psi = operator.from_vec(x, nr, nt)                  # step 3
    sigma = screening_mass(plane, psi)                  # step 4
    theta = gt_m @ sigma                                # step 5
    g = ghost_values(plane, -theta)
    b2 = operator.to_vec(f_m - operator.ghost_rhs(plane, g))
    x = lu.solve(np.ascontiguousarray(b2.real)) + 1j * lu.solve(np.ascontiguousarray(b2.imag))
    return psi, sigma, theta, operator.from_vec(x, nr, nt)   # step 6


def solve(plane, rho, gt, return_parts=False):
    """Seven-step solve (Sec. 5.1).  rho: (n_r, n_t, n_phi) FP64 at the cell
    centres; gt: DGF table [m, t, s].  Returns phi (n_r, n_t, n_phi)."""
    N = plane.n_phi
    M = N // 2 + 1
    rho_hat = dft.forward(rho)                          # step 2
    f = 4.0 * np.pi * plane.G * rho_hat                 # (n_r, n_t, M)
    psi = np.zeros_like(f)
    phi_hat = np.zeros_like(f)
    sigma = np.zeros((len(boundary_points(plane)), M), dtype=complex)
    theta = np.zeros_like(sigma)
    for m in range(M):
        psi[:, :, m], sigma[:, m], theta[:, m], phi_hat[:, :, m] = solve_mode(plane, m, f[:, :, m], gt[m])
    phi = dft.inverse(phi_hat, N)                        # step 7
    if return_parts:
        return phi, dict(rho_hat=rho_hat, f=f, psi=psi, sigma=sigma, theta=theta,
                         phi_hat=phi_hat)
    return phi
