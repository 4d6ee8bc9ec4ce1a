"""The per-mode 2-D Helmholtz operator L_m (Eqs. helmholz_sph, helmholz_cyl).

Ghost cells carry Dirichlet data: ``apply`` takes the field with its ghost
ring, ``matrix`` is the operator with all ghost values zero (their
contribution belongs to the right-hand side, see ``ghost_rhs``).  Unknowns are
numbered ``(j-1) * n_r + (i-1)`` (radial index fastest).
"""
import numpy as np
import scipy.sparse as sp


def apply(plane, m, u):
    """L_m u on the domain cells. ``u`` has shape (n_r+2, n_t+2) incl. ghosts."""
    nr, nt = plane.n_r, plane.n_t
    i = slice(1, nr + 1)
    j = slice(1, nt + 1)
    c = u[i, j]
    out = (plane.aE[i][:, None] * (u[2:nr + 2, j] - c)
           + plane.aW[i][:, None] * (u[0:nr, j] - c)
           + plane.P[i][:, None] * (plane.aN[j][None, :] * (u[i, 2:nt + 2] - c)
                                    + plane.aS[j][None, :] * (u[i, 0:nt] - c))
           - plane.s2(m) * plane.Q[i][:, None] * plane.T[j][None, :] * c)
    return out


def with_ghosts(plane, interior, ghost=None):
    """Embed an (n_r, n_t) array into the ghost-ring layout (ghosts zero or
    taken from ``ghost``)."""
    shape = (plane.n_r + 2, plane.n_t + 2) + interior.shape[2:]
    u = np.zeros(shape, dtype=interior.dtype) if ghost is None else ghost.copy()
    u[1:-1, 1:-1] = interior
    return u


def matrix(plane, m):
    """Sparse L_m with zero ghost values, CSR, size (n_r n_t)^2."""
    nr, nt = plane.n_r, plane.n_t
    ii, jj = np.meshgrid(np.arange(1, nr + 1), np.arange(1, nt + 1), indexing="ij")
    row = (jj - 1) * nr + (ii - 1)
    d = plane.diag(m)
    rows, cols, vals = [row.ravel()], [row.ravel()], [d.ravel()]
    aE = np.broadcast_to(plane.aE[1:nr + 1][:, None], (nr, nt))
    aW = np.broadcast_to(plane.aW[1:nr + 1][:, None], (nr, nt))
    aN = plane.P[1:nr + 1][:, None] * plane.aN[1:nt + 1][None, :]
    aS = plane.P[1:nr + 1][:, None] * plane.aS[1:nt + 1][None, :]
    for coef, di, dj in ((aE, 1, 0), (aW, -1, 0), (aN, 0, 1), (aS, 0, -1)):
        ni, nj = ii + di, jj + dj
        ok = (ni >= 1) & (ni <= nr) & (nj >= 1) & (nj <= nt)
        rows.append(row[ok])
        cols.append(((nj - 1) * nr + (ni - 1))[ok])
        vals.append(coef[ok])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nr * nt, nr * nt))


def ghost_rhs(plane, g):
    """Contribution of Dirichlet ghost data ``g`` (full ghost-ring array,
    interior ignored) to L_m u, i.e. L_m u = matrix @ u + ghost_rhs."""
    nr, nt = plane.n_r, plane.n_t
    out = np.zeros((nr, nt) + g.shape[2:], dtype=g.dtype)
    P = plane.P[1:nr + 1].reshape((nr,) + (1,) * (g.ndim - 2))
    out[0] += plane.aW[1] * g[0, 1:nt + 1]
    out[-1] += plane.aE[nr] * g[nr + 1, 1:nt + 1]
    out[:, 0] += P * plane.aS[1] * g[1:nr + 1, 0]
    out[:, -1] += P * plane.aN[nt] * g[1:nr + 1, nt + 1]
    return out


def to_vec(a):
    """(n_r, n_t, ...) -> (n_r n_t, ...) with the radial index fastest."""
    return a.transpose((1, 0) + tuple(range(2, a.ndim))).reshape((-1,) + a.shape[2:])


def from_vec(v, nr, nt):
    return v.reshape((nt, nr) + v.shape[1:]).transpose((1, 0) + tuple(range(2, v.ndim + 1)))
