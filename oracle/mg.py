"""The paper's per-mode multigrid (Sec. 3, App. A), FP64, written plainly.

Readings fixed here (the paper leaves them open):
* Level hierarchy: factor-two coarsening of both axes while the shorter one
  has more than 16 cells, or more than 4 cells and the plane more than 1024
  cells; coarse faces are every other fine face (Sec. 5.2 power-of-two
  rule); the coarse operator is re-discretised from those faces.  The paper
  leaves the size of the directly solved coarsest level open; on strongly
  stretched logarithmic grids it sets the m = 0 convergence rate (256 x 128,
  r_out/r_in = 400, tol 1e-8: 40 V-cycles with an 8 x 4 coarsest level, 26
  with 16 x 8, 21 with 32 x 16, 16 with 64 x 32, the count App. B quotes).
* Coarsest level: exact (sparse direct) solve; Sec. 3.3 allows a direct
  solver.
* Smoother (Sec. 3.2, Algorithm 1): one smoothing cycle relaxes all radial
  lines, then all polar / vertical lines (the order the text gives).  Lines
  are relaxed in zebra order (Sec. 5.2): lines with even 0-based index first,
  then odd.  Each line is relaxed by N_SOR SOR sweeps in even-odd order (even
  0-based positions first), with the right-hand side of the line (source
  minus the other direction's couplings) frozen for the line.  Defaults
  nu1 = nu2 = 2 smoothing cycles, N_SOR = 2.
* Per-line relaxation parameter: App. A, Eq. omega_opt_mu with mu_1 from the
  WKB Rayleigh quotient (p = 1) on the line's tridiagonal system, whose
  diagonal is the full 2-D diagonal of L_m (including lambda^m); x_0 and
  x_{N+1} are the ghost centres.
* Restriction: Eq. restriction_sph / restriction_weight_cyl as the text
  and the figure describe it: each fine defect is weighted by the area S of
  its overlap with the coarse cell in the (xi, eta) plane, which is the fine
  cell itself, S = |xi_{i+1/2} - xi_{i-1/2}| |eta_{j+1/2} - eta_{j-1/2}|,
  xi = r^2, eta = theta (spherical) or xi = R, eta = z (cylindrical).  The
  printed formula measures from the cell centres instead; taken literally it
  makes the m = 0 mode diverge on logarithmic grids, against App. B.
* Prolongation: Eq. prolongation_sph / prolongation_weight_cyl, bilinear in
  (xi, eta) from the four surrounding coarse centres.  A missing coarse
  neighbour is the coarse ghost: 0 next to a Dirichlet side, (-1)^m times its
  neighbour across a pole or the cylinder axis (Sec. 4.2 parity relation),
  and its neighbour itself across a Neumann face or the spherical origin.
* Convergence (App. B): the volume-weighted L2 norm of the defect of each
  real component, relative to that of the right-hand side (the defect of the
  zero initial guess), floored at ``floor``; a plane is done when both
  components meet it.
* Cycle: the V-cycle of Sec. 3 (gamma = 1).  gamma > 1 is not the paper's:
  a level whose coarser neighbour is not the coarsest level runs gamma
  cycles per visit on its coarse equation, each starting from the previous
  correction (gamma = 2: the textbook W-cycle; the coarsest level, solved
  exactly, is visited once).  It exists to study where the low modes lose
  convergence; no kernel runs it.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import operator
from .geometry import SPHERICAL

ZERO, PARITY, EVEN = 0, 1, 2


class Level:
    def __init__(self, plane, neumann_inner):
        self.plane = plane
        self.neumann_inner = neumann_inner
        if neumann_inner:
            plane.aW[1] = 0.0
        g = plane.geometry
        if neumann_inner:
            self.ghost_L = EVEN
        elif not plane.has_inner():
            self.ghost_L = PARITY if g != SPHERICAL else EVEN
        else:
            self.ghost_L = ZERO
        self.ghost_R = ZERO
        self.ghost_B = ZERO if plane.has_lower() else PARITY
        self.ghost_T = ZERO if plane.has_upper() else PARITY
        if g == SPHERICAL:
            self.xi, self.eta = plane.r.x ** 2, plane.t.x
        else:
            self.xi, self.eta = plane.r.x, plane.t.x


class Hierarchy:
    def __init__(self, plane, neumann_inner=False, min_cells=16, nu1=2, nu2=2, n_sor=2,
                 max_coarse=1024, gamma=1):
        planes = [plane]
        while True:
            nr, nt = planes[-1].n_r, planes[-1].n_t
            if not (min(nr, nt) > min_cells or (min(nr, nt) > 4 and nr * nt > max_coarse)):
                break
            planes.append(planes[-1].coarsen())
        self.levels = [Level(p, neumann_inner) for p in planes]
        self.nu1, self.nu2, self.n_sor, self.gamma = nu1, nu2, n_sor, gamma
        self._omega = {}
        self._coarse = {}

    # -- App. A ---------------------------------------------------------------
    def omega(self, lev, m):
        key = (lev, m)
        if key not in self._omega:
            p = self.levels[lev].plane
            d = p.diag(m)
            nr, nt = p.n_r, p.n_t
            om_r = np.array([wkb_omega(p.aW[1:nr + 1], p.aE[1:nr + 1], d[:, j], p.r.x)
                             for j in range(nt)])
            om_t = np.array([wkb_omega(p.P[i + 1] * p.aS[1:nt + 1], p.P[i + 1] * p.aN[1:nt + 1],
                                       d[i, :], p.t.x) for i in range(nr)])
            self._omega[key] = (om_r, om_t)
        return self._omega[key]

    def coarse_lu(self, m):
        if m not in self._coarse:
            p = self.levels[-1].plane
            self._coarse[m] = spla.splu(operator.matrix(p, m).tocsc())
        return self._coarse[m]

    # -- Sec. 3.2 -------------------------------------------------------------
    def smooth(self, lev, m, u, f, cycles):
        """``cycles`` alternating line-smoothing cycles on u (n_r+2, n_t+2),
        zero ghosts, complex; f (n_r, n_t)."""
        p = self.levels[lev].plane
        nr, nt = p.n_r, p.n_t
        d = p.diag(m)
        om_r, om_t = self.omega(lev, m)
        aE, aW, P, aN, aS = p.aE, p.aW, p.P, p.aN, p.aS
        for _ in range(cycles):
            # radial lines (constant j), zebra over j
            for color in (0, 1):
                js = np.arange(1 + color, nt + 1, 2)
                fl = f[:, js - 1] - P[1:nr + 1, None] * (aN[js] * u[1:nr + 1, js + 1]
                                                         + aS[js] * u[1:nr + 1, js - 1])
                w = om_r[js - 1]
                for _ in range(self.n_sor):
                    for par in (0, 1):
                        ii = np.arange(1 + par, nr + 1, 2)
                        tmp = (fl[ii - 1] - aE[ii, None] * u[ii + 1][:, js]
                               - aW[ii, None] * u[ii - 1][:, js]) / d[np.ix_(ii - 1, js - 1)]
                        u[np.ix_(ii, js)] = (1.0 - w) * u[np.ix_(ii, js)] + w * tmp
            # polar / vertical lines (constant i), zebra over i
            for color in (0, 1):
                ii = np.arange(1 + color, nr + 1, 2)
                gl = f[ii - 1, :] - (aE[ii, None] * u[ii + 1, 1:nt + 1]
                                     + aW[ii, None] * u[ii - 1, 1:nt + 1])
                w = om_t[ii - 1][:, None]
                for _ in range(self.n_sor):
                    for par in (0, 1):
                        js = np.arange(1 + par, nt + 1, 2)
                        tmp = (gl[:, js - 1] - P[ii, None] * (aN[js] * u[ii][:, js + 1]
                                                              + aS[js] * u[ii][:, js - 1])) \
                            / d[np.ix_(ii - 1, js - 1)]
                        u[np.ix_(ii, js)] = (1.0 - w) * u[np.ix_(ii, js)] + w * tmp
        return u

    # -- Sec. 3.1 -------------------------------------------------------------
    def residual(self, lev, m, u, f):
        return f - operator.apply(self.levels[lev].plane, m, u)

    def restrict(self, lev, r):
        """Fine defect r (n_r, n_t) at ``lev`` -> coarse (n_r/2, n_t/2)."""
        F, C = self.levels[lev], self.levels[lev + 1]
        ncr, nct = C.plane.n_r, C.plane.n_t
        p = F.plane
        if p.geometry == SPHERICAL:
            a = np.abs(p.r.F[2:p.n_r + 2] ** 2 - p.r.F[1:p.n_r + 1] ** 2)
        else:
            a = np.abs(p.r.F[2:p.n_r + 2] - p.r.F[1:p.n_r + 1])
        b = np.abs(p.t.F[2:p.n_t + 2] - p.t.F[1:p.n_t + 1])
        num = 0.0
        den = 0.0
        for da in (0, 1):
            for db in (0, 1):
                S = a[da::2][:, None] * b[db::2][None, :]
                num = num + S * r[da::2, db::2]
                den = den + S
        return num / den

    def _coarse_with_ghosts(self, C, m, e):
        ncr, nct = C.plane.n_r, C.plane.n_t
        g = np.zeros((ncr + 2, nct + 2), dtype=e.dtype)
        g[1:-1, 1:-1] = e
        sgn = (-1.0) ** m
        for rule, dst, src in ((C.ghost_L, (0, slice(1, nct + 1)), (1, slice(1, nct + 1))),
                               (C.ghost_R, (ncr + 1, slice(1, nct + 1)), (ncr, slice(1, nct + 1))),
                               (C.ghost_B, (slice(1, ncr + 1), 0), (slice(1, ncr + 1), 1)),
                               (C.ghost_T, (slice(1, ncr + 1), nct + 1), (slice(1, ncr + 1), nct))):
            if rule == PARITY:
                g[dst] = sgn * g[src]
            elif rule == EVEN:
                g[dst] = g[src]
        return g

    def prolong(self, lev, m, e):
        """Coarse correction e (n_r/2, n_t/2) at lev+1 -> fine (n_r, n_t) at lev."""
        F, C = self.levels[lev], self.levels[lev + 1]
        nr, nt = F.plane.n_r, F.plane.n_t
        g = self._coarse_with_ghosts(C, m, e)
        i = np.arange(1, nr + 1)
        j = np.arange(1, nt + 1)
        I1 = np.where(i % 2 == 1, (i + 1) // 2 - 1, (i + 1) // 2)
        J1 = np.where(j % 2 == 1, (j + 1) // 2 - 1, (j + 1) // 2)
        I2, J2 = I1 + 1, J1 + 1
        xf, yf = F.xi[i], F.eta[j]
        wx1 = np.abs(C.xi[I2] - xf) / np.abs(C.xi[I2] - C.xi[I1])    # weight of I1
        wx2 = np.abs(C.xi[I1] - xf) / np.abs(C.xi[I2] - C.xi[I1])
        wy1 = np.abs(C.eta[J2] - yf) / np.abs(C.eta[J2] - C.eta[J1])
        wy2 = np.abs(C.eta[J1] - yf) / np.abs(C.eta[J2] - C.eta[J1])
        return (wx1[:, None] * wy1[None, :] * g[np.ix_(I1, J1)]
                + wx2[:, None] * wy1[None, :] * g[np.ix_(I2, J1)]
                + wx1[:, None] * wy2[None, :] * g[np.ix_(I1, J2)]
                + wx2[:, None] * wy2[None, :] * g[np.ix_(I2, J2)])

    # -- V-cycle ----------------------------------------------------------------
    def vcycle(self, lev, m, u, f):
        """One V-cycle (W-cycle for gamma = 2) on L_m u = f at ``lev``; u with
        ghosts, modified in place."""
        p = self.levels[lev].plane
        if lev == len(self.levels) - 1:
            lu = self.coarse_lu(m)
            b = operator.to_vec(f)
            x = lu.solve(np.ascontiguousarray(b.real)) + 1j * lu.solve(np.ascontiguousarray(b.imag))
            u[1:-1, 1:-1] = operator.from_vec(x, p.n_r, p.n_t)
            return u
        self.smooth(lev, m, u, f, self.nu1)
        r = self.residual(lev, m, u, f)
        fc = self.restrict(lev, r)
        C = self.levels[lev + 1].plane
        ec = np.zeros((C.n_r + 2, C.n_t + 2), dtype=u.dtype)
        # the coarsest level is solved exactly: one visit is enough
        visits = self.gamma if lev + 2 < len(self.levels) else 1
        for _ in range(visits):
            self.vcycle(lev + 1, m, ec, fc)
        u[1:-1, 1:-1] += self.prolong(lev, m, ec[1:-1, 1:-1])
        self.smooth(lev, m, u, f, self.nu2)
        return u

    def norm(self, r):
        """Volume-weighted L2 norms of the real and imaginary parts."""
        w = self.levels[0].plane.volume_weights()
        ws = w.sum()
        return (np.sqrt((w * r.real**2).sum() / ws), np.sqrt((w * r.imag**2).sum() / ws))

    def solve(self, m, f, tol, floor=0.0, max_cycles=100, u0=None):
        """Iterate V-cycles from u0 (default 0) until the criterion holds.
        Returns (u interior, cycles, history of the defect norms)."""
        p = self.levels[0].plane
        u = np.zeros((p.n_r + 2, p.n_t + 2), dtype=complex)
        if u0 is not None:
            u[1:-1, 1:-1] = u0
        nf = self.norm(f)
        thr = (tol * max(nf[0], floor), tol * max(nf[1], floor))
        hist = []
        cycles = 0
        while True:
            nr_ = self.norm(self.residual(0, m, u, f))
            hist.append(nr_)
            if (nr_[0] <= thr[0] and nr_[1] <= thr[1]) or cycles >= max_cycles:
                break
            self.vcycle(0, m, u, f)
            cycles += 1
        return u[1:-1, 1:-1], cycles, hist


def wkb_omega(a, c, b, x):
    """App. A: omega = 2 / (1 + sqrt(1 - mu_1^2)) for the tridiagonal system
    a_j u_{j-1} + b_j u_j + c_j u_{j+1} = f_j (j = 1..N) on points x_0..x_{N+1}
    (x_0, x_{N+1} the boundary points), with
    mu_1 = sum (a_j + c_j) cos(pi delta_j / L) w_j / sum b_j w_j,
    w_j = sin^2(pi (x_j - x_0) / L), delta_j = x_j - x_{j-1}, L = x_{N+1} - x_0."""
    N = len(b)
    L = x[N + 1] - x[0]
    xj = x[1:N + 1]
    delta = x[1:N + 1] - x[0:N]
    w = np.sin(np.pi * (xj - x[0]) / L) ** 2
    mu = np.sum((a + c) * np.cos(np.pi * delta / L) * w) / np.sum(b * w)
    rho = min(abs(mu), 1.0)
    return 2.0 / (1.0 + np.sqrt(1.0 - rho**2))
