"""Finite-volume geometry of one (r, theta) or (R, z) plane.

Sec. 2.1 (Eq. poisson_discrete) gives the general finite-volume Laplacian;
Sec. 2.1.1 specialises it to spherical coordinates (Eqs. cell_centers_sph,
vol_sph, surface_sph and the directional operators nabla^2_r, nabla^2_theta,
nabla^2_phi with the factors R_i and T_j); Sec. 2.1.2 does the same for
cylindrical coordinates (nabla^2_R, nabla^2_phi, nabla^2_z with W_i).

Conventions used throughout the oracle
--------------------------------------
* An axis has ``n`` domain cells and one ghost cell on each side.  Cell ``c``
  (``c = 0 .. n+1``; 0 and n+1 are the ghosts) spans the faces
  ``F[c] .. F[c+1]``; ``F`` has ``n + 3`` entries.
* Ghost faces continue the spacing law of the axis (uniform: constant step,
  logarithmic: constant ratio) and ghost centres use the same centroid formula
  as domain cells.
* A face of zero area (a radial face at r = 0, a polar face at theta = 0 or
  pi) carries no flux: its coefficient is exactly zero.
* The plane operator acting on mode m is

    L_m u = aE_i (u_{i+1,j} - u_ij) + aW_i (u_{i-1,j} - u_ij)
          + P_i [ aN_j (u_{i,j+1} - u_ij) + aS_j (u_{i,j-1} - u_ij) ]
          - Q_i T_j s_m^2 u_ij,     s_m = sin(m pi / N_phi) / (pi / N_phi)

  spherical:   aE/aW from nabla^2_r, aN/aS from nabla^2_theta without R_i,
               P = Q = R_i, T = T_j              (Eq. eigenv_sph)
  cylindrical: aE/aW from nabla^2_R, aN/aS from nabla^2_z,
               P = 1, Q = W_i, T = 1             (Eq. eigenv_cyl)
"""
import numpy as np

SPHERICAL, CYLINDRICAL = 0, 1
UNIFORM, LOG = 0, 1
POLE_TOL = 1e-12


def spacing_faces(lo, hi, n, spacing, k_first, k_last):
    # face number k bounds cells k and k+1 (cell c spans faces c-1 .. c)
    """Faces number k = k_first..k_last of the law that puts face 0 at ``lo``
    and face n at ``hi`` (uniform: lo + k (hi-lo)/n; log: lo (hi/lo)^(k/n))."""
    k = np.arange(k_first, k_last + 1, dtype=np.float64)
    if spacing == LOG:
        if lo <= 0.0:
            raise ValueError("logarithmic spacing needs a positive lower bound")
        return lo * (hi / lo) ** (k / n)
    return lo + k * ((hi - lo) / n)


class Axis:
    """One coordinate direction; ``kind`` is 'r_sph', 'r_cyl', 'theta' or 'z'."""

    def __init__(self, kind, faces, spacing=UNIFORM):
        self.kind = kind
        self.spacing = spacing
        self.F = np.asarray(faces, dtype=np.float64)
        self.n = len(self.F) - 3
        F0, F1 = self.F[:-1], self.F[1:]
        if kind == "r_sph":      # Eq. cell_centers_sph, first line
            self.x = 0.75 * (F1**4 - F0**4) / (F1**3 - F0**3)
        elif kind == "r_cyl":    # Sec. 2.1.2, R_i
            self.x = (2.0 / 3.0) * (F1**3 - F0**3) / (F1**2 - F0**2)
        elif kind == "theta":    # Eq. cell_centers_sph, second line
            self.x = ((np.sin(F1) - np.sin(F0) + F0 * np.cos(F0) - F1 * np.cos(F1))
                      / (np.cos(F0) - np.cos(F1)))
        elif kind == "z":
            self.x = 0.5 * (F0 + F1)
        else:
            raise ValueError(kind)

    @classmethod
    def make(cls, kind, n, lo, hi, spacing=UNIFORM):
        ax = cls(kind, spacing_faces(lo, hi, n, spacing, -1, n + 1), spacing)
        ax.law = (lo, hi, n, spacing)
        return ax

    def cells(self, c_first, c_last):
        """Axis made of the cells c_first..c_last (original numbering, 0 and
        n+1 being the ghosts) of the spacing law this axis was made from, plus
        one ghost cell on each side of that range."""
        lo, hi, n, spacing = self.law
        ax = Axis(self.kind, spacing_faces(lo, hi, n, spacing, c_first - 2, c_last + 1), spacing)
        ax.law = self.law
        return ax

    def sin_faces(self):
        """sin of the polar faces, exactly zero on a pole."""
        s = np.sin(self.F)
        s[np.abs(self.F) < POLE_TOL] = 0.0
        s[np.abs(self.F - np.pi) < POLE_TOL] = 0.0
        return s


class Plane:
    """Geometry and operator tables of one 2-D mode plane.

    ``r`` is the radial axis, ``t`` the polar (spherical) or vertical
    (cylindrical) axis; ``n_phi`` the number of azimuthal cells of the 3-D
    grid (Delta phi = 2 pi / n_phi).  ``G`` is the gravitational constant.
    """

    def __init__(self, geometry, r_axis, t_axis, n_phi, G=1.0):
        self.geometry = geometry
        self.r, self.t = r_axis, t_axis
        self.n_r, self.n_t = r_axis.n, t_axis.n
        self.n_phi = n_phi
        self.n_modes = n_phi // 2 + 1
        self.G = G
        self.dphi = 2.0 * np.pi / n_phi
        self._tables()

    @classmethod
    def make(cls, geometry, n_r, n_t, n_phi, spacing, r_in, r_out,
             t_min=None, t_max=None, G=1.0):
        if geometry == SPHERICAL:
            t_min = 0.0 if t_min is None else t_min
            t_max = np.pi if t_max is None else t_max
            r = Axis.make("r_sph", n_r, r_in, r_out, spacing)
            t = Axis.make("theta", n_t, t_min, t_max)
        else:
            half = 0.5 * (r_out - r_in)
            t_min = -half if t_min is None else t_min
            t_max = half if t_max is None else t_max
            r = Axis.make("r_cyl", n_r, r_in, r_out, spacing)
            t = Axis.make("z", n_t, t_min, t_max)
        return cls(geometry, r, t, n_phi, G)

    # -- tables ---------------------------------------------------------
    def _tables(self):
        Fr, xr = self.r.F, self.r.x
        Ft, xt = self.t.F, self.t.x
        nr, nt = self.n_r, self.n_t
        c = np.arange(nr + 2)
        d_up = np.zeros(nr + 2)
        d_dn = np.zeros(nr + 2)
        d_up[:-1] = xr[1:] - xr[:-1]          # x_{c+1} - x_c
        d_dn[1:] = xr[1:] - xr[:-1]           # x_c - x_{c-1}
        aE = np.zeros(nr + 2)
        aW = np.zeros(nr + 2)
        Fo, Fi = Fr[c + 1], Fr[c]
        if self.geometry == SPHERICAL:
            vr = Fo**3 - Fi**3
            aE[:-1] = (3.0 * Fo**2 / vr)[:-1] / d_up[:-1]       # nabla^2_r
            aW[1:] = (3.0 * Fi**2 / vr)[1:] / d_dn[1:]
            R = 1.5 / xr * (Fo**2 - Fi**2) / vr                 # script R_i
            self.P, self.Q = R, R
            self.vol_r = vr / 3.0
        else:
            ar = Fo**2 - Fi**2
            aE[:-1] = (2.0 * Fo / ar)[:-1] / d_up[:-1]          # nabla^2_R
            aW[1:] = (2.0 * Fi / ar)[1:] / d_dn[1:]
            self.P = np.ones(nr + 2)
            self.Q = 2.0 / (xr * (Fo + Fi))                     # script W_i
            self.vol_r = ar / 2.0
        self.aE, self.aW = aE, aW

        k = np.arange(nt + 2)
        e_up = np.zeros(nt + 2)
        e_dn = np.zeros(nt + 2)
        e_up[:-1] = xt[1:] - xt[:-1]
        e_dn[1:] = xt[1:] - xt[:-1]
        aN = np.zeros(nt + 2)
        aS = np.zeros(nt + 2)
        if self.geometry == SPHERICAL:
            sF = self.t.sin_faces()
            vt = np.cos(Ft[k]) - np.cos(Ft[k + 1])
            aN[:-1] = (sF[k + 1] / vt)[:-1] / e_up[:-1]         # nabla^2_theta / R_i
            aS[1:] = (sF[k] / vt)[1:] / e_dn[1:]
            self.T = (Ft[k + 1] - Ft[k]) / (np.sin(xt) * vt)    # script T_j
            self.vol_t = vt
        else:
            dz = Ft[k + 1] - Ft[k]
            aN[:-1] = (1.0 / dz)[:-1] / e_up[:-1]               # nabla^2_z
            aS[1:] = (1.0 / dz)[1:] / e_dn[1:]
            self.T = np.ones(nt + 2)
            self.vol_t = dz
        self.aN, self.aS = aN, aS
        # 3-D cell volumes incl. ghosts (Eqs. vol_sph, vol_cyl)
        self.dV = np.outer(self.vol_r, self.vol_t) * self.dphi

    # -- helpers -----------------------------------------------------------
    def s2(self, m):
        """[sin(m pi/N)/(pi/N)]^2 (Eqs. eigenv_sph, eigenv_cyl)."""
        N = self.n_phi
        return (np.sin(m * np.pi / N) / (np.pi / N)) ** 2

    def diag(self, m):
        """Diagonal of L_m on the domain cells, shape (n_r, n_t)."""
        i = slice(1, self.n_r + 1)
        j = slice(1, self.n_t + 1)
        return (-(self.aE[i] + self.aW[i])[:, None]
                - self.P[i][:, None] * (self.aN[j] + self.aS[j])[None, :]
                - self.s2(m) * self.Q[i][:, None] * self.T[j][None, :])

    def has_inner(self):
        """Inner radial boundary present (face r_in has non-zero area)."""
        return self.r.F[1] > 0.0

    def has_lower(self):
        if self.geometry == SPHERICAL:
            return self.t.sin_faces()[1] != 0.0
        return True

    def has_upper(self):
        if self.geometry == SPHERICAL:
            return self.t.sin_faces()[self.n_t + 1] != 0.0
        return True

    def volume_weights(self):
        """Domain-cell 3-D volumes, shape (n_r, n_t)."""
        return self.dV[1:self.n_r + 1, 1:self.n_t + 1]

    def coarsen(self):
        """The next coarser plane: every other face of each axis (the same
        spacing law with half the cells), one ghost cell per side."""
        return Plane(self.geometry, _coarse_axis(self.r), _coarse_axis(self.t),
                     self.n_phi, self.G)


def _coarse_axis(ax):
    """Coarse faces are the fine domain faces 0, 2, .., n; the coarse ghost
    faces continue the same law (ratio F[3]/F[1] or step F[3]-F[1])."""
    n = ax.n
    if n % 2:
        raise ValueError("axis cannot be coarsened")
    inner = ax.F[1:n + 2:2]
    if ax.spacing == LOG:
        q = inner[1] / inner[0]
        faces = np.concatenate([[inner[0] / q], inner, [inner[-1] * q]])
    else:
        d = inner[1] - inner[0]
        faces = np.concatenate([[inner[0] - d], inner, [inner[-1] + d]])
    return Axis(ax.kind, faces, ax.spacing)
