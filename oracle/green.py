"""Azimuthal Fourier modes of the continuous Green's function -G/|x - x'|.

Sec. 4.2, Eq. DGF_bc_sph (spherical) and Eq. DGF_bc_cyl (cylindrical):

    G^m(t, s) = -G sum_{k=0}^{N-1} cos(2 pi m k / N) / d_k(t, s)

with d_k^2 = A - B cos(2 pi k / N),  A = r^2 + r'^2 - 2 r r' cos(th) cos(th'),
B = 2 r r' sin(th) sin(th')  (spherical), or
d_k^2 = R^2 + R'^2 - 2 R R' cos(2 pi k / N) + (z - z')^2  (cylindrical),
and its radial derivative with respect to the field point (Sec. 4.2, the
Neumann data of the extended-domain construction):

    dG^m/dr = G sum_k [C - D cos(2 pi k/N)] cos(2 pi m k/N) / d_k^3,
    C = r - r' cos(th) cos(th'), D = r' sin(th) sin(th')   (spherical),
    C = R, D = R'                                          (cylindrical).

The paper's sums run to N in the derivative formulas; one period, k = 0..N-1,
is used everywhere.  The sums carry no 1/N: they are the unnormalised
transform, which is what the boundary convolution needs when sigma and Theta
use the normalised forward transform.
"""
import numpy as np

from .geometry import SPHERICAL


def _trig(N):
    k = np.arange(N)
    c1 = np.cos(2.0 * np.pi * k / N)
    m = np.arange(N // 2 + 1)[:, None]
    cm = np.cos(2.0 * np.pi * ((m * k[None, :]) % N) / N)
    return c1, cm


def mode_sum(geometry, N, G, xt, yt, xs, ys):
    """G^m for arrays of field points (xt, yt) and source points (xs, ys)
    (broadcast together); returns shape (..., N/2+1)."""
    c1, cm = _trig(N)
    xt, yt, xs, ys = (np.asarray(a, dtype=np.float64)[..., None] for a in (xt, yt, xs, ys))
    if geometry == SPHERICAL:
        A = xt**2 + xs**2 - 2.0 * xt * xs * np.cos(yt) * np.cos(ys)
        B = 2.0 * xt * xs * np.sin(yt) * np.sin(ys)
        d = np.sqrt(A - B * c1)
    else:
        d = np.sqrt(xt**2 + xs**2 - 2.0 * xt * xs * c1 + (yt - ys) ** 2)
    return -G * (1.0 / d) @ cm.T


def mode_sum_dr(geometry, N, G, xt, yt, xs, ys):
    """Radial derivative (field point) of ``mode_sum``."""
    c1, cm = _trig(N)
    xt, yt, xs, ys = (np.asarray(a, dtype=np.float64)[..., None] for a in (xt, yt, xs, ys))
    if geometry == SPHERICAL:
        A = xt**2 + xs**2 - 2.0 * xt * xs * np.cos(yt) * np.cos(ys)
        B = 2.0 * xt * xs * np.sin(yt) * np.sin(ys)
        C = xt - xs * np.cos(yt) * np.cos(ys)
        D = xs * np.sin(yt) * np.sin(ys)
        d2 = A - B * c1
    else:
        C = xt + 0.0 * xs
        D = xs + 0.0 * xt
        d2 = xt**2 + xs**2 - 2.0 * xt * xs * c1 + (yt - ys) ** 2
    return G * ((C - D * c1) / d2**1.5) @ cm.T
