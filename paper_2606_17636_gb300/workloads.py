"""Seeded synthetic densities for the solver's workloads.

This module only draws random numbers and evaluates densities; it holds none
of the solver's arithmetic.  Densities are sampled at the midpoint of each
cell's coordinate interval (radius, polar angle or height, azimuth), computed
from the grid law given by the caller's parameters.  Every draw comes from
``numpy.random.Generator(PCG64(20261203 + workload_id))``.

Workloads (sizes n_r x n_theta_or_z x n_phi):
  1  cylindrical, uniform R in [0, 1], z in [-0.5, 0.5], 32^3; one uniform
     sphere of radius 0.3 at (R, phi, z) = (0.4, 0, 0), density 1 inside.
  2  spherical, log r in [0.1, 10], 128 x 64 x 128; four Gaussian clumps.
  3  spherical, log r in [0.05, 20], 256 x 128 x 256; lognormal field
     (Gaussian field with P(k) ~ k^-3 on a periodic 256^3 box [-10, 10]^3,
     unit variance, rho = exp(g - 1/2)) sampled trilinearly, zero for r > 10.
  4  cylindrical, uniform R in [0.2, 4], z in [-1, 1], 512 x 256 x 512;
     exponential disc exp(-R) sech^2(z / 0.05 R) (1 + 0.3 cos(2 phi - 2.5 ln R))
     times (1 + 0.01 white noise).
  5  sixteen problems: even index spherical log r in [0.05, 20], odd index
     cylindrical uniform R in [4/33, 4] (an inner cavity of 2, 4 or 8 cells'
     width, so that r = 0 is a cell face), z in [-2, 2]; N x N/2 x N with
     N in {64, 128, 256} (each size at least twice); four Gaussian clumps.
"""
import numpy as np

SPHERICAL, CYLINDRICAL = 0, 1
UNIFORM, LOG = 0, 1
SEED = 20261203


def rng_for(workload_id):
    return np.random.Generator(np.random.PCG64(SEED + workload_id))


def _law(lo, hi, n, spacing):
    k = np.arange(n + 1, dtype=np.float64)
    if spacing == LOG:
        return lo * (hi / lo) ** (k / n)
    return lo + k * ((hi - lo) / n)


def midpoints(spec):
    """Sample coordinates (r, t, phi) of a problem spec, each 1-D."""
    fr = _law(spec["r_in"], spec["r_out"], spec["n_r"], spec["spacing"])
    ft = _law(spec["t_min"], spec["t_max"], spec["n_tz"], UNIFORM)
    r = 0.5 * (fr[1:] + fr[:-1])
    t = 0.5 * (ft[1:] + ft[:-1])
    ph = (np.arange(spec["n_phi"]) + 0.5) * (2.0 * np.pi / spec["n_phi"])
    return r, t, ph


def cartesian(spec):
    r, t, ph = midpoints(spec)
    R = r[:, None, None]
    T = t[None, :, None]
    P = ph[None, None, :]
    if spec["geometry"] == SPHERICAL:
        return R * np.sin(T) * np.cos(P), R * np.sin(T) * np.sin(P), R * np.cos(T) + 0 * P
    return R * np.cos(P) + 0 * T, R * np.sin(P) + 0 * T, T + 0 * R + 0 * P


def spec(geometry, n_r, n_tz, n_phi, spacing, r_in, r_out, t_min=None, t_max=None):
    if t_min is None:
        if geometry == SPHERICAL:
            t_min, t_max = 0.0, np.pi
        else:
            t_min, t_max = -0.5 * (r_out - r_in), 0.5 * (r_out - r_in)
    return dict(geometry=geometry, n_r=n_r, n_tz=n_tz, n_phi=n_phi, spacing=spacing,
                r_in=r_in, r_out=r_out, t_min=t_min, t_max=t_max)


def _clumps(sp, rng, n=4):
    x, y, z = cartesian(sp)
    rho = np.zeros(np.broadcast(x, y, z).shape)
    for _ in range(n):
        if sp["geometry"] == SPHERICAL:
            lo, hi = max(0.3, sp["r_in"] * 3), min(5.0, sp["r_out"] / 2)
            if hi <= lo:       # narrow shells: clumps in the middle half of the shell
                d = sp["r_out"] - sp["r_in"]
                lo, hi = sp["r_in"] + 0.25 * d, sp["r_in"] + 0.75 * d
            rc = np.exp(rng.uniform(np.log(lo), np.log(hi)))
            ct = rng.uniform(-0.7, 0.7)
            pc = rng.uniform(0.0, 2 * np.pi)
            st = np.sqrt(1 - ct * ct)
            cx, cy, cz = rc * st * np.cos(pc), rc * st * np.sin(pc), rc * ct
        else:
            Rc = rng.uniform(sp["r_in"] + 0.25 * (sp["r_out"] - sp["r_in"]),
                             sp["r_in"] + 0.75 * (sp["r_out"] - sp["r_in"]))
            pc = rng.uniform(0.0, 2 * np.pi)
            zc = rng.uniform(0.5 * sp["t_min"], 0.5 * sp["t_max"])
            cx, cy, cz = Rc * np.cos(pc), Rc * np.sin(pc), zc
        w = rng.uniform(0.2, 1.0)
        amp = rng.uniform(0.5, 2.0)
        rho += amp * np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2 * w * w))
    return rho


def _lognormal_box(rng, n=256, L=20.0):
    k1 = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    kz = 2 * np.pi * np.fft.rfftfreq(n, d=L / n)
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2)
    amp = np.zeros_like(kk)
    ok = kk >= 2 * np.pi / L
    amp[ok] = kk[ok] ** -1.5                      # sqrt of P(k) ~ k^-3
    noise = rng.standard_normal((n, n, n))
    g = np.fft.irfftn(np.fft.rfftn(noise) * amp, s=(n, n, n), axes=(0, 1, 2))
    g = (g - g.mean()) / g.std()
    return np.exp(g - 0.5)


def _trilinear(box, L, x, y, z):
    n = box.shape[0]
    h = L / n
    out = np.empty(np.broadcast(x, y, z).shape)
    X, Y, Z = np.broadcast_arrays(x, y, z)
    for sl in range(X.shape[0]):
        u = (X[sl] + L / 2) / h - 0.5
        v = (Y[sl] + L / 2) / h - 0.5
        w = (Z[sl] + L / 2) / h - 0.5
        i0, j0, k0 = np.floor(u).astype(int), np.floor(v).astype(int), np.floor(w).astype(int)
        fu, fv, fw = u - i0, v - j0, w - k0
        acc = 0.0
        for di in (0, 1):
            for dj in (0, 1):
                for dk in (0, 1):
                    wt = (fu if di else 1 - fu) * (fv if dj else 1 - fv) * (fw if dk else 1 - fw)
                    acc = acc + wt * box[(i0 + di) % n, (j0 + dj) % n, (k0 + dk) % n]
        out[sl] = acc
    return out


BASE = {
    1: (dict(geometry=CYLINDRICAL, n_r=32, n_tz=32, n_phi=32, spacing=UNIFORM, r_in=0.0,
             r_out=1.0, t_min=-0.5, t_max=0.5), 1e-10, 0),
    2: (dict(geometry=SPHERICAL, n_r=128, n_tz=64, n_phi=128, spacing=LOG, r_in=0.1,
             r_out=10.0, t_min=0.0, t_max=np.pi), 1e-10, 0),
    3: (dict(geometry=SPHERICAL, n_r=256, n_tz=128, n_phi=256, spacing=LOG, r_in=0.05,
             r_out=20.0, t_min=0.0, t_max=np.pi), 1e-8, 1),
    4: (dict(geometry=CYLINDRICAL, n_r=512, n_tz=256, n_phi=512, spacing=UNIFORM, r_in=0.2,
             r_out=4.0, t_min=-1.0, t_max=1.0), 1e-8, 1),
}


def workload(workload_id):
    """Problem spec(s) and density for one workload: dict with 'spec', 'rho',
    'tol', 'precision' (0 FP64, 1 mixed); workload 5 returns a list."""
    rng = rng_for(workload_id)
    if workload_id == 1:
        sp = dict(BASE[1][0])
        x, y, z = cartesian(sp)
        d = np.sqrt((x - 0.4) ** 2 + y**2 + z**2)
        return dict(spec=sp, rho=(d < 0.3).astype(np.float64), tol=1e-10, precision=0)
    if workload_id == 2:
        sp = dict(BASE[2][0])
        return dict(spec=sp, rho=_clumps(sp, rng), tol=1e-10, precision=0)
    if workload_id == 3:
        sp = dict(BASE[3][0])
        box = _lognormal_box(rng)
        x, y, z = cartesian(sp)
        rho = _trilinear(box, 20.0, x, y, z)
        r, _, _ = midpoints(sp)
        rho *= (r < 10.0)[:, None, None]
        return dict(spec=sp, rho=rho, tol=1e-8, precision=1)
    if workload_id == 4:
        sp = dict(BASE[4][0])
        r, t, ph = midpoints(sp)
        R = r[:, None, None]
        Z = t[None, :, None]
        P = ph[None, None, :]
        rho = (np.exp(-R) / np.cosh(Z / (0.05 * R)) ** 2
               * (1 + 0.3 * np.cos(2 * P - 2.5 * np.log(R))))
        rho = rho * (1 + 0.01 * rng.standard_normal(rho.shape))
        return dict(spec=sp, rho=rho, tol=1e-8, precision=1)
    if workload_id == 5:
        sizes = [64, 64, 128, 128, 256, 256] + list(rng.choice([64, 128, 256], size=10))
        rng.shuffle(sizes)
        out = []
        for i, N in enumerate(sizes):
            N = int(N)
            if i % 2 == 0:
                sp = spec(SPHERICAL, N, N // 2, N, LOG, 0.05, 20.0)
            else:
                sp = spec(CYLINDRICAL, N, N // 2, N, UNIFORM, 4.0 / 33.0, 4.0, -2.0, 2.0)
            out.append(dict(spec=sp, rho=_clumps(sp, rng), tol=1e-8, precision=1))
        return out
    raise ValueError(workload_id)


def scaled(workload_id, shrink):
    """A workload's geometry and density law at sizes divided by ``shrink``
    (for parity cases the oracle finishes in seconds)."""
    base_sp, tol, precision = BASE[workload_id]
    sp = dict(base_sp)
    for k in ("n_r", "n_tz", "n_phi"):
        sp[k] = max(8, sp[k] // shrink)
    rng = rng_for(100 + workload_id)
    if workload_id in (2, 3):
        rho = _clumps(sp, rng)
    elif workload_id == 1:
        x, y, z = cartesian(sp)
        rho = (np.sqrt((x - 0.4) ** 2 + y**2 + z**2) < 0.3).astype(np.float64)
    else:
        r, t, ph = midpoints(sp)
        R, Z, P = r[:, None, None], t[None, :, None], ph[None, None, :]
        rho = np.exp(-R) / np.cosh(Z / (0.05 * R)) ** 2 * (1 + 0.3 * np.cos(2 * P - 2.5 * np.log(R)))
        rho = rho * (1 + 0.01 * rng.standard_normal(rho.shape))
    return dict(spec=sp, rho=np.ascontiguousarray(rho, dtype=np.float64), tol=tol,
                precision=precision)
