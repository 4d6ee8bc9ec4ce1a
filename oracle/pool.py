"""The oracle's seven-step solve (Sec. 5.1) with its per-mode work spread over
spawned worker processes.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only ``tests/`` and
the CPU-baseline / reference legs of ``bench.py`` use it.

The azimuthal modes are independent from step 3 to step 6 (both Helmholtz
solves, the screening mass and the boundary convolution) and in the DGF
tables of step 1, so each worker runs the unchanged single-mode functions of
``james`` and ``dgf`` on a contiguous chunk of modes.  The arithmetic of
every mode is exactly that of ``james.solve``; only where it runs differs.
Workers are started with the ``spawn`` method (safe in a process that
already holds a GPU context) and run single-threaded BLAS.
"""
import multiprocessing as mp
import os

import numpy as np

from . import dft, dgf, james
from .geometry import Plane

_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def plane_from(desc):
    """desc: (geometry, n_r, n_t, n_phi, spacing, r_in, r_out, t_min, t_max)."""
    g, nr, nt, nphi, sp, ri, ro, tmin, tmax = desc
    return Plane.make(g, nr, nt, nphi, sp, ri, ro, t_min=tmin, t_max=tmax)


def _init_worker():
    for k in _THREAD_VARS:
        os.environ[k] = "1"


def _dgf_chunk(args):
    desc, modes = args
    return modes, dgf.dgf(plane_from(desc), modes=modes)


def _solve_chunk(args):
    desc, modes, f, gt = args
    p = plane_from(desc)
    out = np.empty(f.shape, dtype=complex)
    for k, m in enumerate(modes):
        out[:, :, k] = james.solve_mode(p, m, f[:, :, k], gt[k])[3]
    return modes, out


def _chunks(n, parts):
    parts = max(1, min(parts, n))
    bounds = np.linspace(0, n, parts + 1).round().astype(int)
    return [list(range(bounds[q], bounds[q + 1])) for q in range(parts) if bounds[q + 1] > bounds[q]]


class ModePool:
    """A pool of `procs` spawned single-threaded workers (default: every core)."""

    def __init__(self, procs=None):
        self.procs = procs or os.cpu_count() or 1
        saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        for k in _THREAD_VARS:      # spawned children inherit these at start-up
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_init_worker)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def close(self):
        self.pool.terminate()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def dgf(self, desc, modes=None):
        """Gt[k, t, s] for `modes` (default all), as ``dgf.dgf``."""
        p = plane_from(desc)
        modes = list(range(p.n_modes)) if modes is None else list(modes)
        nb = len(james.boundary_points(p))
        out = np.zeros((len(modes), nb, nb))
        # several chunks per worker: the extended-domain modes differ in cost
        jobs = [(desc, [modes[i] for i in c]) for c in _chunks(len(modes), 4 * self.procs)]
        pos = {m: k for k, m in enumerate(modes)}
        for ms, g in self.pool.imap_unordered(_dgf_chunk, jobs):
            for k, m in enumerate(ms):
                out[pos[m]] = g[k]
        return out

    def solve(self, desc, rho, gt):
        """phi (n_r, n_t, n_phi) of ``james.solve(plane, rho, gt)``: steps 2
        and 7 here, steps 3-6 of each mode in a worker."""
        p = plane_from(desc)
        N = p.n_phi
        f = 4.0 * np.pi * p.G * dft.forward(rho)            # step 2
        M = f.shape[2]
        phi_hat = np.empty_like(f)
        jobs = [(desc, c, np.ascontiguousarray(f[:, :, c[0]:c[-1] + 1]), gt[c[0]:c[-1] + 1])
                for c in _chunks(M, self.procs)]
        for ms, part in self.pool.imap_unordered(_solve_chunk, jobs):
            phi_hat[:, :, ms[0]:ms[-1] + 1] = part
        return dft.inverse(phi_hat, N)                        # step 7
