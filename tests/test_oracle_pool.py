"""The oracle's process pool runs the unchanged per-mode functions: its DGF
tables and solution equal the single-process ones bit for bit."""
import numpy as np

from oracle import dgf, james
from oracle.geometry import CYLINDRICAL, LOG, SPHERICAL, UNIFORM
from oracle.pool import ModePool, plane_from


def test_pool_equals_single_process():
    cases = [(SPHERICAL, 32, 16, 8, LOG, 0.1, 10.0, 0.0, np.pi),
             (CYLINDRICAL, 16, 16, 8, UNIFORM, 0.2, 1.0, -0.4, 0.4)]
    with ModePool(3) as pool:
        for desc in cases:
            p = plane_from(desc)
            rho = np.random.default_rng(5).random((p.n_r, p.n_t, p.n_phi))
            gt = dgf.dgf(p)
            assert np.array_equal(pool.dgf(desc), gt)
            assert np.array_equal(pool.dgf(desc, modes=[3, 1]), gt[[3, 1]])
            assert np.array_equal(pool.solve(desc, rho, gt), james.solve(p, rho, gt))
