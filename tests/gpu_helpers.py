"""Shared helpers of the GPU parity tests: problem specs, oracle planes,
layout conversions (GPU planes are [m][j][i], oracle arrays [i][j][m])."""
import numpy as np

from oracle.geometry import Plane
from paper_2606_17636_gb300 import workloads


def oracle_plane(spec):
    return Plane.make(spec["geometry"], spec["n_r"], spec["n_tz"], spec["n_phi"], spec["spacing"],
                      spec["r_in"], spec["r_out"], t_min=spec["t_min"], t_max=spec["t_max"])


def to_oracle(planes):
    """GPU planes [M, n_t, n_r] -> oracle layout [n_r, n_t, M]."""
    return np.ascontiguousarray(np.transpose(planes, (2, 1, 0)))


def to_gpu(arr):
    return np.ascontiguousarray(np.transpose(arr, (2, 1, 0)))


def rel_l2(plane, a, ref):
    w = plane.volume_weights()[:, :, None]
    return float(np.sqrt((w * np.abs(a - ref) ** 2).sum() / (w * np.abs(ref) ** 2).sum()))


SMALL = {
    "cyl_axis": workloads.spec(workloads.CYLINDRICAL, 32, 32, 16, workloads.UNIFORM, 0.0, 1.0, -0.5, 0.5),
    "sph_log": workloads.spec(workloads.SPHERICAL, 64, 32, 16, workloads.LOG, 0.1, 10.0),
    "cyl_cavity": workloads.spec(workloads.CYLINDRICAL, 32, 64, 8, workloads.UNIFORM, 0.2, 1.0),
    "sph_partial": workloads.spec(workloads.SPHERICAL, 32, 32, 8, workloads.UNIFORM, 1.0, 2.0,
                                  0.25 * np.pi, 0.75 * np.pi),
    # a polar range off the equator: the polar operator is not mirror-symmetric,
    # so the coarsest solve takes the general separable layout (the others the
    # mirror-symmetric one)
    "sph_offcentre": workloads.spec(workloads.SPHERICAL, 32, 32, 8, workloads.UNIFORM, 1.0, 2.0,
                                    0.3 * np.pi, 0.65 * np.pi),
}


def clumps(spec, seed):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(workloads._clumps(spec, rng))
