"""Parity at the benchmark's full size: the 256 x 128 x 256 log-spherical
lognormal workload, solved through psolve_solve in the captured-graph
configuration the benchmark times, checked against the oracle mode by mode
on sampled azimuthal modes (each oracle mode is an independent direct solve
of Sec. 5.1 steps 3-6 with its own DGF table)."""
import numpy as np
import pytest

from gpu_helpers import oracle_plane

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLED = (0, 1, 3, 64, 128)


@pytest.fixture(scope="module")
def ps():
    import paper_2606_17636_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def full():
    from oracle import dft, dgf, james
    from paper_2606_17636_gb300 import workloads
    w = workloads.workload(3)
    p = oracle_plane(w["spec"])
    f = 4.0 * np.pi * p.G * dft.forward(w["rho"])
    gt = dgf.dgf(p, modes=SAMPLED)
    ref = {m: james.solve_mode(p, m, f[:, :, m], gt[k])[3] for k, m in enumerate(SAMPLED)}
    return w, p, ref


def _solve(ps, w, precision, tol):
    s = ps.Solver.from_spec(w["spec"], precision=precision, use_graph=True)
    phi, rc = s.solve(torch.from_numpy(w["rho"]).cuda(), tol=tol)
    st = s.stats()
    s.close()
    assert rc == ps.OK
    return phi.cpu().numpy(), st


def _norm_v(p, a):
    """Volume-weighted L2 norm of a mode plane (n_r, n_t)."""
    return float(np.sqrt((p.volume_weights() * np.abs(a) ** 2).sum()))


def _real_space_share(p, a, m, N):
    """Contribution of mode m's coefficient plane to the volume-weighted L2
    norm of the real field over all N azimuthal cells."""
    c = 1.0 if m in (0, N // 2) else 2.0
    return np.sqrt(c * N) * _norm_v(p, a)


def test_fp64_full_size_matches_oracle_on_sampled_modes(ps, full):
    """tol 1e-11: the m = 0 problem of this 400:1 logarithmic grid stops
    improving near a relative residual of 3e-12 in FP64 (its rounding floor),
    so 1e-11 is the tightest tolerance every mode reaches."""
    from oracle import dft
    w, p, ref = full
    phi, st = _solve(ps, w, ps.FP64, 1e-11)
    modes = dft.forward(phi)
    for m in SAMPLED:
        err = _norm_v(p, modes[:, :, m] - ref[m]) / _norm_v(p, ref[m])
        assert err <= 1e-10, (m, err)


def test_mixed_full_size_matches_oracle_on_sampled_modes(ps, full):
    """At tol 1e-8 the mixed path's error on each sampled mode equals the FP64
    path's at the same tolerance (the grid's residual-to-error amplification
    sets it); at tol 1e-10 each sampled mode's share of the real-space error
    is below 1e-7 of the potential's norm."""
    from oracle import dft
    w, p, ref = full
    N = w["spec"]["n_phi"]
    out = {}
    for prec in (ps.FP64, ps.MIXED):
        for tol in (1e-8, 1e-10):
            phi, st = _solve(ps, w, prec, tol)
            assert st["rel_residual_psi"] <= tol and st["rel_residual_phi"] <= tol
            out[prec, tol] = (phi, dft.forward(phi))
    norm = float(np.sqrt((p.volume_weights()[:, :, None] * out[ps.FP64, 1e-10][0] ** 2).sum()))
    for m in SAMPLED:
        e64 = _real_space_share(p, out[ps.FP64, 1e-8][1][:, :, m] - ref[m], m, N)
        emx = _real_space_share(p, out[ps.MIXED, 1e-8][1][:, :, m] - ref[m], m, N)
        assert emx <= 1.05 * e64 + 1e-9 * norm, (m, emx / norm, e64 / norm)
        e10 = _real_space_share(p, out[ps.MIXED, 1e-10][1][:, :, m] - ref[m], m, N)
        assert e10 <= 1e-7 * norm, (m, e10 / norm)
    # the two precisions agree on the whole field at equal tolerance
    wv = p.volume_weights()[:, :, None]
    d = out[ps.MIXED, 1e-8][0] - out[ps.FP64, 1e-8][0]
    dn = float(np.sqrt((wv * d ** 2).sum()))
    assert dn <= 1e-9 * norm, dn / norm
    # whole-field error of the mixed path at tol 1e-8 against the FP64 path
    # at tol 1e-11 (itself within 1e-10 of the oracle on every sampled mode)
    ref64, _ = _solve(ps, w, ps.FP64, 1e-11)
    e = float(np.sqrt((wv * (out[ps.MIXED, 1e-8][0] - ref64) ** 2).sum()))
    assert e <= 1e-7 * float(np.sqrt((wv * ref64 ** 2).sum())), e
