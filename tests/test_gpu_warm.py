"""Warm start (psolve_set_warm_start): later solves start the Psi solve from
the previous Psi and the Phi solve from the previous Phi (App. B).  For a
slightly changed density the result equals a cold solve at the same
tolerance and needs fewer V-cycles."""
import numpy as np
import pytest

from gpu_helpers import clumps, oracle_plane, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import paper_2606_17636_gb300 as m
    m.lib()
    return m


def _densities():
    from paper_2606_17636_gb300 import workloads as wl
    sp = wl.spec(wl.SPHERICAL, 128, 64, 16, wl.LOG, 0.1, 10.0)
    rho1 = clumps(sp, 31)
    _, _, ph = wl.midpoints(sp)
    rho2 = rho1 * (1.0 + 1e-3 * np.cos(2.0 * ph)[None, None, :])   # a slowly growing m = 2 perturbation
    return sp, rho1, rho2


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_warm_start_matches_cold_solve_with_fewer_cycles(ps, graph, precision):
    from oracle import dgf, james
    sp, rho1, rho2 = _densities()
    tol = 1e-10
    r2 = torch.from_numpy(rho2).cuda()
    cold = ps.Solver.from_spec(sp, precision=precision, use_graph=graph)
    phi_c, rc = cold.solve(r2, tol=tol)
    st_c = cold.stats()
    warm = ps.Solver.from_spec(sp, precision=precision, use_graph=graph)
    warm.set_warm_start(True)
    warm.solve(torch.from_numpy(rho1).cuda(), tol=tol)
    phi_w, rc = warm.solve(r2, tol=tol)
    st_w = warm.stats()
    assert st_w["iterations_psi"] < st_c["iterations_psi"], (st_w, st_c)
    assert st_w["iterations_phi"] < st_c["iterations_phi"], (st_w, st_c)
    assert st_w["rel_residual_psi"] <= tol and st_w["rel_residual_phi"] <= tol
    p = oracle_plane(sp)
    ref = james.solve(p, rho2, dgf.dgf(p))
    assert rel_l2(p, phi_c.cpu().numpy(), ref) <= 1e-7
    assert rel_l2(p, phi_w.cpu().numpy(), ref) <= 1e-7
    assert rel_l2(p, phi_w.cpu().numpy(), phi_c.cpu().numpy()) <= 1e-7
    # back to cold starts: the same counts as a cold solve
    warm.set_warm_start(False)
    warm.solve(r2, tol=tol)
    st_c2 = warm.stats()
    assert (st_c2["iterations_psi"], st_c2["iterations_phi"]) == (st_c["iterations_psi"], st_c["iterations_phi"])
    cold.close()
    warm.close()
