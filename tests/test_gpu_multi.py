"""Several densities of one geometry per solve (psolve_create_multi): every
density's potential equals its own single solve -- bit for bit on the FP64
path, whose planes iterate independently; within rounding on the mixed path,
where the cluster-resident tail takes the last planes at a different
iteration -- and matches the oracle."""
import numpy as np
import pytest

from gpu_helpers import SMALL, clumps, oracle_plane, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import paper_2606_17636_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("key", ["sph_log", "cyl_cavity"])
@pytest.mark.parametrize("precision,graph", [(0, True), (1, True), (1, False)])
def test_multi_density_solve_matches_single_solves(ps, key, precision, graph):
    sp = SMALL[key]
    nd = 3
    rhos = [clumps(sp, 70 + k) for k in range(nd)]
    multi = ps.Solver.from_spec(sp, precision=precision, use_graph=graph, n_densities=nd)
    assert multi.shape == (nd, sp["n_r"], sp["n_tz"], sp["n_phi"])
    rho = torch.from_numpy(np.stack(rhos)).cuda()
    phi, rc = multi.solve(rho, tol=1e-10)
    assert rc == ps.OK
    st = multi.stats()
    assert st["rel_residual_psi"] <= 1e-10 and st["rel_residual_phi"] <= 1e-10
    single = ps.Solver.from_spec(sp, precision=precision, use_graph=graph)
    for k in range(nd):
        ref, _ = single.solve(torch.from_numpy(rhos[k]).cuda(), tol=1e-10)
        if precision == 0:
            assert torch.equal(phi[k], ref)
        else:
            d = float(torch.linalg.vector_norm(phi[k] - ref) / torch.linalg.vector_norm(ref))
            assert d <= 1e-8, (k, d)
    # the last density against the oracle
    from oracle import dgf, james
    p = oracle_plane(sp)
    ref = james.solve(p, rhos[-1], dgf.dgf(p))
    assert rel_l2(p, phi[-1].cpu().numpy(), ref) <= (1e-10 if precision == 0 else 1e-7)
    multi.close()
    single.close()


def test_multi_density_argument_checks(ps):
    with pytest.raises(ps.PSolveError) as e:
        ps.Solver.from_spec(SMALL["sph_log"], n_densities=65)
    assert e.value.code == ps.ERR_ARG
