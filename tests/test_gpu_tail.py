"""The cluster-resident tail of the multigrid solves (psolve_set_tail): once
few mode planes remain active (App. B: the low modes need the most
V-cycles), one launch finishes them with a thread-block cluster per plane
that keeps the plane's multigrid hierarchy in distributed shared memory.
Its iterations are the batched iterations' arithmetic, so results and cycle
counts match the batched loop, and the solution matches the oracle."""
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


def _pair(ps, sp, **kw):
    on = ps.Solver.from_spec(sp, precision=ps.MIXED, **kw)
    off = ps.Solver.from_spec(sp, precision=ps.MIXED, **kw)
    off.set_tail(0)
    return on, off


@pytest.mark.parametrize("key", list(SMALL))
def test_tail_matches_batched_iteration_and_oracle(ps, key):
    from oracle import dgf, james
    sp = SMALL[key]
    rho_np = clumps(sp, 31)
    rho = torch.from_numpy(rho_np).cuda()
    on, off = _pair(ps, sp)
    planes, ctas = on.tail()
    assert planes >= 1 and ctas >= 2, (planes, ctas)
    assert off.tail() == (0, 0)
    p = oracle_plane(sp)
    ref = james.solve(p, rho_np, dgf.dgf(p))
    for tol in (1e-8, 1e-10):
        a, _ = on.solve(rho, tol=tol)
        b, _ = off.solve(rho, tol=tol)
        sa, sb = on.stats(), off.stats()
        assert sa["rel_residual_psi"] <= tol and sa["rel_residual_phi"] <= tol
        for k in ("cycles_psi", "cycles_phi"):
            assert max(abs(x - y) for x, y in zip(sa[k], sb[k])) <= 1, (k, sa[k], sb[k])
        ea, eb = rel_l2(p, a.cpu().numpy(), ref), rel_l2(p, b.cpu().numpy(), ref)
        assert ea <= 1.05 * eb + 1e-9, (tol, ea, eb)
    assert ea <= 1e-7, ea
    on.close()
    off.close()


def test_tail_is_deterministic_in_graph_and_eager_modes(ps):
    sp = SMALL["cyl_cavity"]
    rho = torch.from_numpy(clumps(sp, 32)).cuda()
    g = ps.Solver.from_spec(sp, precision=ps.MIXED, use_graph=True)
    e = ps.Solver.from_spec(sp, precision=ps.MIXED, use_graph=False)
    pg = torch.empty_like(rho)
    g.solve(rho, pg, tol=1e-9)
    first = pg.clone()
    g.solve(rho, pg, tol=1e-9)
    pe, _ = e.solve(rho, tol=1e-9)
    assert torch.equal(pg, first) and torch.equal(pg, pe)
    assert g.stats()["cycles_psi"] == e.stats()["cycles_psi"]
    g.close()
    e.close()


def test_many_planes_in_the_tail(ps):
    """A density with power in many modes, a tail of up to 7 planes and a
    cap of 2: every cap gives the same per-mode cycle counts (within one)
    and the same potential."""
    sp = dict(SMALL["sph_log"], n_phi=32)
    rho = torch.from_numpy(clumps(sp, 33)).cuda()
    out = {}
    for cap in (0, 2, 7):
        s = ps.Solver.from_spec(sp, precision=ps.MIXED)
        s.set_tail(cap)
        planes = s.tail()[0]
        assert (planes == 0) if cap == 0 else (planes == 2 if cap == 2 else planes >= 2), (cap, planes)
        phi, _ = s.solve(rho, tol=1e-9)
        out[cap] = (phi.clone(), s.stats())
        s.close()
    base, st0 = out[0]
    for cap in (2, 7):
        phi, st = out[cap]
        d = float(torch.linalg.vector_norm(phi - base) / torch.linalg.vector_norm(base))
        assert d <= 1e-8, (cap, d)
        for k in ("cycles_psi", "cycles_phi"):
            assert max(abs(x - y) for x, y in zip(st[k], st0[k])) <= 1, (cap, k)
        assert st["iterations_psi"] == max(st["cycles_psi"])


def test_tail_reports_cycle_cap_and_non_finite(ps):
    sp = SMALL["sph_log"]
    rho = torch.from_numpy(clumps(sp, 34)).cuda()
    s = ps.Solver.from_spec(sp, precision=ps.MIXED, max_cycles=3)
    assert s.tail()[0] >= 1
    phi, rc = s.solve(rho, tol=1e-13, raise_on_error=False)
    assert rc == ps.ERR_NOT_CONVERGED and torch.isfinite(phi).all()
    assert max(s.stats()["cycles_psi"]) == 3
    s.close()
    s = ps.Solver.from_spec(sp, precision=ps.MIXED)
    bad = rho.clone()
    bad[5, 3, :] = float("inf")
    _, rc = s.solve(bad, raise_on_error=False)
    assert rc == ps.ERR_NONFINITE
    phi, rc = s.solve(rho, raise_on_error=False)   # the handle recovers
    assert rc == ps.OK and torch.isfinite(phi).all()
    s.close()


def test_tail_argument_checks(ps):
    s = ps.Solver.from_spec(SMALL["sph_log"], precision=ps.MIXED)
    with pytest.raises(ps.PSolveError) as e:
        s.set_tail(-2)
    assert e.value.code == ps.ERR_ARG
    s.set_tail(1)
    assert s.tail()[0] == 1
    s.set_tail(-1)
    assert s.tail()[0] >= 1
    s.close()
    d = ps.Solver.from_spec(SMALL["sph_log"], precision=ps.FP64)
    assert d.tail() == (0, 0)     # the FP64 path keeps the batched loop
    d.close()


def test_live_handles_of_different_sizes_share_the_kernel(ps):
    """Handles of different tail layouts alive together, created small to
    large and large to small, each solved twice: the kernel's launch limits
    are process-wide and must admit every handle's layout."""
    keys = ["cyl_axis", "sph_log", "cyl_cavity", "sph_partial"]
    for order in (keys, keys[::-1]):
        solvers = [ps.Solver.from_spec(SMALL[k], precision=ps.MIXED) for k in order]
        rhos = [torch.from_numpy(clumps(SMALL[k], 40 + i)).cuda() for i, k in enumerate(order)]
        first = [s.solve(r, tol=1e-8)[0].clone() for s, r in zip(solvers, rhos)]
        for s, r, f in zip(solvers, rhos, first):
            assert s.tail()[0] >= 1
            assert torch.equal(s.solve(r, tol=1e-8)[0], f)
        for s in solvers:
            s.close()
