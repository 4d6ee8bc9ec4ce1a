"""Solves from host memory with the copies overlapped (psolve_solve_host):
the staged solves give bitwise the results of device-resident solves on the
same handle (the same kernels on staging buffers), in graph and eager mode,
with pinned and pageable buffers, repeated result buffers, warm starts and
several densities per handle; and the setup-time split of psolve_create."""
import ctypes

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


def _densities(sp, seeds, pin=True):
    out = []
    for s in seeds:
        t = torch.from_numpy(clumps(sp, s))
        out.append(t.pin_memory() if pin else t)
    return out


@pytest.mark.parametrize("key,precision,use_graph", [("sph_log", 1, True), ("cyl_cavity", 0, True),
                                                     ("cyl_axis", 1, False)])
def test_host_solves_equal_device_solves(ps, key, precision, use_graph):
    sp = SMALL[key]
    s = ps.Solver.from_spec(sp, precision=precision, use_graph=use_graph)
    rhos = _densities(sp, (60, 61, 62))
    ref = []
    for r in rhos:
        phi, _ = s.solve(r.cuda(), tol=1e-10)
        ref.append(phi.cpu())
    phis, status, rc = s.solve_host(rhos, tol=1e-10)
    assert rc == ps.OK and status == [ps.OK] * 3
    for got, want in zip(phis, ref):
        assert torch.equal(got, want)
    # the same device solves against the oracle, for the first density
    from oracle import dgf, james
    p = oracle_plane(sp)
    oref = james.solve(p, rhos[0].numpy(), dgf.dgf(p))
    assert rel_l2(p, phis[0].numpy(), oref) <= (1e-9 if precision == 0 else 1e-7)
    # pageable buffers and one repeated result buffer: the last solve wins
    pageable = _densities(sp, (60, 61, 62), pin=False)
    out = torch.zeros(s.shape, dtype=torch.float64)
    phis2, status2, rc2 = s.solve_host(pageable, [out] * 3, tol=1e-10)
    assert rc2 == ps.OK and status2 == [ps.OK] * 3
    assert torch.equal(out, ref[2])
    s.close()


def test_warm_started_host_sequence_equals_device_sequence(ps):
    sp = SMALL["sph_log"]
    seeds = (70, 71, 72, 73)
    dev = ps.Solver.from_spec(sp, precision=ps.MIXED)
    host = ps.Solver.from_spec(sp, precision=ps.MIXED)
    dev.set_warm_start(True)
    host.set_warm_start(True)
    base = torch.from_numpy(clumps(sp, 74))
    rhos = [(base * (1.0 + 0.01 * k)).contiguous().pin_memory() for k in range(len(seeds))]
    ref, its = [], []
    for r in rhos:
        phi, _ = dev.solve(r.cuda(), tol=1e-9)
        ref.append(phi.cpu())
        st = dev.stats()
        its.append((st["iterations_psi"], st["iterations_phi"]))
    phis, status, rc = host.solve_host(rhos, tol=1e-9)
    assert rc == ps.OK
    for got, want in zip(phis, ref):
        assert torch.equal(got, want)
    st = host.stats()
    assert (st["iterations_psi"], st["iterations_phi"]) == its[-1]
    assert its[-1][0] < its[0][0]           # the later solves started warm
    dev.close()
    host.close()


def test_host_solves_with_several_densities(ps):
    sp = SMALL["cyl_cavity"]
    s = ps.Solver.from_spec(sp, precision=ps.MIXED, n_densities=2)
    one = ps.Solver.from_spec(sp, precision=ps.MIXED)
    pairs = [torch.stack([torch.from_numpy(clumps(sp, 80 + 2 * k)),
                          torch.from_numpy(clumps(sp, 81 + 2 * k))]).contiguous().pin_memory()
             for k in range(2)]
    phis, status, rc = s.solve_host(pairs, tol=1e-10)
    assert rc == ps.OK and status == [ps.OK, ps.OK]
    for pr, got in zip(pairs, phis):
        for b in range(2):
            want, _ = one.solve(pr[b].cuda(), tol=1e-10)
            assert rel_l2(oracle_plane(sp), got[b].numpy(), want.cpu().numpy()) <= 1e-9
    s.close()
    one.close()


def test_host_solve_arguments_and_setup_times(ps):
    sp = SMALL["sph_log"]
    s = ps.Solver.from_spec(sp, precision=ps.MIXED)
    phis, status, rc = s.solve_host([], [])
    assert rc == ps.OK and phis == [] and status == []
    with pytest.raises(ValueError):
        s.solve_host([torch.zeros(3, dtype=torch.float64)])
    L = ps.lib()
    R = (ctypes.c_void_p * 1)(None)
    F = (ctypes.c_void_p * 1)(None)
    assert L.psolve_solve_host(s.h, 1, R, F, 1e-8, None) == ps.ERR_ARG
    assert L.psolve_solve_host(s.h, -1, R, F, 1e-8, None) == ps.ERR_ARG
    # a non-finite density reports its status and leaves the others intact
    good = torch.from_numpy(clumps(sp, 90)).pin_memory()
    bad = good.clone()
    bad[3, 2, 1] = float("nan")
    phis, status, rc = s.solve_host([good, bad, good], tol=1e-9, raise_on_error=False)
    assert rc == ps.ERR_NONFINITE
    assert status[0] == ps.OK and status[1] == ps.ERR_NONFINITE and status[2] == ps.OK
    want, _ = s.solve(good.cuda(), tol=1e-9)
    assert torch.equal(phis[2], want.cpu())
    setup_ms, dgf_ms = s.setup_times()
    assert 0.0 < dgf_ms <= setup_ms
    assert setup_ms == pytest.approx(s.stats()["setup_ms"])
    s.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_stage_times_split_the_solve(ps, use_graph):
    """psolve_get_stage_times: the five stages of the last solve (event marks
    on the handle's stream, event nodes in the captured graph) add up to the
    solve's own device time."""
    sp = SMALL["sph_log"]
    s = ps.Solver.from_spec(sp, precision=ps.MIXED, use_graph=use_graph)
    with pytest.raises(ps.PSolveError):
        s.stage_times()
    rho = torch.from_numpy(clumps(sp, 95)).cuda()
    phi = torch.empty_like(rho)
    s.solve(rho, phi, tol=1e-9)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.solve(rho, phi, tol=1e-9)
    e1.record()
    torch.cuda.synchronize()
    st = s.stage_times()
    assert set(st) == set(ps.Solver.STAGES)
    assert all(v > 0.0 for v in st.values()), st
    total = e0.elapsed_time(e1)
    assert sum(st.values()) <= total * 1.01 + 0.05, (st, total)
    if use_graph:   # host gaps of the eager loop are not in the marks' spans alone
        assert sum(st.values()) >= 0.8 * total, (st, total)
    assert st["mg_psi"] > st["fft_forward"] and st["mg_phi"] > st["fft_inverse"]
    s.close()
