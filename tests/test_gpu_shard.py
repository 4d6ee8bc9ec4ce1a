"""The library's building blocks of a mode-sharded solve, on one GPU: slab
transforms along phi, the mode-subset solve (Sec. 5.1 steps 3-6 for listed
modes), and the sharded pipeline of paper_2606_17636_gb300/shard.py on a
one-rank NCCL group.  Splitting the modes over ranks leaves every mode's
answer unchanged (the modes are independent, Sec. 2.2)."""
import os
import socket

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
def test_slab_transforms_equal_the_whole_transform(ps, key):
    sp = SMALL[key]
    s = ps.Solver.from_spec(sp, precision=ps.FP64)
    rho = torch.from_numpy(clumps(sp, 50)).cuda()
    f = s.stage_forward(rho)
    n_r = sp["n_r"]
    inv = s.stage_inverse(f)
    # the transform packs two real rows (i, i + 1) into one complex sequence,
    # counted from the slab's first row (a last unpaired row is packed with
    # zeros): slabs with even ends pair the rows as the whole transform does
    # (bitwise equal), others agree to rounding
    for a, b in ((0, 5), (6, n_r - 2), (n_r - 4, n_r), (0, n_r), (5, n_r - 3), (n_r - 3, n_r)):
        fr = s.stage_forward_rows(rho[a:b].contiguous())
        back = s.stage_inverse_rows(fr.contiguous())
        if a % 2 == 0 and b % 2 == 0:
            assert torch.equal(fr, f[:, :, a:b]) and torch.equal(back, inv[a:b])
        else:
            assert (fr - f[:, :, a:b]).abs().max() <= 1e-14 * f.abs().max()
            assert (back - inv[a:b]).abs().max() <= 1e-14 * inv.abs().max()
    with pytest.raises(ps.PSolveError):
        s.stage_forward_rows(rho[:0].contiguous())
    s.close()


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-12, 1e-12), (1, 1e-10, 1e-8)])
def test_mode_subsets_reproduce_the_whole_solve(ps, precision, tol, bound):
    from paper_2606_17636_gb300 import shard
    from oracle import dgf, james
    key = "sph_log"
    sp = SMALL[key]
    rho_np = clumps(sp, 51)
    rho = torch.from_numpy(rho_np).cuda()
    s = ps.Solver.from_spec(sp, precision=precision, use_graph=False)
    whole, _ = s.solve(rho, tol=tol)
    whole = whole.clone()
    f = s.stage_forward(rho)
    M = s.n_modes
    phi_hat = torch.zeros_like(f)
    for mine in shard.lpt_assign(shard.initial_costs(M), 3):
        idx = torch.tensor(mine, dtype=torch.long, device="cuda")
        out, rc = s.solve_modes(mine, f.index_select(0, idx).contiguous(), tol=tol)
        assert rc == ps.OK
        st = s.stats()
        assert all(st["cycles_psi"][m] == 0 for m in range(M) if m not in mine)
        phi_hat[idx] = out
    phi = s.stage_inverse(phi_hat)
    d = float(torch.linalg.vector_norm(phi - whole) / torch.linalg.vector_norm(whole))
    assert d <= bound, d
    p = oracle_plane(sp)
    ref = james.solve(p, rho_np, dgf.dgf(p))
    assert rel_l2(p, phi.cpu().numpy(), ref) <= (1e-10 if precision == 0 else 1e-7)
    # argument checks
    one = f[:1].contiguous()
    for bad in ([M], [-1], [0, 0]):
        _, rc = s.solve_modes(bad, f[:len(bad)].contiguous(), raise_on_error=False)
        assert rc == ps.ERR_ARG
    out, rc = s.solve_modes([], f[:0].contiguous())
    assert rc == ps.OK and out.numel() == 0
    s.close()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_sharded_pipeline_on_one_nccl_rank(ps):
    import torch.distributed as td
    from paper_2606_17636_gb300 import shard
    sp = SMALL["cyl_cavity"]
    rho = torch.from_numpy(clumps(sp, 52)).cuda()
    td.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % _free_port(), rank=0,
                          world_size=1)
    try:
        s = ps.Solver.from_spec(sp, precision=ps.MIXED, use_graph=False)
        whole, _ = s.solve(rho, tol=1e-10)
        whole = whole.clone()
        ms = shard.ModeShardedSolve(sp["n_r"], sp["n_tz"], s.n_modes, shard.LibraryCompute(s))
        for _ in range(2):
            phi = ms.solve(rho, tol=1e-10)
            assert ms.last_rc == ps.OK
            d = float(torch.linalg.vector_norm(phi - whole) / torch.linalg.vector_norm(whole))
            assert d <= 1e-8, d
        # the second solve's costs are the first solve's cycles per mode
        assert ms.costs[0] == max(ms.costs)
        s.close()
    finally:
        td.destroy_process_group()
