"""The mode-sharded solve's host logic (paper_2606_17636_gb300/shard.py) on
CPU ranks: longest-processing-time assignment of modes by cost (App. B: m = 0
is the slowest mode), radial slabs, and the two all-to-all exchanges, which
must reproduce the single-rank arrays bit for bit.  The compute steps are a
stand-in here (a transform along phi per row, a per-mode map that reads the
whole plane in order, and the inverse transform); on GPUs they are the
library's slab transforms and mode-subset solve."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2606_17636_gb300 import shard  # noqa: E402


def test_lpt_balances_a_skewed_cycle_profile():
    # App. B-like profile: m = 0 needs 40 cycles, m = 1 16, then falling fast
    costs = [40, 16, 9, 6, 4, 3, 3, 2, 2, 2] + [1] * 119
    total = sum(costs)
    for n in (2, 3, 4, 8):
        owners = shard.lpt_assign(costs, n)
        assert sorted(m for o in owners for m in o) == list(range(len(costs)))
        loads = [sum(costs[m] for m in o) for o in owners]
        # LPT: the largest load is within the larger of the biggest item and
        # 4/3 of the mean (Graham's bound for LPT)
        assert max(loads) <= max(max(costs), 4.0 / 3.0 * total / n) + 1e-9, (n, loads)
        # m = 0 dominates: it sits on a rank of its own when it exceeds the mean
        if costs[0] >= total / n:
            r0 = next(q for q, o in enumerate(owners) if 0 in o)
            assert owners[r0] == [0] or loads[r0] <= costs[0] + max(costs[1:]), owners[r0]
        # contiguous blocks of modes do worse on this profile
        blocks = [list(range(q * len(costs) // n, (q + 1) * len(costs) // n)) for q in range(n)]
        assert max(loads) <= max(sum(costs[m] for m in b) for b in blocks)


def test_lpt_is_deterministic_and_handles_ties():
    assert shard.lpt_assign([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    assert shard.lpt_assign([5], 3) == [[0], [], []]
    assert shard.lpt_assign(shard.initial_costs(5), 1) == [[0, 1, 2, 3, 4]]


def test_radial_slabs_cover_the_rows():
    for n_r, n in ((256, 8), (256, 3), (7, 4), (4, 4)):
        s = shard.radial_slabs(n_r, n)
        assert s[0][0] == 0 and s[-1][1] == n_r
        assert all(a[1] == b[0] for a, b in zip(s, s[1:]))
        assert max(b - a for a, b in s) - min(b - a for a, b in s) <= 1


class _Compute:
    """Deterministic stand-ins for the three compute steps."""

    def __init__(self, n_phi):
        self.n_phi = n_phi

    def forward_rows(self, rho_rows):
        f = torch.fft.rfft(rho_rows, dim=2) / self.n_phi          # [rows][n_tz][M]
        return f.permute(2, 1, 0).contiguous()                    # [M][n_tz][rows]

    def solve_modes(self, modes, planes, tol):
        # reads every row of each full plane in order: a wrong assembly of
        # the slabs changes the result
        out = torch.cumsum(planes, dim=2) * torch.tensor([m + 1.0 for m in modes],
                                                         dtype=torch.float64)[:, None, None]
        return out, [3 * m + 1 for m in modes], 0

    def inverse_rows(self, phi_hat_rows):
        x = phi_hat_rows.permute(2, 1, 0)                          # [rows][n_tz][M]
        return torch.fft.irfft(x * self.n_phi, n=self.n_phi, dim=2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q, n_r, n_tz, n_phi):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as td
    from paper_2606_17636_gb300 import shard as sh
    td.init_process_group("gloo", rank=rank, world_size=ws)
    g = torch.Generator().manual_seed(7)
    rho = torch.rand((n_r, n_tz, n_phi), generator=g, dtype=torch.float64)
    comp = _Compute(n_phi)
    s = sh.ModeShardedSolve(n_r, n_tz, n_phi // 2 + 1, comp)
    i0, i1 = s.my_rows
    out = []
    for _ in range(2):     # the second solve uses owners from the first one's cycles
        f_rows = comp.forward_rows(rho[i0:i1].contiguous())
        planes = s.forward_exchange(f_rows)
        out.append((s.owners[rank][:], planes.clone(), s.solve(rho[i0:i1].contiguous())))
    q.put((rank, (i0, i1), out, s.costs))
    td.barrier()
    td.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_gloo_ranks_reproduce_the_single_rank_arrays(ws):
    n_r, n_tz, n_phi = 11, 4, 16
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, ws, port, q, n_r, n_tz, n_phi)) for k in range(ws)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # single-rank reference: the same steps on the whole array
    g = torch.Generator().manual_seed(7)
    rho = torch.rand((n_r, n_tz, n_phi), generator=g, dtype=torch.float64)
    comp = _Compute(n_phi)
    f_all = comp.forward_rows(rho)
    M = n_phi // 2 + 1
    ref_phi = comp.inverse_rows(comp.solve_modes(list(range(M)), f_all, 0)[0])
    for step in range(2):
        owners = [r[2][step][0] for r in res]
        assert sorted(m for o in owners for m in o) == list(range(M))
        for r in res:
            mine, planes, phi_rows = r[2][step]
            # forward exchange: full planes of the rank's own modes
            assert torch.equal(planes, f_all[mine])
            # whole pipeline: the rank's rows of the single-rank potential
            i0, i1 = r[1]
            assert torch.equal(phi_rows, ref_phi[i0:i1])
    # the costs every rank learned are the cycles of every mode
    for r in res:
        assert r[3] == [float(3 * m + 1) for m in range(M)]
    # after the first solve the owners follow LPT over those costs
    assert [r[2][1][0] for r in res] == shard.lpt_assign([3 * m + 1 for m in range(M)], ws)
