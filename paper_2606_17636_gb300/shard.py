"""Mode-sharded solve of one problem over several GPUs (one rank per GPU).

The azimuthal modes of Sec. 2.2 are independent through the two Helmholtz
solves, the screening mass and the boundary convolution (Sec. 5.1 steps
3-6), so a problem shards by mode.  The exchange steps mirror the paper's
own parallel layout (Sec. 5.2: the transform runs on the processes' own
cells, the multigrid per mode):

1. every rank transforms its radial slab of the density along phi
   (``psolve_stage_forward_rows``): [M][n_tz][rows] complex;
2. an all-to-all moves each mode's slab pieces to the rank that owns the
   mode, which assembles the mode's full (r, theta) / (R, z) planes;
3. every rank runs steps 3-6 for its own modes (``psolve_solve_modes``);
4. the reverse all-to-all returns every mode's potential, restricted to each
   rank's slab, for the inverse transform of that slab.

Modes are assigned by longest-processing-time-first over a cost per mode: the
V-cycles each mode took in the previous solve (App. B: m = 0 is by far the
slowest), with a decreasing estimate before the first solve.  The exchange
moves FP64 complex planes as flat float64 buffers with
``torch.distributed.all_to_all_single`` (NCCL on GPUs, gloo on CPU ranks).

The compute steps are a pluggable object (``LibraryCompute`` runs the CUDA
library); the exchange and bookkeeping here are plain tensor moves.
"""
import torch
import torch.distributed as dist


def lpt_assign(costs, n_ranks):
    """Longest processing time first: modes sorted by decreasing cost (ties:
    lower mode first), each given to the rank with the smallest load so far
    (ties: lower rank).  Returns the sorted mode list of every rank."""
    load = [0.0] * n_ranks
    owners = [[] for _ in range(n_ranks)]
    for m in sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k)):
        r = min(range(n_ranks), key=lambda q: (load[q], q))
        owners[r].append(m)
        load[r] += float(costs[m])
    return [sorted(o) for o in owners]


def initial_costs(n_modes):
    """Cost estimate before any solve: App. B's V-cycle counts fall from
    about 16 at m = 0 to one cycle for m >~ 30."""
    return [1.0 + 15.0 / (1.0 + m) for m in range(n_modes)]


def radial_slabs(n_r, n_ranks):
    """Contiguous radial row ranges [i0, i1), as even as possible."""
    base, extra = divmod(n_r, n_ranks)
    out, i0 = [], 0
    for q in range(n_ranks):
        i1 = i0 + base + (1 if q < extra else 0)
        out.append((i0, i1))
        i0 = i1
    return out


def _flat(t):
    return torch.view_as_real(t).reshape(-1) if t.is_complex() else t.reshape(-1)


class LibraryCompute:
    """The CUDA library's steps for one rank (a full handle of the problem)."""

    def __init__(self, solver):
        self.s = solver

    def forward_rows(self, rho_rows):
        return self.s.stage_forward_rows(rho_rows)

    def solve_modes(self, modes, f_planes, tol):
        phi, rc = self.s.solve_modes(modes, f_planes, tol=tol, raise_on_error=False)
        st = self.s.stats()
        cycles = [st["cycles_psi"][m] + st["cycles_phi"][m] for m in modes]
        return phi, cycles, rc

    def inverse_rows(self, phi_hat_rows):
        return self.s.stage_inverse_rows(phi_hat_rows)


class ModeShardedSolve:
    """One problem solved by every rank of the process group together."""

    def __init__(self, n_r, n_tz, n_modes, compute, group=None):
        self.n_r, self.n_tz, self.M = n_r, n_tz, n_modes
        self.compute = compute
        self.group = group
        self.rank = dist.get_rank(group)
        self.ws = dist.get_world_size(group)
        self.slabs = radial_slabs(n_r, self.ws)
        self.costs = initial_costs(n_modes)
        self.owners = lpt_assign(self.costs, self.ws)
        self.last_rc = 0

    @property
    def my_rows(self):
        return self.slabs[self.rank]

    def _exchange(self, pieces_out, shapes_in, device):
        """all_to_all of complex tensors: pieces_out[q] goes to rank q, and
        a tensor of shapes_in[q] arrives from rank q."""
        send = torch.cat([_flat(p.contiguous()) for p in pieces_out])
        in_splits = [2 * p.numel() for p in pieces_out]
        out_splits = [2 * s[0] * s[1] * s[2] for s in shapes_in]
        recv = torch.empty(sum(out_splits), dtype=torch.float64, device=device)
        dist.all_to_all_single(recv, send, out_splits, in_splits, group=self.group)
        out, o = [], 0
        for s, n in zip(shapes_in, out_splits):
            out.append(torch.view_as_complex(recv[o:o + n].view(*s, 2)))
            o += n
        return out

    def forward_exchange(self, f_rows):
        """[M][n_tz][my rows] -> this rank's modes as full planes
        [n_own][n_tz][n_r] (list order of self.owners[rank])."""
        mine = self.owners[self.rank]
        idx = [torch.tensor(o, dtype=torch.long, device=f_rows.device) for o in self.owners]
        pieces = [f_rows.index_select(0, i) if len(o) else f_rows[:0] for i, o in zip(idx, self.owners)]
        shapes = [(len(mine), self.n_tz, i1 - i0) for (i0, i1) in self.slabs]
        parts = self._exchange(pieces, shapes, f_rows.device)
        return torch.cat(parts, dim=2).contiguous() if mine else f_rows.new_zeros((0, self.n_tz, self.n_r))

    def reverse_exchange(self, phi_planes, device):
        """This rank's modes [n_own][n_tz][n_r] -> every mode on my rows
        [M][n_tz][my rows]."""
        i0, i1 = self.my_rows
        pieces = [phi_planes[:, :, a:b] for (a, b) in self.slabs]
        shapes = [(len(o), self.n_tz, i1 - i0) for o in self.owners]
        parts = self._exchange(pieces, shapes, device)
        out = torch.empty((self.M, self.n_tz, i1 - i0), dtype=torch.complex128, device=device)
        for o, part in zip(self.owners, parts):
            if o:
                out[torch.tensor(o, dtype=torch.long, device=device)] = part
        return out

    def update_costs(self, cycles_mine):
        """All ranks learn every mode's V-cycles of this solve; the next
        solve's owners follow from them by LPT."""
        mine = self.owners[self.rank]
        c = torch.zeros(self.M, dtype=torch.float64)
        for m, v in zip(mine, cycles_mine):
            c[m] = float(v)
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        c = c.to(dev)
        dist.all_reduce(c, group=self.group)
        self.costs = [max(1.0, float(x)) for x in c.cpu()]
        self.owners = lpt_assign(self.costs, self.ws)

    def solve(self, rho_rows, tol=1e-8):
        """rho_rows: this rank's radial slab [rows][n_tz][n_phi] (FP64);
        returns the potential on the same rows."""
        f_rows = self.compute.forward_rows(rho_rows)
        planes = self.forward_exchange(f_rows)
        phi_planes, cycles, rc = self.compute.solve_modes(self.owners[self.rank], planes, tol)
        phi_hat_rows = self.reverse_exchange(phi_planes, f_rows.device)
        out = self.compute.inverse_rows(phi_hat_rows)
        self.last_rc = rc
        self.update_costs(cycles)
        return out
