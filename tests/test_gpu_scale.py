"""Scale invariance of the solve.  The problem is linear and the convergence
test (App. B) compares ratios of volume-weighted sums of squares, so a density
scaled by a power of two gives the solution scaled by the same power, with
the same per-mode cycle counts.  The scales put the squares of the right-hand
side and of the residual outside binary32's range (below its smallest
subnormal, above its largest finite value), where sums of squares taken
plainly in FP32 would vanish (every mode "converged" before its first
V-cycle) or overflow (every mode non-finite).  2^-100 is the magnitude of
4 pi G rho for gas densities in cgs units."""
import numpy as np
import pytest

from gpu_helpers import SMALL, clumps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import paper_2606_17636_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("key", ["sph_log", "cyl_cavity"])
@pytest.mark.parametrize("prec,k", [("MIXED", -80), ("MIXED", 64), ("FP64", -100), ("FP64", 200)])
def test_solution_scales_with_the_density(ps, key, prec, k):
    sp = SMALL[key]
    rho = clumps(sp, 41)
    tol = 1e-8
    s = ps.Solver.from_spec(sp, precision=getattr(ps, prec))
    phi, _ = s.solve(torch.from_numpy(rho).cuda(), tol=tol)
    st = s.stats()
    phi_s, _ = s.solve(torch.from_numpy(np.ldexp(rho, k)).cuda(), tol=tol)
    st_s = s.stats()
    s.close()
    assert all(v == 0 for v in st_s["status"]), st_s["status"]
    assert st_s["rel_residual_psi"] <= tol and st_s["rel_residual_phi"] <= tol
    for c in ("cycles_psi", "cycles_phi"):
        assert max(abs(a - b) for a, b in zip(st[c], st_s[c])) <= 1, (c, st[c], st_s[c])
    a, b = np.ldexp(phi_s.cpu().numpy(), -k), phi.cpu().numpy()
    err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert err <= 1e-7, err
