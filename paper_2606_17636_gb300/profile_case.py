"""A profiling case: one solve of a workload's geometry with host-driven
(eager) launches, so that a profiler sees every kernel on its own, and
cudaProfilerStart / cudaProfilerStop around the part to capture.

  python -m paper_2606_17636_gb300.profile_case [--n-phi N] [--precision mixed|fp64]
      [--schedule nu_pre,nu_post,n_sor,lines_r,cols_t,nu_pre_fused,nu_post_fused]
      [--tail -1|0|n] [--smooth-first]

The geometry and density are workload 3's (256 x 128 x 256 log-spherical,
r in [0.05, 20], lognormal density); --n-phi changes the azimuthal
resolution (a smaller case of the same kernels: fewer mode planes, the
density resampled by Gaussian clumps of the workloads module).  Set-up (plan,
DGF tables) and one warm-up solve run before the profiled range, which holds
one level-0 smoothing cycle over all modes (--smooth-first) and one solve.
Start a profiler with its capture off at start (ncu --profile-from-start off).
"""
import argparse

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-phi", type=int, default=256)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--schedule", default="2,2,1,4,16,3,3")
    ap.add_argument("--tail", type=int, default=0)
    ap.add_argument("--smooth-first", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-8)
    a = ap.parse_args(argv)
    import torch

    import paper_2606_17636_gb300 as ps
    from paper_2606_17636_gb300 import workloads
    if a.n_phi == 256:
        w = workloads.workload(3)
        sp, rho_np = w["spec"], w["rho"]
    else:
        sp = workloads.spec(workloads.SPHERICAL, 256, 128, a.n_phi, workloads.LOG, 0.05, 20.0)
        rho_np = workloads._clumps(sp, workloads.rng_for(3))
    prec = ps.MIXED if a.precision == "mixed" else ps.FP64
    s = ps.Solver.from_spec(sp, precision=prec, use_graph=False)
    nu1, nu2, nsor, lines, cols, nu1f, nu2f = (int(x) for x in a.schedule.split(","))
    s.set_schedule(nu1, nu2, nsor, lines_r=lines, cols_t=cols, nu_pre_fused=nu1f, nu_post_fused=nu2f,
                   tail_planes=a.tail)
    rho = torch.from_numpy(np.ascontiguousarray(rho_np)).cuda()
    phi, _ = s.solve(rho, tol=a.tol)
    cdt = torch.complex64 if prec == ps.MIXED else torch.complex128
    e = torch.zeros((s.n_modes, sp["n_tz"], sp["n_r"]), dtype=cdt, device="cuda")
    f = torch.randn((s.n_modes, sp["n_tz"], sp["n_r"]), dtype=cdt, device="cuda")
    if a.smooth_first:
        s.stage_smooth(0, e, f, 1)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    if a.smooth_first:
        s.stage_smooth(0, e, f, 1)
    phi, rc = s.solve(rho, tol=a.tol)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    st = s.stats()
    s.close()
    print("solve rc %d, iterations %d + %d" % (rc, st["iterations_psi"], st["iterations_phi"]), flush=True)
    return rc


if __name__ == "__main__":
    raise SystemExit(main())
