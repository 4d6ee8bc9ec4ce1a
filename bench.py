#!/usr/bin/env python
"""Throughput of the spectral-multigrid Poisson solve.

Workload: 256 x 128 x 256 log-spherical grid, r in [0.05, 20], seeded
lognormal density (see paper_2606_17636_gb300/workloads.py, workload 3),
tolerance 1e-8 relative residual per mode, mixed precision (FP32 V-cycles in
FP64 iterative refinement); the plain FP64 GPU path is timed on the same
input for comparison.  One step = one full solve (density in, potential out).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own replica of the problem on its own
GPU (independent problems: weak scaling, no collective on the data path);
rank 0 prints one JSON line with the whole-job throughput.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = 3
TOL = 1e-8
METRIC = "solves/s at 256x128x256 log-spherical: mixed vs FP64 GPU at 1e-8 rel residual"
CONFIG = {"workload": "log-spherical 256x128x256, r in [0.05, 20], lognormal density (k^-3), "
                      "tol 1e-8 per mode", "n_r": 256, "n_theta": 128, "n_phi": 256,
          "geometry": "spherical", "spacing": "log", "precision": "mixed (FP32 V-cycles, FP64 residual/update)"}


def args_():
    a = argparse.ArgumentParser()
    a.add_argument("--gpus", type=int, default=1)
    a.add_argument("--steps", type=int, default=40)
    a.add_argument("--warmup", type=int, default=3)
    a.add_argument("--impl", default="ours", choices=["ours", "reference"])
    a.add_argument("--no-baseline", action="store_true")
    a.add_argument("--no-serving", action="store_true", help="skip the sixteen-problem one-graph batch")
    a.add_argument("--no-tune", action="store_true",
                   help="keep the default smoothing schedule and tile shapes (skip psolve_autotune)")
    a.add_argument("--no-setup4", action="store_true",
                   help="skip timing psolve_create for the 512 x 256 x 512 cylindrical workload")
    a.add_argument("--replicas", action="store_true",
                   help="with N > 1 GPUs: only the independent copies of the problem per GPU (weak "
                        "scaling, the headline value), without the one-problem mode-sharded measurement")
    a.add_argument("--eager", action="store_true",
                   help="host-driven loop instead of the captured graph (for per-kernel profiling)")
    return a.parse_args()


def dist():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as td
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        td.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as td
        td.barrier()


def allmax(ws, v, dev):
    if ws == 1:
        return v
    import torch
    import torch.distributed as td
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-i", str(index), "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# --------------------------------------------------------------------------
# CPU oracle baseline (the reference arm: the oracle timed as it stands)
# --------------------------------------------------------------------------
def oracle_desc(spec):
    return (spec["geometry"], spec["n_r"], spec["n_tz"], spec["n_phi"], spec["spacing"],
            spec["r_in"], spec["r_out"], spec["t_min"], spec["t_max"])


def oracle_timings(rho, spec, warmup=0, steps=3, procs=None, single_thread_repeats=0):
    """Time the oracle's full solve (Sec. 5.1 steps 2-7, all azimuthal modes,
    the real DGF tables) on the host cores: the DGF tables (setup, excluded
    from the timing as the paper excludes them) are computed first by a pool
    of `procs` spawned single-threaded workers; then `warmup` untimed and
    `steps` timed full solves with the modes spread over that pool, and
    `single_thread_repeats` timed solves in one worker process.  Returns a
    dict of seconds."""
    from oracle.pool import ModePool
    desc = oracle_desc(spec)
    out = {"procs": procs or os.cpu_count() or 1}
    with ModePool(out["procs"]) as pool:
        t0 = time.perf_counter()
        gt = pool.dgf(desc)
        out["dgf_setup_s"] = time.perf_counter() - t0
        for _ in range(warmup):
            pool.solve(desc, rho, gt)
        times = []
        for _ in range(steps):
            t0 = time.perf_counter()
            pool.solve(desc, rho, gt)
            times.append(time.perf_counter() - t0)
        out["solve_s"] = times
    if single_thread_repeats:
        with ModePool(1) as one:
            times = []
            for _ in range(single_thread_repeats):
                t0 = time.perf_counter()
                one.solve(desc, rho, gt)
                times.append(time.perf_counter() - t0)
        out["solve_1thread_s"] = times
    return out


def cpu_info():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def reference_arm(a, ws, rank):
    """The oracle's full solve timed on the host cores, one solve per step."""
    if rank != 0:
        return
    from paper_2606_17636_gb300 import workloads
    w = workloads.workload(WORKLOAD)
    tm = oracle_timings(w["rho"], w["spec"], warmup=a.warmup, steps=a.steps)
    per = statistics.mean(tm["solve_s"])
    v = 1.0 / per
    sample = ("%d full solves (all %d modes, Sec. 5.1 steps 2-7, DGF tables computed first and "
              "excluded: %.1f s), modes spread over %d single-threaded processes"
              % (a.steps, w["spec"]["n_phi"] // 2 + 1, tm["dgf_setup_s"], tm["procs"]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG, precision="f64 (CPU oracle, sparse direct per mode)"),
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": tm["procs"], "kind": "oracle",
                             "sample": sample, "cpu": cpu_info(),
                             "median_s": statistics.median(tm["solve_s"])},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def time_solves(torch, s, rho, phi, steps, stream, tag):
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push(tag)
    ev0.record(stream)
    for _ in range(steps):
        s.solve(rho, phi, tol=TOL)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    return ev0.elapsed_time(ev1) / 1e3


def ours(a, ws, rank, local):
    import numpy as np
    import torch

    import paper_2606_17636_gb300 as ps
    from paper_2606_17636_gb300 import workloads
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0 and not a.no_baseline:      # CPU baseline first, before the GPU is timed
        w0 = workloads.workload(WORKLOAD)
        base = oracle_timings(w0["rho"], w0["spec"], steps=3, single_thread_repeats=1)
    w = workloads.workload(WORKLOAD)
    spec = w["spec"]
    stream = torch.cuda.current_stream()
    rho_host = torch.from_numpy(w["rho"]).pin_memory()
    rho = rho_host.to(dev)
    phi = torch.empty_like(rho)
    sm = ps.Solver.from_spec(spec, precision=ps.MIXED, use_graph=not a.eager)
    sd = ps.Solver.from_spec(spec, precision=ps.FP64, use_graph=not a.eager)
    # schedules and tile shapes picked by the library's autotuner on this
    # input (untimed setup, like the plan itself)
    tune = None
    if not a.no_tune:
        tune = {"mixed": sm.autotune(rho, tol=TOL, phi=phi), "fp64": sd.autotune(rho, tol=TOL, phi=phi)}
    for _ in range(max(3, a.warmup)):
        sm.solve(rho, phi, tol=TOL)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    clk = Clocks(local)
    time.sleep(0.5)                         # let the sampler start before the timed region
    t = time_solves(torch, sm, rho, phi, a.steps, stream, "bench_mixed")
    barrier(ws)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t = allmax(ws, t, dev)
    st = sm.stats()
    stages = sm.stage_times()               # the last timed solve, from its event nodes
    value = ws * a.steps / t
    # FP64 GPU path on the same input and tolerance
    phi64 = torch.empty_like(rho)
    for _ in range(2):
        sd.solve(rho, phi64, tol=TOL)
    k64 = max(2, a.steps // 2)
    t64 = allmax(ws, time_solves(torch, sd, rho, phi64, k64, stream, "bench_fp64"), dev)
    st64 = sd.stats()
    stages64 = sd.stage_times()
    fp64_value = ws * k64 / t64
    diff = float(torch.linalg.vector_norm(phi - phi64) / torch.linalg.vector_norm(phi64))
    # accuracy of the timed mixed result (tuned schedule, tol 1e-8) against a
    # tight FP64 solve (tol 1e-11, the tightest every mode reaches here);
    # relative L2, volume-weighted
    phi_t = torch.empty_like(rho)
    sd.solve(rho, phi_t, tol=1e-11)
    wv = torch.from_numpy(cell_volumes(spec)).to(dev)[:, :, None]
    err_tight = float(torch.sqrt((wv * (phi - phi_t) ** 2).sum() / (wv * phi_t ** 2).sum()))
    err_tight_plain = float(torch.linalg.vector_norm(phi - phi_t) / torch.linalg.vector_norm(phi_t))
    # end to end through the public call with host buffers: psolve_solve_host
    # uploads each solve's density from pinned host memory and downloads its
    # potential, overlapping both with the solves; every step copies its own
    # bytes (the same pinned buffers every step).  One untimed call first (it
    # allocates the staging buffers and captures the graph for them).
    phi_host = torch.empty_like(rho_host).pin_memory()
    sm.solve_host([rho_host] * 3, [phi_host] * 3, tol=TOL)
    torch.cuda.synchronize()
    barrier(ws)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    _, e2e_status, _ = sm.solve_host([rho_host] * a.steps, [phi_host] * a.steps, tol=TOL)
    ev1.record(stream)
    torch.cuda.synchronize()
    te2e = allmax(ws, ev0.elapsed_time(ev1) / 1e3, dev)
    e2e = ws * a.steps / te2e
    e2e_err = float(torch.linalg.vector_norm(phi_host.to(dev) - phi) / torch.linalg.vector_norm(phi))
    # time stepping with warm start (App. B): a sequence of slowly changing
    # densities (a growing m = 2 perturbation, 2 % over the run), each solve
    # starting from the previous Psi and Phi; all densities resident in HBM
    _, _, ph = workloads.midpoints(spec)
    pert = torch.from_numpy(np.cos(2.0 * ph)).to(dev)
    nk = a.steps + 3
    rhos = [rho * (1.0 + (0.02 * k / nk) * pert) for k in range(nk)]
    sw = ps.Solver.from_spec(spec, precision=ps.MIXED, use_graph=not a.eager)
    if not a.no_tune:
        sw.autotune(rho, tol=TOL, phi=phi)   # the mixed handle's choice, from the process cache
    sw.set_warm_start(True)
    for k in range(3):
        sw.solve(rhos[k], phi, tol=TOL)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_warm")
    ev0.record(stream)
    for k in range(3, nk):
        sw.solve(rhos[k], phi, tol=TOL)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    tw = allmax(ws, ev0.elapsed_time(ev1) / 1e3, dev)
    stw = sw.stats()
    warm = {"value": ws * a.steps / tw, "unit": "solves/s", "ms_per_step": 1e3 * tw / a.steps,
            "iterations_last": [stw["iterations_psi"], stw["iterations_phi"]],
            "density": "rho_k = rho (1 + 0.02 k / K cos 2 phi), k = 0..K+2 (first 3 untimed); "
                       "each solve starts from the previous Psi and Phi"}
    sw.close()
    del rhos
    # dominant kernel, timed alone on the same stream: one alternating-line
    # smoothing cycle of the finest level over all modes, FP32 planes
    roof = vcycle_roofline(torch, ps, sm, stream)
    roof_stream = smoother_roofline(torch, ps, sm, stream)
    fp64_peak = fp64_peak_tflops(torch)
    roof_fft = fft_roofline(torch, ps, sd, fp64_peak)
    roof_res = residual_roofline(torch, ps, sm, stream, fp64_peak)
    launches = launches_per_solve(sm, st)
    serve = serving(torch, ps, workloads) if (rank == 0 and not a.no_serving) else None
    multi = multi_density(torch, ps, workloads, w) if (rank == 0 and not a.no_serving) else None
    setup4 = setup_large(torch, ps, workloads) if (rank == 0 and not a.no_setup4) else None
    # N > 1: one problem sharded by mode over all GPUs, beside the replicas
    shard_one = sharded_measure(a, ws, rank, local, min(a.steps, 10)) if (ws > 1 and not a.replicas) else None
    if rank != 0:
        return
    cells = spec["n_r"] * spec["n_tz"] * spec["n_phi"]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(CONFIG, l2="working set ~0.45 GB per solve > 129 MB L2; no flush needed",
                       parallelism=("replicas: an independent problem per GPU" if ws > 1 else "single GPU")),
        "cell_updates_per_s": value * cells,
        "fp64_gpu": {"value": fp64_value, "unit": "solves/s", "ms_per_step": 1e3 * t64 / k64,
                     "speedup_mixed_vs_fp64": value / fp64_value, "stage_ms": stages64},
        "stage_ms": stages,
        "mixed_vs_fp64_rel_l2": diff,
        "mixed_vs_fp64_tol1e-11_rel_l2": err_tight,
        "mixed_vs_fp64_tol1e-11_rel_l2_unweighted": err_tight_plain,
        "schedule": {"mixed": sm.schedule(), "fp64": sd.schedule(),
                     "autotune": {k: {"ms": v["ms"], "candidates": v["candidates"]} for k, v in tune.items()}
                     if tune else None},
        "solver": {"iterations_psi": st["iterations_psi"], "iterations_phi": st["iterations_phi"],
                   "rel_residual_psi": st["rel_residual_psi"], "rel_residual_phi": st["rel_residual_phi"],
                   "sum_mode_cycles_psi": sum(st["cycles_psi"]), "sum_mode_cycles_phi": sum(st["cycles_phi"]),
                   "cycles_m0": [st["cycles_psi"][0], st["cycles_phi"][0]],
                   "fp64_iterations": [st64["iterations_psi"], st64["iterations_phi"]],
                   "setup_ms": st["setup_ms"], "dgf_ms": sm.setup_times()[1]},
        "e2e": {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": rho.numel() * 8,
                "api": "psolve_solve_host (copies overlapped with the solves)",
                "result_vs_device_solve_rel_l2": e2e_err,
                "d2h_bytes_per_step": phi.numel() * 8},
        "gpu_launches": launches * a.steps,
        "whole_solve_hbm": whole_solve_hbm(spec, st, 1e3 * t / a.steps, sm.n_boundary),
        "warm_timestepping": warm,
        "roofline": roof,
        "roofline_streaming": roof_stream,
        "roofline_fft": roof_fft,
        "roofline_residual": roof_res,
        "serving": serve,
        "multi_density": multi,
        "setup_workload4": setup4,
        "sharded_one_problem": shard_one,
        "clocks": clocks,
    }
    if not a.no_baseline:
        med = statistics.median(base["solve_s"])
        one = base["solve_1thread_s"][0]
        line["cpu_baseline"] = {"value": 1.0 / med, "unit": "solves/s", "cores": base["procs"], "kind": "oracle",
                                "sample": "full oracle solves of this workload (all %d modes, DGF tables "
                                          "computed first and excluded: %.1f s): median of %d with the modes "
                                          "spread over %d single-threaded processes, and 1 in one process"
                                          % (spec["n_phi"] // 2 + 1, base["dgf_setup_s"], len(base["solve_s"]),
                                             base["procs"]),
                                "single_thread": {"value": 1.0 / one, "unit": "solves/s", "cores": 1},
                                "cpu": cpu_info()}
    print(json.dumps(line), flush=True)


def sharded_measure(a, ws, rank, local, steps):
    """N > 1 GPUs: one problem of the workload solved by all ranks together,
    its azimuthal modes sharded over the GPUs (paper_2606_17636_gb300/shard.py:
    slab transforms, an all-to-all to the modes' owners, mode-subset solves,
    the reverse all-to-all; modes assigned by LPT over the previous solve's
    V-cycles).  Returns (on every rank) solves of the one problem per second
    of the whole job (strong scaling) and its end-to-end figure."""
    import numpy as np
    import torch

    import paper_2606_17636_gb300 as ps
    from paper_2606_17636_gb300 import shard, workloads
    dev = torch.device("cuda", local)
    w = workloads.workload(WORKLOAD)
    spec = w["spec"]
    stream = torch.cuda.current_stream()
    s = ps.Solver.from_spec(spec, precision=ps.MIXED, use_graph=False)
    if not a.no_tune:
        rho_full = torch.from_numpy(w["rho"]).to(dev)
        s.autotune(rho_full, tol=TOL)
        del rho_full
    ms = shard.ModeShardedSolve(spec["n_r"], spec["n_tz"], s.n_modes, shard.LibraryCompute(s))
    i0, i1 = ms.my_rows
    rho_host = torch.from_numpy(np.ascontiguousarray(w["rho"][i0:i1])).pin_memory()
    rho_rows = rho_host.to(dev)
    for _ in range(max(3, a.warmup)):
        ms.solve(rho_rows, TOL)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        phi_rows = ms.solve(rho_rows, TOL)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    t = allmax(ws, ev0.elapsed_time(ev1) / 1e3, dev)
    # end to end: the slab of the density from pinned host memory and the
    # slab of the potential back, inside the timed region
    phi_host = torch.empty((i1 - i0, spec["n_tz"], spec["n_phi"]), dtype=torch.float64).pin_memory()
    barrier(ws)
    ev0.record(stream)
    for _ in range(steps):
        rho_rows.copy_(rho_host, non_blocking=True)
        phi_rows = ms.solve(rho_rows, TOL)
        phi_host.copy_(phi_rows, non_blocking=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    te2e = allmax(ws, ev0.elapsed_time(ev1) / 1e3, dev)
    out = {"workload": "one workload-3 problem, modes sharded over %d GPUs (LPT over V-cycles, "
                       "all-to-all exchanges, host-driven mode-subset solves)" % ws,
           "scaling": "strong", "steps": steps, "value": steps / t, "unit": "solves/s",
           "ms_per_step": 1e3 * t / steps, "owners_last": [len(o) for o in ms.owners],
           "e2e": {"value": steps / te2e, "unit": "solves/s",
                   "h2d_bytes_per_step": rho_rows.numel() * 8 * ws,
                   "d2h_bytes_per_step": phi_rows.numel() * 8 * ws}}
    s.close()
    return out


def multi_density(torch, ps, workloads, w, nd=8, warm=2, runs=5):
    """One plan, nd densities of the workload's geometry per solve
    (psolve_create_multi): the workload's density and nd - 1 seeded
    variations of it, mixed precision, captured graph, tol 1e-8.  The modes of
    all densities iterate together, so the slow low modes share the late
    iterations.  Reports solves (densities) per second."""
    import numpy as np
    spec = w["spec"]
    rng = np.random.default_rng(7)
    _, _, ph = workloads.midpoints(spec)
    rhos = [w["rho"]] + [w["rho"] * (1.0 + 0.2 * rng.uniform(-1, 1) * np.cos((k + 1) * ph))[None, None, :]
                         for k in range(nd - 1)]
    rho = torch.from_numpy(np.ascontiguousarray(np.stack(rhos))).cuda()
    s = ps.Solver.from_spec(spec, precision=ps.MIXED, n_densities=nd)
    phi = torch.empty_like(rho)
    for _ in range(warm):
        s.solve(rho, phi, tol=TOL)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(runs):
        s.solve(rho, phi, tol=TOL)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    st = s.stats()
    s.close()
    return {"n_densities": nd, "solves_per_s": nd * runs / t, "ms_per_call": 1e3 * t / runs,
            "iterations": [st["iterations_psi"], st["iterations_phi"]],
            "densities": "the workload's density and %d variations rho (1 + a_k cos((k+1) phi)), "
                         "a_k uniform in [-0.2, 0.2]" % (nd - 1)}


def serving(torch, ps, workloads, warm=2, runs=5):
    """Workload 5 (serving-style): sixteen independent seeded problems of
    uneven sizes (spherical log r in [0.05, 20] and cylindrical R in [4/33, 4]
    with an inner cavity, N x N/2 x N with N in {64, 128, 256}), mixed
    precision, all in ONE captured CUDA graph (psolve_batch_*) with every
    problem on its own branch.  Reports the aggregate solves/s and the p50 /
    p99 per-problem completion latency within a launch (completion events in
    the graph), against the same problems solved one by one in FP64."""
    import numpy as np
    ws = workloads.workload(5)
    t0 = time.perf_counter()
    mixed = [ps.Solver.from_spec(w["spec"], precision=ps.MIXED) for w in ws]
    setup_s = time.perf_counter() - t0
    rhos = [torch.from_numpy(w["rho"]).cuda() for w in ws]
    phis = [torch.empty_like(r) for r in rhos]
    b = ps.Batch(mixed, rhos, phis, tol=TOL)
    for _ in range(warm):
        b.run()
    lat = []
    t0 = time.perf_counter()
    for _ in range(runs):
        lat += b.run()[1]
    t_batch = time.perf_counter() - t0
    b.close()
    for s in mixed:
        s.close()
    seq = []
    for w, r in zip(ws, rhos):
        s = ps.Solver.from_spec(w["spec"], precision=ps.FP64)
        phi = torch.empty_like(r)
        s.solve(r, phi, tol=TOL)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.solve(r, phi, tol=TOL)
        e1.record()
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1))
        s.close()
    sizes = [(w["spec"]["geometry"], w["spec"]["n_r"]) for w in ws]
    return {"workload": "16 problems: even index spherical log r in [0.05, 20], odd index cylindrical "
                        "R in [4/33, 4], z in [-2, 2]; N x N/2 x N, N in {64, 128, 256}; Gaussian clumps; "
                        "tol 1e-8",
            "sizes": [("sph" if g == 0 else "cyl") + str(n) for g, n in sizes],
            "one_graph_mixed": {"solves_per_s": len(ws) * runs / t_batch,
                                "latency_ms_p50": float(np.percentile(lat, 50)),
                                "latency_ms_p99": float(np.percentile(lat, 99)),
                                "launches_timed": runs, "host_wall_per_launch_ms": 1e3 * t_batch / runs},
            "sequential_fp64": {"solves_per_s": len(ws) / (sum(seq) / 1e3),
                                "latency_ms_p50": float(np.percentile(seq, 50)),
                                "latency_ms_p99": float(np.percentile(seq, 99))},
            "setup_s_16_handles": setup_s}


def cell_volumes(spec):
    """Cell volumes per unit azimuth [n_r][n_tz] from the face positions (the
    weights of the volume-weighted relative L2 error)."""
    import numpy as np
    from paper_2606_17636_gb300 import workloads
    fr = workloads._law(spec["r_in"], spec["r_out"], spec["n_r"], spec["spacing"])
    ft = workloads._law(spec["t_min"], spec["t_max"], spec["n_tz"], workloads.UNIFORM)
    if spec["geometry"] == workloads.SPHERICAL:
        return np.outer(np.diff(fr ** 3) / 3.0, -np.diff(np.cos(ft)))
    return np.outer(np.diff(fr ** 2) / 2.0, np.diff(ft))


def whole_solve_hbm(spec, st, ms, nb):
    """The whole mixed solve against the measured HBM bandwidth: the
    algorithmic bytes of solve_algorithmic_bytes (with this solve's
    per-mode cycle counts) over its time.  A low fraction says the solve is
    bound by latency and the FP64 pipe, not by bytes."""
    b = solve_algorithmic_bytes(spec, st, nb)
    pk = peaks().get("hbm_gbs")
    ach = b / (ms * 1e-3) / 1e9
    return {"algorithmic_bytes": b, "achieved_gbs": ach, "peak_gbs": pk,
            "frac": (ach / pk) if pk else None, "ms": ms}


def solve_algorithmic_bytes(spec, st, nb):
    """What a mixed solve must move through HBM (the per-unknown model of
    the solver's design: per real unknown of a mode plane, a V-cycle moves
    152 B (two smoothing directions x 4 cycles x 12 B, residual and
    restriction 9 B, prolongation and correction 9 B, times 4/3 for the
    coarser levels) and a refinement step 40 B (FP64 residual 20 B, FP64
    update 20 B)); plus both transforms (32 B per cell) and one read of the
    DGF tables."""
    unknowns = 2 * spec["n_r"] * spec["n_tz"]          # Re and Im of one mode plane
    cycles = sum(st["cycles_psi"]) + sum(st["cycles_phi"])
    steps = cycles + 2 * len(st["cycles_psi"])         # residual evaluations: cycles + 1 per mode and solve
    cells = spec["n_r"] * spec["n_tz"] * spec["n_phi"]
    dgf = 8 * len(st["cycles_psi"]) * nb * nb          # nb boundary points per mode
    return unknowns * (152 * cycles + 40 * steps) + 32 * cells + dgf


def launches_per_solve(s, st):
    """Kernel launches of one solve: the fixed ones plus each multigrid
    loop.  A loop iteration is the residual/retirement kernel and, while
    planes remain, one V-cycle (on every level below the fused one nu_pre
    smoothing cycles of two passes, a restriction, later a prolongation and
    nu_post cycles; the fused V-cycle) and the update, which rides on the
    last smoothing pass when there is one.  With I iterations
    the loop runs I + 1 residuals and I V-cycles; with the cluster-resident
    tail (P planes) it hands over after the first iteration k that leaves at
    most P planes active (k + 1 residuals and V-cycles), then one tail
    launch finishes them."""
    sc = s.schedule()
    first = s.fused_level()
    vcycle = first * (2 * sc["nu_pre"] + 1 + 1 + 2 * sc["nu_post"]) + 1   # + fused
    vcycle += 0 if (first > 0 and sc["nu_post"] > 0) else 1             # + update
    fixed = 1 + 1 + 3 + 1 + 1 + 1           # fft, init x2, screening/boundary/ghosts, ifft, status
    tail_planes = s.tail()[0]

    def loop(cycles):
        it = max(cycles)
        if tail_planes > 0:
            for k in range(it):
                if 0 < sum(1 for c in cycles if c > k) <= tail_planes:
                    return (k + 1) * (1 + vcycle) + 1
        return (it + 1) + it * vcycle
    return fixed + loop(st["cycles_psi"]) + loop(st["cycles_phi"])


# FP32 flops per cell of a fused smoothed level and V-cycle: a line
# relaxation pass costs 16 + 16 n_sor per cell (neighbour-line source 10,
# inverse diagonal 6, each even-odd SOR sweep 16); nu_pre + nu_post cycles of
# 2 passes each; defect restriction and prolongation add 40 (424 for the
# default schedule nu = (2, 2), n_sor = 2).
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of full-batch
# launches on workload 3 (all 129 modes), from the ncu captures of the
# profiling case (python -m paper_2606_17636_gb300.profile_case
# --schedule 2,1,2,4,16,2,2 --smooth-first): one k_vsmem launch, one
# finest-level smoothing cycle (k_rpass2 + k_tpass2) and the first stencil
# launch of k_residual.  They hold for the kernels as captured; a changed
# kernel needs a new capture.
VSMEM_TRAFFIC_BYTES = 13804288 + 1536
SMOOTH_CYCLE_TRAFFIC_BYTES = 67736064 + 8047872 + 67791616 + 6110720
RESIDUAL_TRAFFIC_BYTES = 169755136 + 18508544
# ncu sm__inst_executed_pipe_fp64 (percent of peak, sustained active) of the
# kernels bound by the FP64 pipe: k_residual and k_fft_fwd from the same
# capture at 256 x 128 x 256, k_fft_inv and k_boundary at 256 x 128 x 128
# (the same kernels with 65 mode planes)
FP64_PIPE_PCT = {"k_residual": 77.5, "k_fft_fwd": 83.8, "k_fft_inv": 82.3, "k_boundary": 87.1}


def vcycle_flops_per_cell(sched):
    """On the fused levels (their own smoothing counts when set)."""
    nu = (sched["nu_pre_fused"] or sched["nu_pre"]) + (sched["nu_post_fused"] or sched["nu_post"])
    return nu * 2 * (16 + 16 * sched["n_sor"]) + 40
def setup_large(torch, ps, workloads):
    """psolve_create of workload 4 (cylindrical, uniform R in [0.2, 4],
    z in [-1, 1], 512 x 256 x 512; auxiliary-window DGF with 1536 boundary
    points x 257 modes): wall time and its DGF part, on the device the bench
    runs on.  Untimed by the solve clock; one handle, destroyed after."""
    sp = workloads.BASE[4][0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = ps.Solver.from_spec(sp, precision=ps.MIXED, use_graph=False)
    wall = time.perf_counter() - t0
    setup_ms, dgf_ms = s.setup_times()
    nb = s.n_boundary
    s.close()
    torch.cuda.empty_cache()
    return {"workload": "cylindrical 512x256x512, R in [0.2, 4], z in [-1, 1]",
            "create_s": wall, "setup_ms": setup_ms, "dgf_ms": dgf_ms,
            "boundary_points": nb, "modes": sp["n_phi"] // 2 + 1}


def fp32_peak_tflops(torch):
    """SMs (from the device) x 128 FP32 lanes x 2 (FMA) x the maximum SM clock
    (MEASURED_PEAKS.json, else 2.07 GHz)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = peaks().get("sm_max_mhz") or 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


def fp64_peak_tflops(torch):
    """Measured FP64 rate of this GPU: a cuBLAS FP64 GEMM (torch.matmul of
    4096 x 4096 float64 matrices), best of three, 2 N^3 flops."""
    n = 4096
    a = torch.randn((n, n), dtype=torch.float64, device="cuda")
    b = torch.randn((n, n), dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    return 2.0 * n ** 3 / best / 1e12


def fft_roofline(torch, ps, s, fp64_peak, reps=20):
    """The forward azimuthal transform (k_fft_fwd) of the workload, timed
    alone through psolve_stage_forward with CUDA events.  Work: n_r n_tz / 2
    complex FFTs of n_phi points (two real rows packed in one), 5 N log2 N
    flops each, against the measured FP64 GEMM rate: the kernel runs on the
    FP64 pipe (ncu: FP64_PIPE_PCT)."""
    import math
    n_r, n_tz, n_phi = s.grid
    rho = torch.rand((n_r, n_tz, n_phi), dtype=torch.float64, device="cuda")
    for _ in range(3):
        s.stage_forward(rho)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        s.stage_forward(rho)
    e1.record()
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / reps
    flops = (n_r * n_tz / 2) * 5 * n_phi * math.log2(n_phi)
    ach = flops / dt / 1e12
    return {"kernel": "forward azimuthal transform k_fft_fwd", "bound": "fp64", "achieved": ach,
            "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
            "peak_source": "measured: cuBLAS FP64 GEMM 4096^3 on this GPU",
            "ncu_fp64_pipe_pct": FP64_PIPE_PCT["k_fft_fwd"],
            "algorithmic_flops_per_launch": flops, "avg_ms": dt * 1e3,
            "bytes_per_launch": 8.0 * n_r * n_tz * n_phi + 16.0 * n_r * n_tz * (n_phi // 2 + 1)}


def residual_roofline(torch, ps, s, stream, fp64_peak, reps=20):
    """The refinement's FP64 defect (k_residual) over all modes at the
    finest level, timed alone through psolve_stage_residual (each call: the
    full active list, then the kernel) with CUDA events on the library's
    stream.  Algorithmic work per complex cell: 20 FP64 flops (per real
    component f minus five stencil products; the mode's diagonal is part of
    the operator, read from a per-mode table built at setup) and 40 bytes
    (read u and f as FP64 complex, write r as FP32 complex).  The kernel
    runs on the FP64 pipe
    (ncu, FP64_PIPE_PCT), so the bound is the measured FP64 rate; the HBM
    figures are given beside it."""
    M = s.n_modes
    n_r, n_tz = s.shape[0], s.shape[1]
    g = torch.Generator(device="cuda").manual_seed(7)
    u = torch.randn((M, n_tz, n_r), dtype=torch.complex128, device="cuda", generator=g)
    f = torch.randn((M, n_tz, n_r), dtype=torch.complex128, device="cuda", generator=g)
    for _ in range(3):
        s.stage_residual(f, u)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        s.stage_residual(f, u)
    ev1.record(stream)
    torch.cuda.synchronize()
    dt = ev0.elapsed_time(ev1) / 1e3 / reps
    cells = M * n_tz * n_r
    flops, bytes_ = 20.0 * cells, 40.0 * cells
    ach = flops / dt / 1e12
    pk = peaks().get("hbm_gbs")
    full = M == 129 and (n_r, n_tz) == (256, 128)
    return {"kernel": "FP64 residual k_residual (finest level, all %d modes)" % M,
            "bound": "fp64", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": ach / fp64_peak, "peak_source": "measured: cuBLAS FP64 GEMM 4096^3 on this GPU",
            "ncu_fp64_pipe_pct": FP64_PIPE_PCT["k_residual"],
            "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": bytes_,
            "hbm_achieved_gbs": bytes_ / dt / 1e9,
            "hbm_frac": (bytes_ / dt / 1e9 / pk) if pk else None,
            "traffic": RESIDUAL_TRAFFIC_BYTES if full else None,
            "traffic_unit": "bytes per launch (ncu)", "avg_ms": dt * 1e3,
            "note": "each timed call also launches the small active-list reset kernel"}


def vcycle_roofline(torch, ps, s, stream):
    """The dominant kernel: the fused coarse V-cycle (k_vsmem, one block per
    mode plane, levels held in shared memory), all modes, timed alone
    through psolve_stage_vcycle with CUDA events on the library's stream.
    Algorithmic work per launch: M x sum over the fused smoothed levels of
    cells x vcycle_flops_per_cell(schedule) FP32 flops, plus the separable solve
    of the coarsest level (8 n_r n_t^2 + 10 n_r n_t per mode: FP32 polar
    transforms, FP64 radial sweeps)."""
    M = s.n_modes
    lev = s.fused_level()
    n_r, n_tz = s.shape[0], s.shape[1]
    peak32, sms, mhz = fp32_peak_tflops(torch)
    f = torch.randn((M, n_tz >> lev, n_r >> lev), dtype=torch.complex64, device="cuda")
    for _ in range(3):
        s.stage_vcycle(f)
    reps = 20
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_vcycle")
    ev0.record(stream)
    for _ in range(reps):
        s.stage_vcycle(f)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    dt = ev0.elapsed_time(ev1) / 1e3 / reps
    cells, l = 0, lev
    while l < s.n_levels - 1:
        cells += (n_r >> l) * (n_tz >> l)
        l += 1
    cr, ct = n_r >> (s.n_levels - 1), n_tz >> (s.n_levels - 1)
    # separable coarsest solve: two transforms along theta (2 components;
    # FP32 in the mixed path, counted in the general form) and n_theta
    # Thomas solves along r (FP64)
    flops = M * (cells * vcycle_flops_per_cell(s.schedule()) + 8 * cr * ct * ct + 10 * cr * ct)
    ach = flops / dt / 1e12
    return {"kernel": "fused coarse V-cycle k_vsmem (levels %d..%d in shared memory, all %d modes)"
                      % (lev, s.n_levels - 1, M),
            "bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s",
            "frac": ach / peak32,
            "peak_source": "derived: %d SMs (device property) x 128 FP32 lanes x 2 (FMA) x %.0f MHz" % (sms, mhz),
            "traffic": VSMEM_TRAFFIC_BYTES if M == 129 and (n_r, n_tz) == (256, 128) else None,
            "traffic_unit": "bytes per launch (ncu)", "algorithmic_flops_per_launch": flops, "avg_ms": dt * 1e3,
            "note": "one block per mode plane: latency-bound line relaxations"}


def smoother_roofline(torch, ps, s, stream):
    """One alternating-line smoothing cycle (radial zebra pass + polar zebra
    pass, 2 launches) on the finest level over all modes in FP32, timed with
    CUDA events.  Algorithmic bytes per cell per cycle: each zebra pass reads
    e once and f once and writes e once over the plane (8 B float2 each),
    twice (radial, polar): 2 x 24 B = 48 B per complex cell."""
    M = s.n_modes
    n_r, n_tz = s.shape[0], s.shape[1]
    e = torch.zeros((M, n_tz, n_r), dtype=torch.complex64, device="cuda")
    f = torch.randn((M, n_tz, n_r), dtype=torch.complex64, device="cuda")
    for _ in range(3):
        s.stage_smooth(0, e, f, 1)
    reps = 20
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_smoother")
    ev0.record(stream)
    s.stage_smooth(0, e, f, reps)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    dt = ev0.elapsed_time(ev1) / 1e3 / reps
    bytes_ = 48.0 * M * n_tz * n_r
    pk = peaks().get("hbm_gbs")
    ach = bytes_ / dt / 1e9
    return {"kernel": "finest-level smoothing cycle (k_rpass2 + k_tpass2, FP32, all modes)",
            "bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s",
            "frac": (ach / pk) if pk else None, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": SMOOTH_CYCLE_TRAFFIC_BYTES if M == 129 and (n_r, n_tz) == (256, 128) else None,
            "traffic_unit": "bytes per cycle (ncu, two launches)",
            "algorithmic_bytes_per_launch_set": bytes_, "avg_ms": dt * 1e3}


def main():
    a = args_()
    ws, rank, local = dist()
    if a.impl == "reference":
        reference_arm(a, ws, rank)
    else:
        ours(a, ws, rank, local)
    if ws > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
