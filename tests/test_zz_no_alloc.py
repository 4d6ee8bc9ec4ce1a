"""The allocation-free smoothing entry point (psolve_stage_smooth_static),
called through the C ABI, against psolve_stage_smooth on the same inputs.

Collected last, so that it runs both alone in a fresh process and after the
other GPU tests have used the device."""
import ctypes

import numpy as np
import pytest

from gpu_helpers import SMALL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import paper_2606_17636_gb300 as m
    m.lib()
    return m


def _planes(shape, precision, seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return torch.from_numpy(z).to(torch.complex128 if precision == 0 else torch.complex64).cuda()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _compare(got, ref, precision):
    """The static entry point runs the same kernels with the same grid,
    active list and tile shapes as psolve_stage_smooth: the results are
    bitwise equal (a stale or overlapping scratch plane would show)."""
    assert torch.equal(got, ref), (got - ref).abs().max().item()


@pytest.mark.parametrize("key,precision", [("sph_log", 0), ("sph_log", 1), ("cyl_axis", 1),
                                           ("cyl_cavity", 0), ("sph_partial", 1)])
def test_static_smooth_matches_smooth_on_two_calls_in_a_row(ps, key, precision):
    L = ps.lib()
    sp = SMALL[key]
    s = ps.Solver.from_spec(sp, precision=precision, use_graph=False)
    M = s.n_modes
    # two calls in a row (different data, cycles and levels), then the
    # existing entry point on the same inputs
    cases = [(0, 1, 11), (1, 2, 12), (0, 2, 13)]
    inputs, outs = [], []
    for level, cycles, seed in cases:
        shape = (M, sp["n_tz"] >> level, sp["n_r"] >> level)
        e = _planes(shape, precision, seed)
        f = _planes(shape, precision, seed + 100)
        got = e.clone()
        rc = L.psolve_stage_smooth_static(s.h, level, precision, _ptr(got), _ptr(f), cycles)
        assert rc == ps.OK, ps.last_error()
        inputs.append((e, f))
        outs.append(got)
    for (level, cycles, _), (e, f), got in zip(cases, inputs, outs):
        ref = e.clone()
        rc = L.psolve_stage_smooth(s.h, level, precision, _ptr(ref), _ptr(f), cycles)
        assert rc == ps.OK, ps.last_error()
        _compare(got, ref, precision)
    s.close()


def test_static_smooth_rejects_levels_above_the_static_limit(ps):
    from paper_2606_17636_gb300 import workloads
    L = ps.lib()
    sp = workloads.spec(workloads.SPHERICAL, 128, 128, 256, workloads.LOG, 0.05, 20.0)
    s = ps.Solver.from_spec(sp, precision=ps.FP64, use_graph=False)
    M = s.n_modes
    limit = ps.STATIC_SCRATCH_BYTES
    assert M * 128 * 128 * 16 > limit          # level 0 does not fit
    e = _planes((M, 128, 128), 0, 3)
    f = _planes((M, 128, 128), 0, 4)
    before = e.clone()
    assert L.psolve_stage_smooth_static(s.h, 0, 0, _ptr(e), _ptr(f), 1) == ps.ERR_ARG
    assert "static limit" in ps.last_error()
    assert torch.equal(e, before)
    # level 1 fits and still agrees with the existing entry point, twice
    for seed in (5, 6):
        e1 = _planes((M, 64, 64), 0, seed)
        f1 = _planes((M, 64, 64), 0, seed + 10)
        got, ref = e1.clone(), e1.clone()
        assert L.psolve_stage_smooth_static(s.h, 1, 0, _ptr(got), _ptr(f1), 2) == ps.OK, ps.last_error()
        assert L.psolve_stage_smooth(s.h, 1, 0, _ptr(ref), _ptr(f1), 2) == ps.OK, ps.last_error()
        _compare(got, ref, 0)
    s.close()


def test_static_smooth_allocates_no_device_memory(ps):
    """After a first call (which looks up the static array's address), further
    calls at different levels and cycle counts leave the device's free memory
    unchanged: the step's scratch is the static array, nothing is allocated."""
    L = ps.lib()
    sp = SMALL["sph_log"]
    s = ps.Solver.from_spec(sp, precision=1, use_graph=False)
    M = s.n_modes
    bufs = []
    for level, seed in ((0, 21), (1, 22)):
        shape = (M, sp["n_tz"] >> level, sp["n_r"] >> level)
        bufs.append((level, _planes(shape, 1, seed), _planes(shape, 1, seed + 1)))
    level, e, f = bufs[0]
    assert L.psolve_stage_smooth_static(s.h, level, 1, _ptr(e), _ptr(f), 1) == ps.OK, ps.last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for cycles in (1, 3, 2):
        for level, e, f in bufs:
            assert L.psolve_stage_smooth_static(s.h, level, 1, _ptr(e), _ptr(f), cycles) == ps.OK, ps.last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    s.close()
