"""psolve: spectral-multigrid self-gravity solver for one GPU.

Thin ctypes binding of the C ABI in ``include/psolve.h`` (same function
names).  Argument marshalling only: every step of a solve runs in the CUDA
kernels of ``_build/libpsolve.so``.  PyTorch provides device memory (the
library's workspaces come from the torch caching allocator through the
allocation hooks of ``psolve_desc``) and the CUDA stream.  There is no CPU
path: without the built library every call raises.
"""
import ctypes
import os

SPHERICAL, CYLINDRICAL = 0, 1
UNIFORM, LOG = 0, 1
FP64, MIXED = 0, 1
OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_NOT_CONVERGED, ERR_NONFINITE = 0, -1, -2, -3, -4, -5
DGF_AUTO, DGF_AUX, DGF_EXTENDED = 0, 1, 2
COARSEST_AUTO, COARSEST_SMALL, COARSEST_LARGE = 0, 1, 2
STATIC_SCRATCH_BYTES = 32 * 1024 * 1024   # PSOLVE_STATIC_SCRATCH_BYTES

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpsolve.so")
_lib = None

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Desc(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int), ("n_r", ctypes.c_int), ("n_tz", ctypes.c_int),
                ("n_phi", ctypes.c_int), ("spacing", ctypes.c_int), ("r_in", ctypes.c_double),
                ("r_out", ctypes.c_double), ("t_min", ctypes.c_double), ("t_max", ctypes.c_double),
                ("G", ctypes.c_double), ("precision", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("n_sor", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("alloc_fn", ALLOC_FN), ("free_fn", FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("dgf_construction", ctypes.c_int),
                ("coarsest_size", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_modes", ctypes.c_int), ("iterations_psi", ctypes.c_int),
                ("iterations_phi", ctypes.c_int), ("rel_residual_psi", ctypes.c_double),
                ("rel_residual_phi", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("cycles_psi", ctypes.POINTER(ctypes.c_int)),
                ("cycles_phi", ctypes.POINTER(ctypes.c_int)),
                ("status", ctypes.POINTER(ctypes.c_int))]


class Schedule(ctypes.Structure):
    _fields_ = [("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("n_sor", ctypes.c_int),
                ("lines_r", ctypes.c_int), ("cols_t", ctypes.c_int), ("nu_pre_fused", ctypes.c_int),
                ("nu_post_fused", ctypes.c_int), ("ms", ctypes.c_double),
                ("candidates", ctypes.c_int), ("cached", ctypes.c_int), ("tail_planes", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Plan(ctypes.Structure):
    _fields_ = [("n_modes", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("level_n_r", ctypes.c_int * 16), ("level_n_tz", ctypes.c_int * 16),
                ("coarsest", ctypes.c_int), ("coarse_doubles_per_mode", ctypes.c_int),
                ("coarse_check", ctypes.c_double), ("tail_cluster_ctas", ctypes.c_int),
                ("tail_smem_bytes", ctypes.c_int)]


COARSE_FORMS = {0: "separable, mirror-symmetric", 1: "separable", 2: "block-tridiagonal", 3: "dense"}


def plan_inspect(spec, precision=1, n_sor=0, coarsest_size=0):
    """The multigrid plan of a problem spec (psolve_plan_inspect: host only,
    no GPU needed): levels (n_r, n_tz), finest first, and the coarsest-level
    solve's form and factor size per mode."""
    d = Desc()
    d.geometry, d.n_r, d.n_tz, d.n_phi, d.spacing = (spec["geometry"], spec["n_r"], spec["n_tz"],
                                                     spec["n_phi"], spec["spacing"])
    d.r_in, d.r_out = spec["r_in"], spec["r_out"]
    d.t_min = spec.get("t_min") or 0.0
    d.t_max = spec.get("t_max") or 0.0
    d.precision = precision
    d.n_sor = n_sor
    d.coarsest_size = coarsest_size
    p = Plan()
    check(lib().psolve_plan_inspect(ctypes.byref(d), ctypes.byref(p)), "psolve_plan_inspect")
    return {"n_modes": p.n_modes,
            "levels": [(p.level_n_r[l], p.level_n_tz[l]) for l in range(p.n_levels)],
            "coarsest": COARSE_FORMS[p.coarsest], "coarse_doubles_per_mode": p.coarse_doubles_per_mode,
            "coarse_check": p.coarse_check, "tail_cluster_ctas": p.tail_cluster_ctas,
            "tail_smem_bytes": p.tail_smem_bytes}


def lib():
    """The loaded library; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpsolve.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
        sig = {
            "psolve_create": (I, [ctypes.POINTER(P), I, I, I, I, I, D, D]),
            "psolve_create_ex": (I, [ctypes.POINTER(P), ctypes.POINTER(Desc)]),
            "psolve_create_multi": (I, [ctypes.POINTER(P), ctypes.POINTER(Desc), I]),
            "psolve_solve": (I, [P, P, P, D]),
            "psolve_solve_batched": (I, [P, P, P, I, D]),
            "psolve_set_stream": (I, [P, P]),
            "psolve_get_stats": (I, [P, ctypes.POINTER(Stats)]),
            "psolve_get_sizes": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
            "psolve_last_error": (ctypes.c_char_p, []),
            "psolve_destroy": (V, [P]),
            "psolve_stage_forward": (I, [P, P, P]),
            "psolve_stage_inverse": (I, [P, P, P]),
            "psolve_stage_forward_rows": (I, [P, P, I, P]),
            "psolve_stage_inverse_rows": (I, [P, P, I, P]),
            "psolve_solve_modes": (I, [P, ctypes.POINTER(I), I, P, P, D]),
            "psolve_stage_mg_solve": (I, [P, P, P, D, I, ctypes.POINTER(I)]),
            "psolve_stage_smooth": (I, [P, I, I, P, P, I]),
            "psolve_stage_smooth_static": (I, [P, I, I, P, P, I]),
            "psolve_stage_vcycle": (I, [P, I, I, P, P]),
            "psolve_set_warm_start": (I, [P, I]),
            "psolve_set_tail": (I, [P, I]),
            "psolve_get_tail": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
            "psolve_get_fused_level": (I, [P, ctypes.POINTER(ctypes.c_int)]),
            "psolve_stage_restrict": (I, [P, I, I, P, P, P]),
            "psolve_stage_residual": (I, [P, I, P, P, P]),
            "psolve_get_setup_times": (I, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
            "psolve_get_stage_times": (I, [P, ctypes.POINTER(ctypes.c_float)]),
            "psolve_solve_host": (I, [P, I, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
            "psolve_stage_prolong": (I, [P, I, I, P, P]),
            "psolve_stage_screening": (I, [P, P, P]),
            "psolve_stage_boundary": (I, [P, P, P]),
            "psolve_get_dgf": (I, [P, P]),
            "psolve_get_schedule": (I, [P, ctypes.POINTER(Schedule)]),
            "psolve_set_schedule": (I, [P, ctypes.POINTER(Schedule)]),
            "psolve_autotune": (I, [P, P, P, D, ctypes.POINTER(Schedule)]),
            "psolve_plan_inspect": (I, [ctypes.POINTER(Desc), ctypes.POINTER(Plan)]),
            "psolve_batch_create": (I, [ctypes.POINTER(P), P, P, P, I, D]),
            "psolve_batch_run": (I, [P, P, ctypes.POINTER(ctypes.c_float)]),
            "psolve_batch_destroy": (V, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error():
    return lib().psolve_last_error().decode()


def check(rc, what):
    if rc != OK:
        raise PSolveError(rc, "%s failed (%d): %s" % (what, rc, last_error()))
    return rc


class PSolveError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class _TorchAllocator:
    """Allocation hooks that take the library's workspaces from torch."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        except Exception:
            return None
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, user):
        self.live.pop(ptr, None)


class Solver:
    """One planned solver (psolve_create_ex) bound to torch's current stream."""

    def __init__(self, geometry, n_r, n_tz, n_phi, spacing, r_in, r_out, t_min=None, t_max=None,
                 G=1.0, precision=MIXED, max_cycles=0, nu_pre=0, nu_post=0, n_sor=0,
                 use_graph=True, torch_alloc=True, n_densities=1, dgf_construction=DGF_AUTO,
                 coarsest_size=COARSEST_AUTO):
        import torch
        self.torch = torch
        L = lib()
        d = Desc()
        d.geometry, d.n_r, d.n_tz, d.n_phi, d.spacing = geometry, n_r, n_tz, n_phi, spacing
        d.r_in, d.r_out = r_in, r_out
        d.t_min = 0.0 if t_min is None else t_min
        d.t_max = 0.0 if t_max is None else t_max
        d.dgf_construction = dgf_construction
        d.coarsest_size = coarsest_size
        d.G, d.precision, d.max_cycles = G, precision, max_cycles
        d.nu_pre, d.nu_post, d.n_sor, d.use_graph = nu_pre, nu_post, n_sor, int(bool(use_graph))
        self._alloc = _TorchAllocator() if torch_alloc else None
        if self._alloc is not None:
            d.alloc_fn, d.free_fn = self._alloc.alloc, self._alloc.free
        self.desc = d
        self.n_densities = int(n_densities)
        # one density: [n_r][n_tz][n_phi]; several: [n_densities][n_r][n_tz][n_phi]
        self.shape = (n_r, n_tz, n_phi) if self.n_densities == 1 else (self.n_densities, n_r, n_tz, n_phi)
        self.grid = (n_r, n_tz, n_phi)
        h = ctypes.c_void_p()
        if self.n_densities == 1:
            check(L.psolve_create_ex(ctypes.byref(h), ctypes.byref(d)), "psolve_create_ex")
        else:
            check(L.psolve_create_multi(ctypes.byref(h), ctypes.byref(d), self.n_densities),
                  "psolve_create_multi")
        self.h = h
        check(L.psolve_set_stream(h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
              "psolve_set_stream")
        M, nb, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(L.psolve_get_sizes(h, ctypes.byref(M), ctypes.byref(nb), ctypes.byref(nl)),
              "psolve_get_sizes")
        self.n_modes, self.n_boundary, self.n_levels = M.value, nb.value, nl.value

    @classmethod
    def from_spec(cls, spec, **kw):
        return cls(spec["geometry"], spec["n_r"], spec["n_tz"], spec["n_phi"], spec["spacing"],
                   spec["r_in"], spec["r_out"], spec.get("t_min"), spec.get("t_max"), **kw)

    def schedule(self):
        """The smoothing schedule and tile shapes later solves use."""
        s = Schedule()
        check(lib().psolve_get_schedule(self.h, ctypes.byref(s)), "psolve_get_schedule")
        return s.as_dict()

    def set_schedule(self, nu_pre, nu_post, n_sor, lines_r=8, cols_t=0, nu_pre_fused=0, nu_post_fused=0,
                     tail_planes=-1):
        s = Schedule(nu_pre=nu_pre, nu_post=nu_post, n_sor=n_sor, lines_r=lines_r, cols_t=cols_t,
                     nu_pre_fused=nu_pre_fused, nu_post_fused=nu_post_fused, tail_planes=tail_planes)
        check(lib().psolve_set_schedule(self.h, ctypes.byref(s)), "psolve_set_schedule")

    def autotune(self, rho, tol=1e-8, phi=None):
        """Time candidate schedules and tile shapes on rho and keep the
        fastest (psolve_autotune); returns the choice."""
        torch = self.torch
        self._need(rho, self.shape, torch.float64)
        if phi is None:
            phi = torch.empty_like(rho)
        s = Schedule()
        check(lib().psolve_autotune(self.h, _ptr(rho), _ptr(phi), float(tol), ctypes.byref(s)),
              "psolve_autotune")
        return s.as_dict()

    def set_warm_start(self, enable=True):
        """Start later solves from the previous solve's Psi and Phi."""
        check(lib().psolve_set_warm_start(self.h, int(bool(enable))), "psolve_set_warm_start")

    def set_tail(self, max_planes=-1):
        """Cluster-resident tail: -1 as many planes as fit, 0 off, n at most n."""
        check(lib().psolve_set_tail(self.h, int(max_planes)), "psolve_set_tail")

    def tail(self):
        """(planes the tail kernel takes over, CTAs per cluster); (0, 0) when unused."""
        p, c = ctypes.c_int(), ctypes.c_int()
        check(lib().psolve_get_tail(self.h, ctypes.byref(p), ctypes.byref(c)), "psolve_get_tail")
        return p.value, c.value

    def close(self):
        if getattr(self, "h", None):
            lib().psolve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- solve ---------------------------------------------------------------
    def _need(self, t, shape, dtype):
        torch = self.torch
        if not (t.is_cuda and t.dtype == dtype and tuple(t.shape) == tuple(shape) and t.is_contiguous()):
            raise ValueError("expected a contiguous CUDA %s tensor of shape %s" % (dtype, shape))

    def solve(self, rho, phi=None, tol=1e-8, raise_on_error=True):
        torch = self.torch
        self._need(rho, self.shape, torch.float64)
        if phi is None:
            phi = torch.empty_like(rho)
        rc = lib().psolve_solve(self.h, _ptr(rho), _ptr(phi), float(tol))
        if raise_on_error:
            check(rc, "psolve_solve")
        return phi, rc

    def stats(self):
        M = self.n_modes
        cp = (ctypes.c_int * M)()
        cf = (ctypes.c_int * M)()
        stv = (ctypes.c_int * M)()
        s = Stats()
        s.cycles_psi = ctypes.cast(cp, ctypes.POINTER(ctypes.c_int))
        s.cycles_phi = ctypes.cast(cf, ctypes.POINTER(ctypes.c_int))
        s.status = ctypes.cast(stv, ctypes.POINTER(ctypes.c_int))
        check(lib().psolve_get_stats(self.h, ctypes.byref(s)), "psolve_get_stats")
        return dict(n_modes=s.n_modes, iterations_psi=s.iterations_psi,
                    iterations_phi=s.iterations_phi, rel_residual_psi=s.rel_residual_psi,
                    rel_residual_phi=s.rel_residual_phi, setup_ms=s.setup_ms,
                    cycles_psi=list(cp), cycles_phi=list(cf), status=list(stv))

    # -- stages ----------------------------------------------------------------
    def planes(self, level=0, dtype=None):
        """Empty complex planes [M, n_tz_l, n_r_l] of a multigrid level."""
        torch = self.torch
        n_r, n_tz = self.grid[0] >> level, self.grid[1] >> level
        dtype = dtype or torch.complex128
        return torch.zeros((self.n_modes, n_tz, n_r), dtype=dtype, device="cuda")

    def stage_forward(self, rho):
        f = self.planes()
        check(lib().psolve_stage_forward(self.h, _ptr(rho), _ptr(f)), "psolve_stage_forward")
        return f

    def stage_inverse(self, phi_hat):
        phi = self.torch.empty(self.grid, dtype=self.torch.float64, device="cuda")
        check(lib().psolve_stage_inverse(self.h, _ptr(phi_hat), _ptr(phi)), "psolve_stage_inverse")
        return phi

    def stage_forward_rows(self, rho_rows):
        """Transform a radial slab [rows][n_tz][n_phi] -> [M][n_tz][rows] complex."""
        torch = self.torch
        rows = rho_rows.shape[0]
        self._need(rho_rows, (rows, self.grid[1], self.grid[2]), torch.float64)
        f = torch.empty((self.n_modes, self.grid[1], rows), dtype=torch.complex128, device="cuda")
        check(lib().psolve_stage_forward_rows(self.h, _ptr(rho_rows), rows, _ptr(f)),
              "psolve_stage_forward_rows")
        return f

    def stage_inverse_rows(self, phi_hat_rows):
        torch = self.torch
        rows = phi_hat_rows.shape[2]
        self._need(phi_hat_rows, (self.n_modes, self.grid[1], rows), torch.complex128)
        phi = torch.empty((rows, self.grid[1], self.grid[2]), dtype=torch.float64, device="cuda")
        check(lib().psolve_stage_inverse_rows(self.h, _ptr(phi_hat_rows), rows, _ptr(phi)),
              "psolve_stage_inverse_rows")
        return phi

    def solve_modes(self, modes, f_hat, tol=1e-8, raise_on_error=True):
        """Steps 3-6 of Sec. 5.1 for the listed modes: f_hat [n][n_tz][n_r]
        complex (list order) -> (phi_hat of the same layout, return code)."""
        torch = self.torch
        n = len(modes)
        self._need(f_hat, (n, self.grid[1], self.grid[0]), torch.complex128)
        phi = torch.empty_like(f_hat)
        arr = (ctypes.c_int * max(n, 1))(*[int(m) for m in modes])
        rc = lib().psolve_solve_modes(self.h, arr, n, _ptr(f_hat), _ptr(phi), float(tol))
        if raise_on_error:
            check(rc, "psolve_solve_modes")
        return phi, rc

    def stage_mg_solve(self, f_hat, tol=1e-8, u0=None):
        u = self.planes() if u0 is None else u0.clone()
        cyc = (ctypes.c_int * self.n_modes)()
        rc = lib().psolve_stage_mg_solve(self.h, _ptr(f_hat), _ptr(u), float(tol),
                                         int(u0 is not None), cyc)
        return u, list(cyc), rc

    def stage_smooth(self, level, e, f, cycles=1):
        prec = 1 if self.desc.precision == MIXED else 0
        check(lib().psolve_stage_smooth(self.h, level, prec, _ptr(e), _ptr(f), cycles),
              "psolve_stage_smooth")
        return e

    def stage_smooth_static(self, level, e, f, cycles=1):
        """stage_smooth with its working memory in the library's static
        device array (no allocation; concurrent calls on one GPU race)."""
        prec = 1 if self.desc.precision == MIXED else 0
        check(lib().psolve_stage_smooth_static(self.h, level, prec, _ptr(e), _ptr(f), cycles),
              "psolve_stage_smooth_static")
        return e

    def fused_level(self):
        lv = ctypes.c_int()
        check(lib().psolve_get_fused_level(self.h, ctypes.byref(lv)), "psolve_get_fused_level")
        return lv.value

    def stage_vcycle(self, f):
        """Fused coarse V-cycle from the fused level (zero initial guess);
        returns the correction e."""
        level = self.fused_level()
        prec = 1 if self.desc.precision == MIXED else 0
        e = self.planes(level, f.dtype)
        check(lib().psolve_stage_vcycle(self.h, level, prec, _ptr(f), _ptr(e)), "psolve_stage_vcycle")
        return e

    def stage_restrict(self, level, e, f):
        prec = 1 if self.desc.precision == MIXED else 0
        c = self.planes(level + 1, e.dtype)
        check(lib().psolve_stage_restrict(self.h, level, prec, _ptr(e), _ptr(f), _ptr(c)),
              "psolve_stage_restrict")
        return c

    def setup_times(self):
        """(setup_ms, dgf_ms): psolve_create's wall time and its DGF part."""
        a, b = ctypes.c_double(), ctypes.c_double()
        check(lib().psolve_get_setup_times(self.h, ctypes.byref(a), ctypes.byref(b)),
              "psolve_get_setup_times")
        return a.value, b.value

    STAGES = ("fft_forward", "mg_psi", "boundary", "mg_phi", "fft_inverse")

    def stage_times(self):
        """Device ms per stage of the last solve (psolve_get_stage_times)."""
        ms = (ctypes.c_float * 5)()
        check(lib().psolve_get_stage_times(self.h, ms), "psolve_get_stage_times")
        return dict(zip(self.STAGES, list(ms)))

    def solve_host(self, rhos, phis=None, tol=1e-8, raise_on_error=True):
        """Solves from host memory with copies overlapped (psolve_solve_host).
        rhos: list of CPU float64 tensors (pinned for overlap), one per solve;
        phis: CPU float64 tensors for the results (allocated pinned when
        None; a list may repeat a tensor).  Returns (phis, statuses, rc)."""
        torch = self.torch
        n = len(rhos)
        if phis is None:
            phis = [torch.empty(self.shape, dtype=torch.float64).pin_memory() for _ in range(n)]
        if len(phis) != n:
            raise ValueError("one result buffer per density")
        want = 1
        for v in self.shape:
            want *= v
        for t in list(rhos) + list(phis):
            if (t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous()
                    or t.numel() != want):
                raise ValueError("host buffers must be contiguous CPU float64 tensors of %s" % (self.shape,))
        R = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in rhos])
        F = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in phis])
        st = (ctypes.c_int * max(n, 1))()
        rc = lib().psolve_solve_host(self.h, n, R, F, float(tol), st)
        if raise_on_error:
            check(rc, "psolve_solve_host")
        return phis, list(st)[:n], rc

    def stage_residual(self, f, u):
        """FP64 defect r = f - L_m u on the finest level of every mode, in the
        buffer precision (complex64 mixed, complex128 FP64)."""
        prec = 1 if self.desc.precision == MIXED else 0
        r = self.planes(0, self.torch.complex64 if prec else self.torch.complex128)
        check(lib().psolve_stage_residual(self.h, prec, _ptr(f), _ptr(u), _ptr(r)),
              "psolve_stage_residual")
        return r

    def stage_prolong(self, level, e, coarse):
        prec = 1 if self.desc.precision == MIXED else 0
        check(lib().psolve_stage_prolong(self.h, level, prec, _ptr(e), _ptr(coarse)),
              "psolve_stage_prolong")
        return e

    def stage_screening(self, psi_hat):
        s = self.torch.zeros((self.n_modes, self.n_boundary), dtype=self.torch.complex128,
                             device="cuda")
        check(lib().psolve_stage_screening(self.h, _ptr(psi_hat), _ptr(s)), "psolve_stage_screening")
        return s

    def stage_boundary(self, sigma):
        t = self.torch.zeros_like(sigma)
        check(lib().psolve_stage_boundary(self.h, _ptr(sigma), _ptr(t)), "psolve_stage_boundary")
        return t

    def dgf(self):
        g = self.torch.zeros((self.n_modes, self.n_boundary, self.n_boundary),
                             dtype=self.torch.float64, device="cuda")
        check(lib().psolve_get_dgf(self.h, _ptr(g)), "psolve_get_dgf")
        return g


class Batch:
    """Independent problems solved by one captured graph (psolve_batch_*):
    solvers[k] maps rhos[k] to phis[k] (device tensors kept alive here)."""

    def __init__(self, solvers, rhos, phis, tol=1e-8):
        import torch
        self.torch = torch
        n = len(solvers)
        for s, r, p in zip(solvers, rhos, phis):
            s._need(r, s.shape, torch.float64)
            s._need(p, s.shape, torch.float64)
        self.solvers, self.rhos, self.phis = list(solvers), list(rhos), list(phis)
        H = (ctypes.c_void_p * n)(*[s.h.value for s in solvers])
        R = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rhos])
        Q = (ctypes.c_void_p * n)(*[p.data_ptr() for p in phis])
        b = ctypes.c_void_p()
        check(lib().psolve_batch_create(ctypes.byref(b), H, R, Q, n, float(tol)), "psolve_batch_create")
        self.b = b
        self.n = n

    def run(self, raise_on_error=True):
        """Launch on torch's current stream and wait; returns (code, per-problem
        completion times in ms from the launch)."""
        lat = (ctypes.c_float * self.n)()
        rc = lib().psolve_batch_run(self.b, ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream), lat)
        if raise_on_error:
            check(rc, "psolve_batch_run")
        return rc, list(lat)

    def close(self):
        if getattr(self, "b", None):
            lib().psolve_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
