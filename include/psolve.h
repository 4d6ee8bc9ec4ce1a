/*
 * psolve -- spectral-multigrid Poisson solver for one GPU (C ABI).
 *
 * Computes the gravitational potential Phi of a density rho on a spherical
 * (r, theta, phi) or cylindrical (R, z, phi) grid with vacuum boundary
 * conditions, following Mandal, Gressel, Ziegler & Mignone, "A fast
 * spectral-multigrid Poisson solver in non-Cartesian geometries":
 *   Sec. 2.1   finite-volume Laplacian (Eq. poisson_discrete),
 *   Sec. 2.2   azimuthal Fourier decomposition into 2-D Helmholtz problems
 *              (Eqs. helmholz_sph, helmholz_cyl, eigenv_sph, eigenv_cyl),
 *   Sec. 3     multigrid with the alternating approximate line smoother,
 *   Sec. 4     James' screening-mass vacuum boundary conditions with
 *              discrete Green's functions,
 *   Sec. 5.1   the seven-step workflow (density in, potential out).
 *
 * Data layout of every 3-D field passed to the library: FP64, row-major
 * [n_r][n_tz][n_phi] (azimuth fastest), values at cell centres.
 * Mode planes (stage entry points): FP64 complex (re, im interleaved),
 * [M][n_tz][n_r] with M = n_phi/2 + 1 and the radial index fastest.
 *
 * Pointers are DEVICE pointers unless a name ends in _host.  All work is
 * enqueued on the handle's stream; functions that report a status read it
 * back with a synchronisation of that stream.  Handles are not thread-safe.
 * Errors are return codes (never an abort); psolve_last_error() gives the
 * message of the last failing call on the calling thread.
 */
#ifndef PSOLVE_H
#define PSOLVE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psolve_ctx* psolve_t;

enum { PSOLVE_SPHERICAL = 0, PSOLVE_CYLINDRICAL = 1 };
enum { PSOLVE_UNIFORM = 0, PSOLVE_LOG = 1 };
enum { PSOLVE_FP64 = 0, PSOLVE_MIXED = 1 };
enum {
  PSOLVE_OK = 0,
  PSOLVE_ERR_ARG = -1,           /* invalid argument or unsupported grid        */
  PSOLVE_ERR_CUDA = -2,          /* a CUDA call failed                          */
  PSOLVE_ERR_NOMEM = -3,         /* device allocation failed                    */
  PSOLVE_ERR_NOT_CONVERGED = -4, /* max_cycles reached or stagnation above tol  */
  PSOLVE_ERR_NONFINITE = -5      /* NaN / Inf in a residual norm                */
};

/* Allocation hooks: when set, every device workspace of a handle is obtained
 * from alloc(bytes, user) and returned with free(ptr, user); otherwise
 * cudaMalloc / cudaFree are used.  alloc returns NULL on failure, and
 * 256-byte aligned memory otherwise (as cudaMalloc does); a block that is not
 * so aligned is handed back to free and counts as a failed allocation. */
typedef void* (*psolve_alloc_fn)(size_t bytes, void* user);
typedef void (*psolve_free_fn)(void* ptr, void* user);

typedef struct {
  int geometry;        /* PSOLVE_SPHERICAL or PSOLVE_CYLINDRICAL                  */
  int n_r;             /* radial cells, power of two in [8, 1024] (FP64: <= 512)  */
  int n_tz;            /* theta (spherical) or z (cylindrical) cells, power of 2
                          in [8, 1024] (FP64: <= 512); n_r / n_tz in [1/16, 16]  */
  int n_phi;           /* azimuthal cells, power of two, 4 <= n_phi <= 1024       */
  int spacing;         /* radial spacing PSOLVE_UNIFORM or PSOLVE_LOG             */
  double r_in, r_out;  /* radial extent, 0 <= r_in < r_out (log: r_in > 0)        */
  double t_min, t_max; /* theta range (spherical, default 0, pi) or z range
                          (cylindrical, default -(r_out-r_in)/2 .. +...);
                          used only when t_max > t_min                            */
  double G;            /* gravitational constant; 0 selects 1                     */
  int precision;       /* PSOLVE_FP64 or PSOLVE_MIXED                             */
  int max_cycles;      /* V-cycle cap per mode and solve; 0 selects 100           */
  int nu_pre, nu_post; /* smoothing cycles before / after coarse correction; 0 -> 2 */
  int n_sor;           /* SOR sweeps per line relaxation; 0 -> 2                  */
  int use_graph;       /* 1: replay the solve as a captured CUDA graph            */
  psolve_alloc_fn alloc_fn; /* optional allocation hooks (see above)            */
  psolve_free_fn free_fn;
  void* alloc_user;
  int dgf_construction; /* Sec. 4.2: PSOLVE_DGF_AUTO (0: the extended domain for
                          logarithmic radial grids with r_out / r_in >= 100 and
                          n_r >= 32, auxiliary windows otherwise),
                          PSOLVE_DGF_AUX (1) or PSOLVE_DGF_EXTENDED (2, needs
                          logarithmic spacing and n_r >= 32).  The extended
                          domain doubles n_r (and a bounded theta or z range),
                          so it needs n_r <= 512 (and n_tz <= 512 when bounded):
                          PSOLVE_ERR_ARG otherwise                               */
  int coarsest_size;   /* size of the directly solved coarsest level (Sec. 3.3
                          leaves it open); levels halve both sides while the
                          short side exceeds S cells, or exceeds 4 cells with
                          more than C cells in the plane.
                          PSOLVE_COARSEST_SMALL (1): S = 16, C = 1024.
                          PSOLVE_COARSEST_LARGE (2): S = 32, C = 2048 when
                          that coarsest level is separable (its operator is
                          L_r (x) I + D_r (x) L_t), else the small rule.
                          PSOLVE_COARSEST_AUTO (0): the large rule for the
                          mixed path when it leaves at least two levels, the
                          small rule otherwise and for the FP64 path.  The
                          mixed path's FP32 V-cycle solves a separable
                          coarsest level in FP32 (factors computed in FP64
                          and rounded once: a coarse correction needs only a
                          nearby operator's solve), the FP64 path in FP64;
                          the cluster-resident tail needs the small rule.
                          Other values are PSOLVE_ERR_ARG                      */
} psolve_desc;

enum { PSOLVE_DGF_AUTO = 0, PSOLVE_DGF_AUX = 1, PSOLVE_DGF_EXTENDED = 2 };
enum { PSOLVE_COARSEST_AUTO = 0, PSOLVE_COARSEST_SMALL = 1, PSOLVE_COARSEST_LARGE = 2 };

/* Per-solve statistics (psolve_get_stats).  Arrays sized by the caller:
 * cycles_psi / cycles_phi / status hold M entries when non-NULL. */
typedef struct {
  int n_modes;              /* M = n_phi/2 + 1                                   */
  int iterations_psi;       /* outer iterations of the Psi solve (max over modes) */
  int iterations_phi;       /* same for the Phi solve                            */
  double rel_residual_psi;  /* sqrt(sum_m |r^m|^2 / sum_m |f^m|^2), volume-weighted
                               (sums of squares formed in FP32 with power-of-two
                               exponents: about 1e-6 relative, any data scale) */
  double rel_residual_phi;
  double setup_ms;          /* psolve_create wall time (incl. DGF tables)        */
  int* cycles_psi;          /* per-mode V-cycles, Psi solve (may be NULL)        */
  int* cycles_phi;          /* per-mode V-cycles, Phi solve (may be NULL)        */
  int* status;              /* per-mode PSOLVE_OK / NOT_CONVERGED / NONFINITE    */
} psolve_stats;

/* Plan a solver (Sec. 5.1 step 1): geometry and operator tables per
 * multigrid level, per-line relaxation parameters (App. A), coarsest-level
 * factors, discrete Green's function tables (Sec. 4.2) and workspaces.
 * Uses the current device and the legacy default stream until
 * psolve_set_stream.  Returns PSOLVE_OK and *out, or an error (*out NULL). */
int psolve_create(psolve_t* out, int geometry, int n_r, int n_theta_or_z, int n_phi,
                  int radial_spacing, double r_in, double r_out);
/* Same with every option; fields left zero take their defaults. */
int psolve_create_ex(psolve_t* out, const psolve_desc* d);

/* Same-geometry batch: a plan whose solves take n_densities (1..64)
 * densities of the geometry d at once.  psolve_solve's rho and phi then hold
 * n_densities fields back to back ([n_densities][n_r][n_tz][n_phi]).  The
 * modes of all densities iterate together (planes b M + m), so the slow low
 * modes of every density share the late iterations, and the boundary
 * convolution (Eqs. theta_left..theta_top) reads each mode's DGF table once
 * for up to eight densities: a [nb x nb] by [nb x 2 n_densities] product per
 * mode instead of n_densities products with one vector.  Workspaces grow
 * with n_densities; the DGF tables and level tables are shared.  The
 * statistics' per-mode arrays describe the first density; the relative
 * residuals and iteration counts cover all.  Stage entry points act on the
 * first density's planes.  Errors as psolve_create_ex, and PSOLVE_ERR_ARG
 * for n_densities outside 1..64. */
int psolve_create_multi(psolve_t* out, const psolve_desc* d, int n_densities);

/* The multigrid plan psolve_create_ex would build for d, computed on the
 * host only (no device memory, no kernels: usable without a GPU).  Levels
 * follow d->coarsest_size (Sec. 3; the paper leaves the coarsest size open);
 * the coarsest level is solved directly (Sec. 3.3 allows a direct solver)
 * in one of four forms, reported in `coarsest`. */
enum { PSOLVE_COARSE_SEPARABLE_MIRROR = 0, /* separable, mirror-symmetric polar operator */
       PSOLVE_COARSE_SEPARABLE = 1,        /* separable, general polar operator          */
       PSOLVE_COARSE_BLOCK = 2,            /* block-tridiagonal (Schur complements)      */
       PSOLVE_COARSE_DENSE = 3 };          /* dense inverse                              */
typedef struct {
  int n_modes;                 /* M = n_phi / 2 + 1                                 */
  int n_levels;                /* multigrid levels, finest first (at most 16)       */
  int level_n_r[16], level_n_tz[16];
  int coarsest;                /* PSOLVE_COARSE_*                                   */
  int coarse_doubles_per_mode; /* FP64 values of the coarsest-level factors per mode */
  double coarse_check;         /* separable forms: the largest relative residual, over
                                  the modes, of the factors applied to a fixed test
                                  vector (rounding level when sound); else -1     */
  int tail_cluster_ctas;       /* mixed path with the descriptor's n_sor: CTAs per
                                  cluster of the cluster-resident tail (see
                                  psolve_set_tail); 0 when the plan does not allow it */
  int tail_smem_bytes;         /* its shared memory per CTA (0 when not allowed)      */
} psolve_plan;
/* PSOLVE_ERR_ARG (with a message) for an invalid descriptor, as psolve_create_ex. */
int psolve_plan_inspect(const psolve_desc* d, psolve_plan* out);

/* Solve (Sec. 5.1 steps 2-7): rho [n_r][n_tz][n_phi] -> phi (same layout),
 * device pointers, phi must not alias rho.  tol is the relative residual of
 * each mode's Helmholtz problem in the volume-weighted L2 norm (App. B),
 * tol <= 0 selects 1e-8.  Returns PSOLVE_OK, PSOLVE_ERR_NOT_CONVERGED (phi
 * holds the last iterate) or another error. */
int psolve_solve(psolve_t h, const double* rho, double* phi, double tol);

/* n solves of this handle from host memory, with the copies overlapped
 * with the solves (Sec. 5.1 steps 2-7 for each): rho_host[k] ->
 * phi_host[k], host buffers of n_r n_tz n_phi doubles (times the number of
 * densities of a psolve_create_multi handle), layout as psolve_solve.  The
 * handle stages through device buffers of its own (two for rho, two for phi,
 * allocated at the first call through the handle's allocator and kept):
 * while solve k runs on the handle's stream, rho_host[k+1] is uploaded on a
 * second stream and phi of solve k-1 downloaded on a third.  Page-locked
 * host buffers (cudaHostAlloc, or registered) let the copies overlap;
 * pageable ones work but serialise.  phi_host[k] may repeat a pointer (the
 * downloads run in order); rho_host[k] may repeat too.  status (n ints, may
 * be NULL) receives each solve's PSOLVE_OK / NOT_CONVERGED / NONFINITE.
 * With warm start, each solve continues from the one before.  Returns when
 * every potential is on the host: PSOLVE_OK, the first failing solve's code,
 * PSOLVE_ERR_ARG (n < 0, a null buffer) or PSOLVE_ERR_NOMEM. */
int psolve_solve_host(psolve_t h, int n, const double* const* rho_host, double* const* phi_host,
                      double tol, int* status);
/* n independent solves (handles may differ in size and kind), enqueued on
 * each handle's own stream; the same return convention, first error wins. */
int psolve_solve_batched(psolve_t* hs, const double* const* rhos, double* const* phis, int n,
                         double tol);

/* Many independent problems in ONE captured CUDA graph (a serving-style
 * batch; the paper solves one problem at a time).  psolve_batch_create
 * captures, for n distinct handles (of any sizes and kinds) with their
 * device buffers rhos[k] -> phis[k] and tolerance tol, each problem's whole
 * solve (Sec. 5.1 steps 2-7) on its own branch of one graph, so independent
 * problems overlap on the GPU; a completion event follows each problem.
 * The graph keeps the buffers, the tolerance, the handles' schedules and
 * warm-start state as captured: create a new batch after changing any of
 * them.  While a batch exists its handles must not run other work at the
 * same time (the batch uses their workspaces).
 * psolve_batch_run launches the graph on `stream` (cudaStream_t as void*,
 * NULL: the legacy default stream), waits for it, and returns the first
 * non-OK status in handle order (as psolve_solve); latency_ms (n floats, may
 * be NULL) receives each problem's completion time from the launch, in ms.
 * psolve_batch_destroy waits for the device and frees the graph (NULL-safe);
 * the handles stay valid.  Errors: PSOLVE_ERR_ARG (null argument, n < 1, a
 * handle twice, phi aliasing rho), PSOLVE_ERR_CUDA (capture or launch). */
typedef struct psolve_batch_ctx* psolve_batch_t;
int psolve_batch_create(psolve_batch_t* out, psolve_t* hs, const double* const* rhos,
                        double* const* phis, int n, double tol);
int psolve_batch_run(psolve_batch_t b, void* stream, float* latency_ms);
void psolve_batch_destroy(psolve_batch_t b);

/* Wall time of psolve_create (ms, as psolve_stats.setup_ms) and the part of
 * it spent building the discrete Green's function tables (Sec. 4.2: far-field
 * closed forms and window or extended-domain solves).  PSOLVE_ERR_ARG for a
 * null argument. */
int psolve_get_setup_times(psolve_t h, double* setup_ms, double* dgf_ms);
/* Device time of the stages of the handle's last completed solve (Sec. 5.1;
 * the split of the paper's component-wise breakdown), ms: [0] forward
 * transform (step 2), [1] Psi multigrid (step 3, with the cluster-resident
 * tail), [2] screening mass, boundary convolution and ghost right-hand side
 * (steps 4-5), [3] Phi multigrid (step 6), [4] inverse transform (step 7).
 * Recorded by events on the handle's stream (event nodes in a captured
 * solve); for psolve_solve_host, its last solve.  Synchronises the stream.
 * PSOLVE_ERR_ARG for a null argument or before the first solve. */
int psolve_get_stage_times(psolve_t h, float* ms);

/* Warm start for time stepping (Sec. 5.1 and App. B: in a simulation the
 * previous step's solution is the initial guess, which cuts the V-cycles
 * needed).  When enabled, every later psolve_solve / psolve_solve_batched on
 * this handle starts the Psi solve from the previous solve's Psi and the Phi
 * solve from the previous Phi; the first solve after enabling starts from
 * zero (Psi) and Psi (Phi) as usual.  Enabling allocates two mode-plane
 * buffers (2 M n_tz n_r complex FP64) through the handle's allocator
 * (PSOLVE_ERR_NOMEM when that fails); enable = 0 returns to cold starts and
 * keeps the buffers.  A solve that fails with PSOLVE_ERR_NONFINITE or a CUDA
 * error clears the history. */
int psolve_set_warm_start(psolve_t h, int enable);
/* Bind the handle to a CUDA stream (cudaStream_t passed as void*; NULL: the
 * legacy default stream, the initial binding).  Every later call of the
 * handle enqueues its work there; a captured solve is captured again on the
 * next solve.  The caller keeps the stream alive while the handle uses it.
 * Returns PSOLVE_OK or PSOLVE_ERR_ARG (null handle). */
int psolve_set_stream(psolve_t h, void* cuda_stream);

/* Cluster-resident tail of each multigrid solve (App. B: the low modes, m = 0
 * above all, need many more V-cycles than the rest, so a solve ends with
 * iterations on one or a few mode planes).  Once at most P planes remain
 * active, one kernel launch finishes them: each plane gets a cluster of C
 * CTAs (one per SM) holding its whole multigrid hierarchy in distributed
 * shared memory, iterating FP64 residual -> FP32 V-cycle (Sec. 3) -> FP64
 * update on the device until the plane meets the App. B criterion.  The
 * results are those of the batched iteration up to rounding.  Used by the
 * mixed path when the plan allows (separable coarsest level, radial lines of
 * at most 256 cells, the cluster's shared memory holds the plane); P is the
 * number of clusters that fit on the GPU, at most 8.
 * psolve_set_tail: max_planes -1 (default) uses that P, 0 disables the tail
 * kernel, n > 0 caps P at n; a captured solve is captured again.
 * psolve_get_tail: *planes = P in use (0: not used), *cluster_ctas = C.
 * Both return PSOLVE_OK, or PSOLVE_ERR_ARG for a null handle or
 * max_planes < -1. */
int psolve_set_tail(psolve_t h, int max_planes);
int psolve_get_tail(psolve_t h, int* planes, int* cluster_ctas);

/* Smoothing schedule and tile shapes of a handle.  Sec. 3.2 leaves the
 * schedule open (a small number of smoothing cycles per level, typically two
 * or three, and a few SOR sweeps per line); it changes the convergence rate,
 * not the converged answer.  The tile shapes of the level-wide smoothing
 * passes change only how lines are grouped into thread blocks: every tile
 * shape gives bitwise the same result. */
typedef struct {
  int nu_pre, nu_post; /* smoothing cycles before / after coarse correction, 1..8 */
  int n_sor;           /* SOR sweeps per line relaxation, 1..8                    */
  int lines_r;         /* radial lines per block: 4 or 8                          */
  int cols_t;          /* polar columns per block: 8, 16 or 32; 0 = widest that
                          fits (32, or fewer where n_r or 160 KB of shared memory
                          per block is the limit)                                 */
  int nu_pre_fused, nu_post_fused; /* smoothing cycles on the levels of the fused
                          shared-memory V-cycle, 0..8; 0 = nu_pre / nu_post       */
  double ms;           /* psolve_autotune: median solve time of the choice, ms    */
  int candidates;      /* psolve_autotune: candidates timed (0: from a cache)      */
  int cached;          /* psolve_autotune: 1 when the choice came from a cache     */
  int tail_planes;     /* the cluster-resident tail (psolve_set_tail): -1 as many
                          planes as fit, 0 off, n > 0 at most n                   */
} psolve_schedule;

/* The handle's current schedule (ms, candidates, cached = 0; the fused-level
 * counts 0 when they equal nu_pre / nu_post; tail_planes as psolve_set_tail
 * last set it). */
int psolve_get_schedule(psolve_t h, psolve_schedule* s);
/* Install a schedule for later solves (a captured solve is captured again).
 * PSOLVE_ERR_ARG, with the handle unchanged, when a field is out of range. */
int psolve_set_schedule(psolve_t h, const psolve_schedule* s);

/* Autotuner: picks the smoothing schedule and tile shapes of this handle by
 * timing solves of rho (device pointer, layout as psolve_solve) to tolerance
 * tol on the handle's stream, and installs the fastest.
 *   Stage 1, schedules: nu_post <= nu_pre <= 3, n_sor <= 3 (18 schedules,
 *     after the handle's current one when that lies outside them).  Schedules with more post- than
 *     pre-smoothing are not tried: they leave a smoother final residual, whose
 *     error at the same tolerance is larger.
 *   Stage 2, tile shapes: lines_r in {4, 8} x cols_t in {8, 16, 32} with the
 *     stage-1 schedule (shapes that reduce to the same launch are timed once).
 *   Stage 3, when the fused shared-memory V-cycle smooths at least one
 *     level: that kernel's own smoothing counts, nu_post_fused <=
 *     nu_pre_fused <= 3, with the stage-1 and stage-2 choices (5 candidates
 *     besides the stage-1 counts).
 *   Stage 4, when the cluster-resident tail can run with the chosen
 *     schedule: the tail off against on (psolve_set_tail).
 * Each candidate runs one untimed solve (graph capture, caches), then three
 * timed solves (CUDA events on the handle's stream); its time is their
 * median.  Candidates whose solve fails are skipped.  Warm start is
 * suspended while tuning (the history is kept).  phi (device, caller-owned)
 * receives the last solve's potential.
 * Choices are cached per process by the key (geometry, sizes, spacing,
 * extents, precision): a later call with the same key installs the cached
 * choice without timing.  When the environment variable PSOLVE_TUNE_CACHE
 * names a file, it is read on a process-cache miss and every new choice is
 * appended to it (text, one line per key: key nu_pre nu_post n_sor lines_r
 * cols_t nu_pre_fused nu_post_fused ms tail_planes; the last line of a key wins).
 * out (may be NULL) receives the choice.  Returns PSOLVE_OK, or the error of
 * the solve with the handle's current schedule, which then stays installed. */
int psolve_autotune(psolve_t h, const double* rho, double* phi, double tol,
                    psolve_schedule* out);
/* Statistics of the handle's last solve (App. B: per-mode cycle counts and
 * convergence status; the relative residuals of the Psi and Phi solves over
 * all modes).  Synchronises the handle's stream first.  st is caller-owned;
 * its array members, when non-NULL, receive M entries each.  Returns
 * PSOLVE_OK, PSOLVE_ERR_ARG (null argument) or PSOLVE_ERR_CUDA. */
int psolve_get_stats(psolve_t h, psolve_stats* st);
/* Number of boundary points nb (the side of the DGF table), modes M and
 * multigrid levels of the handle; each output pointer may be NULL.  Host
 * only.  Returns PSOLVE_OK or PSOLVE_ERR_ARG (null handle). */
int psolve_get_sizes(psolve_t h, int* n_modes, int* n_boundary, int* n_levels);
/* Message of the last failing call on the calling thread (a thread-local
 * string owned by the library, valid until that thread's next failing
 * call); "" when no call has failed. */
const char* psolve_last_error(void);
/* Frees the handle and every device buffer it owns, after synchronising its
 * stream.  The caller's stream (psolve_set_stream) and buffers are not
 * touched.  NULL is ignored. */
void psolve_destroy(psolve_t h);

/* ---- stage entry points (each runs one step of the solve on all modes) ---- */

/* Sec. 2.2: rho_hat[m][j][i] = (4 pi G / n_phi) sum_k rho[i][j][k] e^{-2 pi i m k / n_phi},
 * i.e. the right-hand side 4 pi G rho^m of the mode equations. */
int psolve_stage_forward(psolve_t h, const double* rho, double* f_hat);
/* The same transforms on a radial slab of n_rows consecutive radial rows
 * (1 <= n_rows <= n_r; the transform along phi does not depend on the
 * radius): rho_rows [n_rows][n_tz][n_phi] -> f_hat_rows [M][n_tz][n_rows]
 * complex, and back (phi_hat_rows [M][n_tz][n_rows] -> phi_rows
 * [n_rows][n_tz][n_phi]).  The building blocks of a mode-sharded solve over
 * several GPUs: each rank transforms its slab, an all-to-all exchange moves
 * every mode's planes to the rank that owns the mode (psolve_solve_modes),
 * and the reverse exchange returns the potential's modes for the inverse
 * transform of each slab. */
int psolve_stage_forward_rows(psolve_t h, const double* rho_rows, int n_rows, double* f_hat_rows);
int psolve_stage_inverse_rows(psolve_t h, const double* phi_hat_rows, int n_rows, double* phi_rows);
/* Sec. 5.1 steps 3-6 (both Helmholtz solves, the screening mass and the
 * boundary convolution) for the n azimuthal modes listed in modes_host
 * (host array of distinct mode numbers 0 <= m < M, any order):
 * f_hat [n][n_tz][n_r] complex FP64 holds 4 pi G rho^m of those modes in
 * list order (device), phi_hat (device, same layout) receives Phi^m.  The
 * modes solve independently of each other (Sec. 2.2), so the result of a
 * mode equals that of a whole-problem solve.  Runs eagerly on the handle's
 * stream without warm start; the statistics describe this call (unlisted
 * modes: zero cycles).  Returns as psolve_solve, PSOLVE_ERR_ARG for a bad
 * list. */
int psolve_solve_modes(psolve_t h, const int* modes_host, int n, const double* f_hat,
                       double* phi_hat, double tol);
/* Sec. 2.2, Eq. Hermitian_symmetry: phi[i][j][k] = Re sum over all n_phi modes
 * with the upper half rebuilt as conjugates; imaginary parts of m = 0 and
 * m = n_phi/2 ignored. */
int psolve_stage_inverse(psolve_t h, const double* phi_hat, double* phi);
/* Sec. 3: solve L_m u = f for every mode with zero ghost values, by the
 * handle's precision mode; f_hat, u_hat as mode planes; u_hat is the initial
 * guess on entry when warm != 0.  cycles_host (M ints, may be NULL) receives
 * the V-cycles per mode. */
int psolve_stage_mg_solve(psolve_t h, const double* f_hat, double* u_hat, double tol, int warm,
                          int* cycles_host);
/* Sec. 3.2 / 3.1 single steps at multigrid level `level` (0 = finest), in
 * FP64 (precision 0) or FP32 (1) planes [M][n_tz_l][n_r_l] complex:
 *   smooth:   `cycles` alternating line-smoothing cycles on e with rhs f;
 *   restrict: coarse = R (f - L e), the area-weighted restriction of the defect;
 *   prolong:  e += P coarse, bilinear prolongation from level+1. */
int psolve_stage_smooth(psolve_t h, int level, int precision, void* e, const void* f, int cycles);
int psolve_stage_restrict(psolve_t h, int level, int precision, const void* e, const void* f,
                          void* coarse);
int psolve_stage_prolong(psolve_t h, int level, int precision, void* e, const void* coarse);
/* Sec. 3 (the refinement's defect, Sec. 3.3): r = f - L_m u on the finest
 * level for every mode, evaluated in FP64 from FP64 u and f and stored in the
 * handle's buffer precision (precision 1: FP32 planes, as the mixed V-cycle
 * consumes it; 0: FP64), with the zero ghost values of the Psi problem.  This
 * is the solve's own residual kernel, with its volume-weighted norms and a
 * convergence test at tolerance 0, so that no mode retires.
 * f, u: device double2 planes [M][n_tz][n_r] (interleaved Re/Im FP64);
 * r: device planes [M][n_tz][n_r] of the buffer precision, overwritten.
 * Caller-owned.  The launches are enqueued on the handle's stream
 * (psolve_set_stream) and the call returns without waiting for them, so
 * that calls can be timed back to back; a launch error is returned at once.
 * PSOLVE_ERR_ARG for a null pointer or a precision other than the
 * handle's. */
int psolve_stage_residual(psolve_t h, int precision, const double* f, const double* u, void* r);
/* Sec. 3: the coarse part of one V-cycle, fused into one kernel: from
 * level `level` (which must be the handle's fused level, see
 * psolve_get_fused_level) down to the coarsest, on L_m e = f with a zero
 * initial guess: nu_pre smoothing cycles, defect restriction, recursion,
 * the direct coarsest solve (see psolve_desc.coarsest_size), prolongation,
 * nu_post smoothing cycles.
 * f, e: planes [M][n_tz_l][n_r_l] complex in FP64 (precision 0) or FP32 (1);
 * e is overwritten.  PSOLVE_ERR_ARG for another level or precision. */
int psolve_stage_vcycle(psolve_t h, int level, int precision, const void* f, void* e);
/* The first multigrid level held in shared memory by the fused V-cycle. */
int psolve_get_fused_level(psolve_t h, int* level);
/* Eqs. charge_sph / charge_cyl: sigma[m][b] (complex) from psi_hat. */
int psolve_stage_screening(psolve_t h, const double* psi_hat, double* sigma);
/* Eqs. theta_left..theta_top: theta[m][t] = sum_s Gt[m][t][s] sigma[m][s]. */
int psolve_stage_boundary(psolve_t h, const double* sigma, double* theta);
/* Copy the DGF table Gt[m][t][s] (FP64, M * nb * nb) to device memory dst. */
int psolve_get_dgf(psolve_t h, double* dst);

/* ---- allocation-free variant (the paper has no counterpart) ---- */

/* Size in bytes of the library's static device scratch array.  Every GPU on
 * which the library's kernels are loaded holds this much device memory until
 * the process exits. */
#define PSOLVE_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* psolve_stage_smooth computed with no device allocation and without the
 * handle's workspaces: for callers that must not allocate device memory at
 * the point of the call -- a host code that has given all remaining device
 * memory to its own pool after creating the handle, or one that cannot afford
 * the device-wide synchronisation cudaMalloc / cudaFree may imply.  Same
 * arguments, layout and result as psolve_stage_smooth (e in/out, f in, both
 * device pointers owned by the caller).  The step's working memory (an
 * active-plane list and one ping-pong copy of the level's planes, 256-byte
 * aligned) is taken from the static array; the handle supplies only its
 * read-only tables and writes none of its workspaces.  The call runs in
 * order on the handle's stream and returns once that stream is idle, so it
 * waits behind any work already enqueued there; it must not be called while
 * that stream is being captured.
 *   Size limit: round_up_256(4 (M + 1)) + M n_tz_l n_r_l (16 for precision 0,
 *   8 for precision 1) bytes must not exceed PSOLVE_STATIC_SCRATCH_BYTES;
 *   larger levels return PSOLVE_ERR_ARG with a message naming the need.
 *   Device: the device current at the handle's creation must be current
 *   (PSOLVE_ERR_ARG otherwise).  The first call on a device looks up the
 *   array's device address with that device current and keeps it for the
 *   life of the process (the address assumes the device's primary context
 *   lives until exit: no cudaDeviceReset in between); make this first call
 *   before any stream capture begins.
 *   Sharing: all calls on a device use the same array, which keeps the last
 *   call's contents; each call rewrites what it reads.  Calls whose work
 *   overlaps on one GPU (other streams, threads or handles) race.
 * Returns PSOLVE_OK, PSOLVE_ERR_ARG or PSOLVE_ERR_CUDA. */
int psolve_stage_smooth_static(psolve_t h, int level, int precision, void* e, const void* f,
                               int cycles);

#ifdef __cplusplus
}
#endif
#endif
