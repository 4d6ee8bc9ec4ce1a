// C ABI of the solver (include/psolve.h): plan creation, the seven-step
// solve (Sec. 5.1) as eager launches or one captured CUDA graph with a
// WHILE node per multigrid solve, stage entry points and statistics.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/psolve.h"
#include "dgf.h"
#include "solver.h"

using namespace ps;

static thread_local std::string g_err;
static const double kPi = 3.14159265358979323846;

struct SolveStats {
  int* cycles = nullptr;
  int* status = nullptr;
  double2* nf2 = nullptr;
  double2* nr2 = nullptr;
  int* iter = nullptr;
};

struct psolve_ctx {
  Arena A;
  psolve_desc d{};
  PlaneGeo g;
  Law rlaw, tlaw;
  int M = 0, nb = 0, construction = -1;
  int nd = 1;   // densities per solve (same geometry): planes p = b M + m
  int P = 0;    // nd M mode planes
  MGSolver mg;
  std::vector<BPoint> bp;
  BDev bdev{};
  double* gt = nullptr;
  double2* tw = nullptr;
  double2 *u = nullptr, *f = nullptr, *sigma = nullptr, *theta = nullptr;
  // warm start: the previous solve's Psi and Phi mode planes as initial guesses
  double2 *psi_prev = nullptr, *phi_prev = nullptr;
  int warm = 0, warm_hist = 0;
  SolveStats sp, sf;
  int* d_worst = nullptr;
  int* h_worst = nullptr;
  cudaStream_t st = 0;
  int device = 0;     // the device current at create: the handle's memory lives there
  double setup_ms = 0;
  double dgf_ms = 0;   // of which the DGF tables (Sec. 4.2)
  // captured solve
  cudaGraphExec_t gexec = nullptr;
  const double* g_rho = nullptr;
  double* g_phi = nullptr;
  double g_tol = -1;
  int g_warm = -1;   // warm state the graph was captured with
  // host-buffer pipeline (psolve_solve_host): device staging buffers, the
  // upload and download streams and their events, per-solve status
  struct Pipe {
    double *rho_dev = nullptr, *rho_b = nullptr, *phi_dev = nullptr, *phi_b = nullptr;
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t in_ready = nullptr, rho_free = nullptr, out_ready = nullptr, phi_free = nullptr;
    int* h_status = nullptr;   // pinned, one int per solve of a call
    int cap = 0;
  };
  Pipe* pipe = nullptr;
  // stage marks of the last solve: start, after the forward transform, after
  // the Psi multigrid, after the boundary steps, after the Phi multigrid, end
  cudaEvent_t mark[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

static size_t plane_bytes(psolve_t h) { return sizeof(double2) * size_t(h->P) * h->d.n_r * h->d.n_tz; }
static int warm_state(psolve_t h) { return h->warm ? (h->warm_hist ? 2 : 1) : 0; }

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

static bool cuda_ok(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
  }
  return true;
}

static bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// worst status over both solves -> d_worst
__global__ void k_worst(const int* a, const int* b, int n, int* out) {
  int w = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int s1 = a[k], s2 = b[k];
    if (s1 == -5 || s2 == -5) w = min(w, -5);
    else if (s1 == -4 || s2 == -4 || s1 == 2 || s2 == 2 || s1 == 1 || s2 == 1) w = min(w, -4);
  }
  for (int o = 16; o > 0; o >>= 1) w = min(w, __shfl_down_sync(0xffffffffu, w, o));
  __shared__ int sw[32];
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) r = min(r, sw[i]);
    *out = r;
  }
}

static void snapshot(psolve_ctx* h, SolveStats& s) {
  const int M = h->P;
  cudaMemcpyAsync(s.cycles, h->mg.d_cycles, sizeof(int) * M, cudaMemcpyDeviceToDevice, h->st);
  cudaMemcpyAsync(s.status, h->mg.d_status, sizeof(int) * M, cudaMemcpyDeviceToDevice, h->st);
  cudaMemcpyAsync(s.nf2, h->mg.d_nf2, sizeof(double2) * M, cudaMemcpyDeviceToDevice, h->st);
  cudaMemcpyAsync(s.nr2, h->mg.d_nr2, sizeof(double2) * M, cudaMemcpyDeviceToDevice, h->st);
  cudaMemcpyAsync(s.iter, h->mg.d_iter, sizeof(int), cudaMemcpyDeviceToDevice, h->st);
}

// Checks a descriptor and fills its defaults (PSOLVE_OK or PSOLVE_ERR_ARG).
static int prepare_desc(const psolve_desc& din, psolve_desc& d) {
  d = din;
  if (d.geometry != PSOLVE_SPHERICAL && d.geometry != PSOLVE_CYLINDRICAL)
    return fail(PSOLVE_ERR_ARG, "geometry must be PSOLVE_SPHERICAL or PSOLVE_CYLINDRICAL");
  if (!pow2(d.n_r) || !pow2(d.n_tz) || d.n_r < 8 || d.n_tz < 8 || d.n_r > 1024 || d.n_tz > 1024)
    return fail(PSOLVE_ERR_ARG, "n_r and n_tz must be powers of two in [8, 1024]");
  if (d.n_r / d.n_tz > 16 || d.n_tz / d.n_r > 16)
    return fail(PSOLVE_ERR_ARG, "n_r / n_tz must lie within [1/16, 16]");
  if (!pow2(d.n_phi) || d.n_phi < 4 || d.n_phi > 1024)
    return fail(PSOLVE_ERR_ARG, "n_phi must be a power of two in [4, 1024]");
  if (d.spacing != PSOLVE_UNIFORM && d.spacing != PSOLVE_LOG)
    return fail(PSOLVE_ERR_ARG, "radial spacing must be PSOLVE_UNIFORM or PSOLVE_LOG");
  if (!(d.r_in >= 0.0) || !(d.r_out > d.r_in) || (d.spacing == PSOLVE_LOG && !(d.r_in > 0.0)))
    return fail(PSOLVE_ERR_ARG, "need 0 <= r_in < r_out (r_in > 0 for logarithmic spacing)");
  if (!(d.t_max > d.t_min)) {
    if (d.geometry == PSOLVE_SPHERICAL) { d.t_min = 0.0; d.t_max = kPi; }
    else { d.t_min = -0.5 * (d.r_out - d.r_in); d.t_max = 0.5 * (d.r_out - d.r_in); }
  }
  if (d.geometry == PSOLVE_SPHERICAL && (d.t_min < -1e-12 || d.t_max > kPi + 1e-12))
    return fail(PSOLVE_ERR_ARG, "theta range must lie within [0, pi]");
  if (d.G == 0.0) d.G = 1.0;
  if (d.max_cycles <= 0) d.max_cycles = 100;
  if (d.nu_pre <= 0) d.nu_pre = 2;
  if (d.nu_post < 0) d.nu_post = 2;
  if (d.nu_post == 0) d.nu_post = 2;
  if (d.n_sor <= 0) d.n_sor = 2;
  if (d.precision != PSOLVE_FP64 && d.precision != PSOLVE_MIXED)
    return fail(PSOLVE_ERR_ARG, "precision must be PSOLVE_FP64 or PSOLVE_MIXED");
  if (d.dgf_construction < PSOLVE_DGF_AUTO || d.dgf_construction > PSOLVE_DGF_EXTENDED)
    return fail(PSOLVE_ERR_ARG, "dgf_construction must be PSOLVE_DGF_AUTO, _AUX or _EXTENDED");
  if (d.coarsest_size < PSOLVE_COARSEST_AUTO || d.coarsest_size > PSOLVE_COARSEST_LARGE)
    return fail(PSOLVE_ERR_ARG, "coarsest_size must be PSOLVE_COARSEST_AUTO, _SMALL or _LARGE");
  if (d.dgf_construction == PSOLVE_DGF_EXTENDED && (d.spacing != PSOLVE_LOG || d.n_r < 32))
    return fail(PSOLVE_ERR_ARG, "the extended-domain DGF needs logarithmic radial spacing and n_r >= 32");
  if (d.precision == PSOLVE_FP64 && (d.n_r > 512 || d.n_tz > 512))
    return fail(PSOLVE_ERR_ARG, "the FP64 path holds lines of at most 512 cells (n_r, n_tz <= 512); "
                                "use PSOLVE_MIXED for longer lines");
  {
    // the extended domain doubles n_r (and a bounded theta or z direction):
    // its multigrid lines must stay within 1024 cells
    const bool ext = d.dgf_construction == PSOLVE_DGF_EXTENDED ||
                     (d.dgf_construction == PSOLVE_DGF_AUTO && d.spacing == PSOLVE_LOG &&
                      d.r_out / d.r_in >= 100.0 && d.n_r >= 32);
    const bool bounded_t = d.geometry == PSOLVE_CYLINDRICAL || d.t_min > 1e-12 || d.t_max < kPi - 1e-12;
    if (ext && (d.n_r > 512 || (bounded_t && d.n_tz > 512)))
      return fail(PSOLVE_ERR_ARG, "the extended-domain DGF (logarithmic grids with r_out / r_in >= 100) "
                                  "needs n_r <= 512 (and n_tz <= 512 for a bounded theta or z range); "
                                  "dgf_construction = PSOLVE_DGF_AUX uses auxiliary windows instead");
  }
  return PSOLVE_OK;
}

// The finest plane's geometry of a prepared descriptor (host arithmetic only).
static void make_geo(const psolve_desc& d, PlaneGeo& g, Law& rlaw, Law& tlaw) {
  const int geo = d.geometry == PSOLVE_SPHERICAL ? SPH : CYL;
  rlaw = Law{d.r_in, d.r_out, d.n_r, d.spacing == PSOLVE_LOG ? LOGS : UNI};
  tlaw = Law{d.t_min, d.t_max, d.n_tz, UNI};
  g.geometry = geo;
  g.n_phi = d.n_phi;
  g.G = d.G;
  g.r = axis_from_law(geo == SPH ? 0 : 1, rlaw, 1, d.n_r);
  g.t = axis_from_law(geo == SPH ? 2 : 3, tlaw, 1, d.n_tz);
  g.build();
}

static int create_impl(psolve_t* out, const psolve_desc* din, int nd) {
  auto t0 = std::chrono::steady_clock::now();
  if (!out || !din) return fail(PSOLVE_ERR_ARG, "null argument");
  *out = nullptr;
  psolve_desc d;
  if (const int rc = prepare_desc(*din, d)) return rc;

  std::unique_ptr<psolve_ctx> h(new psolve_ctx());
  h->d = d;
  cudaGetDevice(&h->device);
  h->A.alloc_fn = d.alloc_fn;
  h->A.free_fn = d.free_fn;
  h->A.user = d.alloc_user;
  make_geo(d, h->g, h->rlaw, h->tlaw);
  h->M = d.n_phi / 2 + 1;
  const int M = h->M;
  h->nd = nd;
  h->P = nd * M;
  const int P = h->P;
  const size_t plane = size_t(d.n_r) * d.n_tz;
  std::string err;
  std::vector<int> modes(M);
  for (int m = 0; m < M; ++m) modes[m] = m;
  MGOptions o;
  o.precision = d.precision;
  o.nu1 = d.nu_pre;
  o.nu2 = d.nu_post;
  o.n_sor = d.n_sor;
  o.max_cycles = d.max_cycles;
  o.coarsest_size = d.coarsest_size;
  std::vector<int> plane_slot;   // several densities: plane b M + m solves mode m
  if (nd > 1) {
    plane_slot.resize(P);
    for (int q = 0; q < P; ++q) plane_slot[q] = q % M;
  }
  if (!h->mg.init(h->A, h->g, false, modes, plane_slot, P, o, err)) {
    h->A.release_all();
    return fail(PSOLVE_ERR_NOMEM, "multigrid setup: " + err);
  }
  h->u = static_cast<double2*>(h->A.get(sizeof(double2) * plane * P));
  h->f = static_cast<double2*>(h->A.get(sizeof(double2) * plane * P));
  // twiddles e^{-2 pi i k / N}
  std::vector<double2> tw(d.n_phi / 2);
  for (int k = 0; k < d.n_phi / 2; ++k)
    tw[k] = make_double2(std::cos(2.0 * kPi * k / d.n_phi), -std::sin(2.0 * kPi * k / d.n_phi));
  h->tw = static_cast<double2*>(h->A.get(sizeof(double2) * tw.size()));
  // boundary points, screening and coupling coefficients
  h->bp = boundary_points(h->g);
  h->nb = int(h->bp.size());
  const int nb = h->nb;
  std::vector<int> adj(nb);
  std::vector<double> sig(nb), cpl(nb);
  std::vector<int> cells, cbp;
  std::vector<int> slot_of_cell(plane, -1);
  for (int b = 0; b < nb; ++b) {
    adj[b] = (h->bp[b].aj - 1) * d.n_r + (h->bp[b].ai - 1);
    sig[b] = h->bp[b].sigma_coef;
    cpl[b] = h->bp[b].couple;
    int& sc = slot_of_cell[adj[b]];
    if (sc < 0) {
      sc = int(cells.size());
      cells.push_back(adj[b]);
      cbp.push_back(b);
      cbp.push_back(-1);
    } else {
      cbp[2 * sc + 1] = b;
    }
  }
  auto up_i = [&](const std::vector<int>& v) {
    int* p = static_cast<int*>(h->A.get(sizeof(int) * std::max<size_t>(1, v.size())));
    if (p) cudaMemcpy(p, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice);
    return p;
  };
  auto up_d = [&](const std::vector<double>& v) {
    double* p = static_cast<double*>(h->A.get(sizeof(double) * std::max<size_t>(1, v.size())));
    if (p) cudaMemcpy(p, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice);
    return p;
  };
  h->bdev.nb = nb;
  h->bdev.ncell = int(cells.size());
  h->bdev.adj = up_i(adj);
  h->bdev.sig = up_d(sig);
  h->bdev.cpl = up_d(cpl);
  h->bdev.cell = up_i(cells);
  h->bdev.cbp = up_i(cbp);
  h->bdev.plane_cells = int(plane);
  h->sigma = static_cast<double2*>(h->A.get(sizeof(double2) * size_t(P) * std::max(nb, 1)));
  h->theta = static_cast<double2*>(h->A.get(sizeof(double2) * size_t(P) * std::max(nb, 1)));
  h->gt = static_cast<double*>(h->A.get(sizeof(double) * size_t(M) * nb * nb));
  for (SolveStats* s : {&h->sp, &h->sf}) {
    s->cycles = static_cast<int*>(h->A.get(sizeof(int) * P));
    s->status = static_cast<int*>(h->A.get(sizeof(int) * P));
    s->nf2 = static_cast<double2*>(h->A.get(sizeof(double2) * P));
    s->nr2 = static_cast<double2*>(h->A.get(sizeof(double2) * P));
    s->iter = static_cast<int*>(h->A.get(sizeof(int)));
  }
  h->d_worst = static_cast<int*>(h->A.get(sizeof(int)));
  if (!h->u || !h->f || !h->tw || !h->gt || !h->theta || !h->d_worst || !h->sf.iter) {
    h->A.release_all();
    return fail(PSOLVE_ERR_NOMEM, "out of device memory");
  }
  cudaMemcpy(h->tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice);
  cudaMallocHost(&h->h_worst, sizeof(int));
  for (cudaEvent_t& e : h->mark)
    if (cudaEventCreate(&e) != cudaSuccess) e = nullptr;
  // discrete Green's function tables (Sec. 5.1 step 1), scratch released after
  {
    const auto td = std::chrono::steady_clock::now();
    Arena scratch;
    scratch.alloc_fn = d.alloc_fn;
    scratch.free_fn = d.free_fn;
    scratch.user = d.alloc_user;
    h->construction = d.dgf_construction;   // the request in, the construction used out
    bool ok = build_dgf(h->g, h->rlaw, h->tlaw, h->bp, h->gt, scratch, h->st, h->construction, err);
    cudaDeviceSynchronize();
    scratch.release_all();
    h->dgf_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - td).count();
    if (!ok) {
      h->A.release_all();
      return fail(err.find("memory") != std::string::npos ? PSOLVE_ERR_NOMEM : PSOLVE_ERR_ARG,
                  "DGF: " + err);
    }
  }
  if (!cuda_ok("create")) {
    h->A.release_all();
    return PSOLVE_ERR_CUDA;
  }
  h->setup_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = h.release();
  return PSOLVE_OK;
}

extern "C" int psolve_plan_inspect(const psolve_desc* din, psolve_plan* out) {
  if (!din || !out) return fail(PSOLVE_ERR_ARG, "null argument");
  psolve_desc d;
  if (const int rc = prepare_desc(*din, d)) return rc;
  try {
    PlaneGeo g;
    Law rl, tl;
    make_geo(d, g, rl, tl);
    const int M = d.n_phi / 2 + 1;
    std::vector<int> modes(M);
    for (int m = 0; m < M; ++m) modes[m] = m;
    Hierarchy H;
    std::string err;
    if (!plan_hierarchy(g, false, modes, d.coarsest_size, d.precision, H, err))
      return fail(PSOLVE_ERR_ARG, "multigrid plan: " + err);
    *out = psolve_plan{};
    out->n_modes = M;
    out->n_levels = int(H.lv.size());
    for (int l = 0; l < out->n_levels && l < 16; ++l) {
      out->level_n_r[l] = H.lv[l].g.r.n;
      out->level_n_tz[l] = H.lv[l].g.t.n;
    }
    if (H.sep_stride > 0) {
      out->coarsest = H.sep_sym ? PSOLVE_COARSE_SEPARABLE_MIRROR : PSOLVE_COARSE_SEPARABLE;
      out->coarse_doubles_per_mode = H.sep_stride;
      out->coarse_check = H.sep_check;
    } else if (H.blk_n > 0) {
      out->coarsest = PSOLVE_COARSE_BLOCK;
      out->coarse_doubles_per_mode = H.blk_nt * H.blk_n * (H.blk_n + 2);
      out->coarse_check = -1.0;
    } else {
      out->coarsest = PSOLVE_COARSE_DENSE;
      out->coarse_doubles_per_mode = H.nc * H.nc;
      out->coarse_check = -1.0;
    }
    if (d.precision == PSOLVE_MIXED) {
      std::vector<int> nr(out->n_levels), nt(out->n_levels);
      for (int l = 0; l < out->n_levels; ++l) { nr[l] = H.lv[l].g.r.n; nt[l] = H.lv[l].g.t.n; }
      TailArgs t{};
      const size_t bytes = tail_layout(nr, nt, d.n_sor, H.sep_stride > 0 && !H.large, t);
      out->tail_cluster_ctas = bytes ? t.C : 0;
      out->tail_smem_bytes = int(bytes);
    }
    return PSOLVE_OK;
  } catch (const std::exception& e) {
    return fail(PSOLVE_ERR_NOMEM, std::string("plan: ") + e.what());
  }
}

extern "C" int psolve_create_ex(psolve_t* out, const psolve_desc* d) {
  try {
    return create_impl(out, d, 1);
  } catch (const std::exception& e) {
    return fail(PSOLVE_ERR_NOMEM, std::string("create: ") + e.what());
  }
}

extern "C" int psolve_create_multi(psolve_t* out, const psolve_desc* d, int n_densities) {
  if (n_densities < 1 || n_densities > 64)
    return fail(PSOLVE_ERR_ARG, "n_densities must lie in 1..64");
  try {
    return create_impl(out, d, n_densities);
  } catch (const std::exception& e) {
    return fail(PSOLVE_ERR_NOMEM, std::string("create: ") + e.what());
  }
}

extern "C" int psolve_create(psolve_t* out, int geometry, int n_r, int n_tz, int n_phi,
                             int spacing, double r_in, double r_out) {
  psolve_desc d{};
  d.geometry = geometry; d.n_r = n_r; d.n_tz = n_tz; d.n_phi = n_phi; d.spacing = spacing;
  d.r_in = r_in; d.r_out = r_out; d.precision = PSOLVE_MIXED; d.use_graph = 1;
  return psolve_create_ex(out, &d);
}

static void pipe_release(psolve_t h) {
  psolve_ctx::Pipe* p = h->pipe;
  if (!p) return;
  if (p->up) cudaStreamSynchronize(p->up);
  if (p->down) cudaStreamSynchronize(p->down);
  for (cudaEvent_t e : {p->in_ready, p->rho_free, p->out_ready, p->phi_free})
    if (e) cudaEventDestroy(e);
  if (p->up) cudaStreamDestroy(p->up);
  if (p->down) cudaStreamDestroy(p->down);
  if (p->h_status) cudaFreeHost(p->h_status);
  delete p;   // the device buffers belong to the handle's arena
  h->pipe = nullptr;
}

extern "C" void psolve_destroy(psolve_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  pipe_release(h);
  for (cudaEvent_t e : h->mark)
    if (e) cudaEventDestroy(e);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->mg.h_cont) cudaFreeHost(h->mg.h_cont);
  if (h->h_worst) cudaFreeHost(h->h_worst);
  h->A.release_all();
  delete h;
}

extern "C" int psolve_get_stage_times(psolve_t h, float* ms) {
  if (!h || !ms) return fail(PSOLVE_ERR_ARG, "null argument");
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(PSOLVE_ERR_CUDA, "stage times");
  for (int k = 0; k < 5; ++k) {
    ms[k] = 0.f;
    if (!h->mark[k] || !h->mark[k + 1] || cudaEventElapsedTime(&ms[k], h->mark[k], h->mark[k + 1]) != cudaSuccess) {
      cudaGetLastError();
      return fail(PSOLVE_ERR_ARG, "no completed solve to report");
    }
  }
  return PSOLVE_OK;
}

extern "C" int psolve_get_setup_times(psolve_t h, double* setup_ms, double* dgf_ms) {
  if (!h || !setup_ms || !dgf_ms) return fail(PSOLVE_ERR_ARG, "null argument");
  *setup_ms = h->setup_ms;
  *dgf_ms = h->dgf_ms;
  return PSOLVE_OK;
}

extern "C" int psolve_set_warm_start(psolve_t h, int enable) {
  if (!h) return fail(PSOLVE_ERR_ARG, "null handle");
  if (enable && !h->psi_prev) {
    h->psi_prev = static_cast<double2*>(h->A.get(plane_bytes(h)));
    h->phi_prev = static_cast<double2*>(h->A.get(plane_bytes(h)));
    if (!h->psi_prev || !h->phi_prev) {
      h->psi_prev = h->phi_prev = nullptr;
      return fail(PSOLVE_ERR_NOMEM, "warm-start buffers: out of device memory");
    }
  }
  h->warm = enable ? 1 : 0;
  h->warm_hist = 0;
  return PSOLVE_OK;
}

extern "C" int psolve_set_stream(psolve_t h, void* s) {
  if (!h) return fail(PSOLVE_ERR_ARG, "null handle");
  h->st = static_cast<cudaStream_t>(s);
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  return PSOLVE_OK;
}

extern "C" int psolve_set_tail(psolve_t h, int max_planes) {
  if (!h) return fail(PSOLVE_ERR_ARG, "null handle");
  if (max_planes < -1) return fail(PSOLVE_ERR_ARG, "max_planes must be -1, 0 or positive");
  h->mg.tail_cap = max_planes;
  h->mg.prepare_tail();
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  return cuda_ok("set_tail") ? PSOLVE_OK : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_get_tail(psolve_t h, int* planes, int* cluster_ctas) {
  if (!h) return fail(PSOLVE_ERR_ARG, "null handle");
  if (planes) *planes = h->mg.tail_planes;
  if (cluster_ctas) *cluster_ctas = h->mg.tail_planes > 0 ? h->mg.tl.C : 0;
  return PSOLVE_OK;
}

extern "C" const char* psolve_last_error(void) { return g_err.c_str(); }

extern "C" int psolve_get_sizes(psolve_t h, int* n_modes, int* n_boundary, int* n_levels) {
  if (!h) return fail(PSOLVE_ERR_ARG, "null handle");
  if (n_modes) *n_modes = h->M;
  if (n_boundary) *n_boundary = h->nb;
  if (n_levels) *n_levels = int(h->mg.lv.size());
  return PSOLVE_OK;
}

// ---------------------------------------------------------------------------
// the solve (Sec. 5.1 steps 2-7)
// ---------------------------------------------------------------------------
static size_t cells(psolve_t h) { return size_t(h->d.n_r) * h->d.n_tz * h->d.n_phi; }
static size_t mode_plane(psolve_t h) { return size_t(h->d.n_r) * h->d.n_tz; }

// Records stage mark k on the handle's stream (an event node when the stream
// is being captured, so that every replay records it).
static void mark(psolve_t h, int k) {
  if (!h->mark[k]) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(h->st, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(h->mark[k], h->st, cudaEventRecordExternal);
  else
    cudaEventRecord(h->mark[k], h->st);
}

static void enqueue_front(psolve_t h, const double* rho) {
  mark(h, 0);
  for (int b = 0; b < h->nd; ++b)
    launch_fft_forward(rho + b * cells(h), h->f + size_t(b) * h->M * mode_plane(h), h->d.n_r, h->d.n_tz,
                       h->d.n_phi, 4.0 * kPi * h->d.G / h->d.n_phi, h->tw, h->st);
  mark(h, 1);
  if (warm_state(h) == 2)
    cudaMemcpyAsync(h->u, h->psi_prev, plane_bytes(h), cudaMemcpyDeviceToDevice, h->st);
  else
    cudaMemsetAsync(h->u, 0, plane_bytes(h), h->st);
  h->mg.zero_guess = warm_state(h) == 2 ? 0 : 1;   // the Psi loop is enqueued next
  h->mg.init_loop(h->st);
}

static void enqueue_middle(psolve_t h) {
  mark(h, 2);
  snapshot(h, h->sp);
  if (h->warm) cudaMemcpyAsync(h->psi_prev, h->u, plane_bytes(h), cudaMemcpyDeviceToDevice, h->st);
  launch_screening(h->bdev, h->u, h->sigma, h->P, h->st);
  if (h->nd == 1) launch_boundary_potential(h->gt, h->sigma, h->theta, h->M, h->nb, h->st);
  else launch_boundary_potential_multi(h->gt, h->sigma, h->theta, h->M, h->nb, h->nd, h->st);
  launch_rhs_ghosts(h->bdev, h->f, h->theta, h->P, h->st);
  // initial guess of the Phi solve: the previous Phi (warm start), else Psi
  if (warm_state(h) == 2)
    cudaMemcpyAsync(h->u, h->phi_prev, plane_bytes(h), cudaMemcpyDeviceToDevice, h->st);
  h->mg.zero_guess = 0;   // the Phi loop starts from Psi or the previous Phi
  h->mg.init_loop(h->st);
  mark(h, 3);
}

static void enqueue_back(psolve_t h, double* phi) {
  mark(h, 4);
  snapshot(h, h->sf);
  if (h->warm) cudaMemcpyAsync(h->phi_prev, h->u, plane_bytes(h), cudaMemcpyDeviceToDevice, h->st);
  for (int b = 0; b < h->nd; ++b)
    launch_fft_inverse(h->u + size_t(b) * h->M * mode_plane(h), phi + b * cells(h), h->d.n_r, h->d.n_tz,
                       h->d.n_phi, h->tw, h->st);
  k_worst<<<1, 256, 0, h->st>>>(h->sp.status, h->sf.status, h->P, h->d_worst);
  cudaMemcpyAsync(h->h_worst, h->d_worst, sizeof(int), cudaMemcpyDeviceToHost, h->st);
  mark(h, 5);
}

static int add_while(psolve_t h, cudaGraph_t graph, double tol, cudaStream_t body_st) {
  cudaGraphConditionalHandle cond;
  if (cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return -1;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraph_t cg;
  if (cudaStreamGetCaptureInfo(h->st, &cs, nullptr, &cg, &deps, nullptr, &ndeps) != cudaSuccess)
    return -1;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = cond;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &p) != cudaSuccess) return -1;
  cudaGraph_t body = p.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(h->st, &node, nullptr, 1,
                                          cudaStreamSetCaptureDependencies) != cudaSuccess)
    return -1;
  if (cudaStreamBeginCaptureToGraph(body_st, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return -1;
  h->mg.loop_body(h->f, h->u, tol, body_st, 1, cond);
  cudaGraph_t out;
  if (cudaStreamEndCapture(body_st, &out) != cudaSuccess) return -1;
  h->mg.tail(h->f, h->u, tol, h->st);   // planes the loop handed over (none: returns at once)
  return 0;
}

static int capture(psolve_t h, const double* rho, double* phi, double tol) {
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  cudaStream_t cap = h->st, body_st;
  bool own = false;
  if (cap == 0) {   // the legacy stream cannot be captured
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return -1;
    own = true;
  }
  cudaStream_t saved = h->st;
  h->st = cap;
  cudaStreamCreateWithFlags(&body_st, cudaStreamNonBlocking);
  cudaGraph_t graph;
  cudaGraphCreate(&graph, 0);
  int rc = 0;
  if (cudaStreamBeginCaptureToGraph(cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
      cudaSuccess)
    rc = -1;
  if (!rc) {
    enqueue_front(h, rho);
    rc = add_while(h, graph, tol, body_st);
    if (!rc) {
      enqueue_middle(h);
      rc = add_while(h, graph, tol, body_st);
    }
    if (!rc) enqueue_back(h, phi);
    cudaGraph_t g2;
    if (cudaStreamEndCapture(cap, &g2) != cudaSuccess) rc = -1;
  }
  if (!rc && cudaGraphInstantiate(&h->gexec, graph, 0) != cudaSuccess) rc = -1;
  cudaGraphDestroy(graph);
  cudaStreamDestroy(body_st);
  h->st = saved;
  if (own) cudaStreamDestroy(cap);
  cudaGetLastError();
  if (rc) { h->gexec = nullptr; return -1; }
  h->g_rho = rho;
  h->g_phi = phi;
  h->g_tol = tol;
  h->g_warm = warm_state(h);
  return 0;
}

// After a warm-start solve the history holds its Psi and Phi (also the last
// iterates of a solve that stopped short of the tolerance); a non-finite or
// failed solve discards it.
static void note_history(psolve_t h, int rc) {
  if (h->warm) h->warm_hist = (rc == PSOLVE_OK || rc == PSOLVE_ERR_NOT_CONVERGED) ? 1 : 0;
}

static int finish(psolve_t h) {
  if (cudaStreamSynchronize(h->st) != cudaSuccess || !cuda_ok("solve"))
    return fail(PSOLVE_ERR_CUDA, g_err.empty() ? "solve failed" : g_err);
  const int w = *h->h_worst;
  if (w == -5) return fail(PSOLVE_ERR_NONFINITE, "non-finite residual norm");
  if (w == -4) return fail(PSOLVE_ERR_NOT_CONVERGED, "a mode did not reach the tolerance");
  return PSOLVE_OK;
}

static int enqueue_solve(psolve_t h, const double* rho, double* phi, double tol) {
  if (h->d.use_graph) {
    if (!h->gexec || h->g_rho != rho || h->g_phi != phi || h->g_tol != tol ||
        h->g_warm != warm_state(h)) {
      if (capture(h, rho, phi, tol) != 0)
        return fail(PSOLVE_ERR_CUDA, "graph capture failed: " + g_err);
    }
    if (cudaGraphLaunch(h->gexec, h->st) != cudaSuccess) return fail(PSOLVE_ERR_CUDA, "graph launch");
    return PSOLVE_OK;
  }
  std::string err;
  enqueue_front(h, rho);
  if (h->mg.eager_solve(h->f, h->u, tol, h->st, err) != 0) return fail(PSOLVE_ERR_CUDA, err);
  enqueue_middle(h);
  if (h->mg.eager_solve(h->f, h->u, tol, h->st, err) != 0) return fail(PSOLVE_ERR_CUDA, err);
  enqueue_back(h, phi);
  return PSOLVE_OK;
}

extern "C" int psolve_solve(psolve_t h, const double* rho, double* phi, double tol) {
  if (!h || !rho || !phi) return fail(PSOLVE_ERR_ARG, "null argument");
  if (rho == phi) return fail(PSOLVE_ERR_ARG, "phi must not alias rho");
  if (tol <= 0) tol = 1e-8;
  int rc = enqueue_solve(h, rho, phi, tol);
  if (rc != PSOLVE_OK) return rc;
  rc = finish(h);
  note_history(h, rc);
  return rc;
}

// ---- solves from host memory, copies overlapped with the solves -------------

static int pipe_ensure(psolve_t h, int n) {
  psolve_ctx::Pipe* p = h->pipe;
  if (!p) {
    p = h->pipe = new psolve_ctx::Pipe();
    const size_t bytes = sizeof(double) * size_t(h->nd) * cells(h);
    p->rho_dev = static_cast<double*>(h->A.get(bytes));
    p->rho_b = static_cast<double*>(h->A.get(bytes));
    p->phi_dev = static_cast<double*>(h->A.get(bytes));
    p->phi_b = static_cast<double*>(h->A.get(bytes));
    bool ok = p->rho_dev && p->rho_b && p->phi_dev && p->phi_b;
    ok = ok && cudaStreamCreateWithFlags(&p->up, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&p->down, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t* e : {&p->in_ready, &p->rho_free, &p->out_ready, &p->phi_free})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      pipe_release(h);
      return fail(PSOLVE_ERR_NOMEM, "host pipeline: staging buffers, streams or events");
    }
  }
  if (n > p->cap) {
    if (p->h_status) cudaFreeHost(p->h_status);
    p->h_status = nullptr;
    p->cap = 0;
    if (cudaMallocHost(&p->h_status, sizeof(int) * size_t(n)) != cudaSuccess) {
      cudaGetLastError();
      return fail(PSOLVE_ERR_NOMEM, "host pipeline: status array");
    }
    p->cap = n;
  }
  return PSOLVE_OK;
}

static int status_code(int worst) {
  return worst == -5 ? PSOLVE_ERR_NONFINITE : worst == -4 ? PSOLVE_ERR_NOT_CONVERGED : PSOLVE_OK;
}

extern "C" int psolve_solve_host(psolve_t h, int n, const double* const* rho_host,
                                 double* const* phi_host, double tol, int* status) {
  if (!h || n < 0 || (n > 0 && (!rho_host || !phi_host)))
    return fail(PSOLVE_ERR_ARG, "null argument or n < 0");
  for (int k = 0; k < n; ++k)
    if (!rho_host[k] || !phi_host[k]) return fail(PSOLVE_ERR_ARG, "null host buffer");
  if (n == 0) return PSOLVE_OK;
  if (tol <= 0) tol = 1e-8;
  int rc = pipe_ensure(h, n);
  if (rc != PSOLVE_OK) return rc;
  psolve_ctx::Pipe* p = h->pipe;
  const size_t cnt = size_t(h->nd) * cells(h), bytes = sizeof(double) * cnt;
  cudaStream_t C = h->st;
  // Stream C (the handle's): wait for the upload, move rho to the solve's
  // buffer, solve, wait until the previous download left phi_b, move phi
  // there.  Stream up: the next upload once rho_b is free.  Stream down: the
  // download of this solve's phi, overlapping the next solve.
  cudaEventRecord(p->phi_free, C);
  cudaMemcpyAsync(p->rho_b, rho_host[0], bytes, cudaMemcpyHostToDevice, p->up);
  cudaEventRecord(p->in_ready, p->up);
  int first = PSOLVE_OK;
  for (int k = 0; k < n; ++k) {
    cudaStreamWaitEvent(C, p->in_ready, 0);
    cudaMemcpyAsync(p->rho_dev, p->rho_b, bytes, cudaMemcpyDeviceToDevice, C);
    cudaEventRecord(p->rho_free, C);
    rc = enqueue_solve(h, p->rho_dev, p->phi_dev, tol);
    if (rc != PSOLVE_OK) {
      first = rc;
      break;
    }
    cudaMemcpyAsync(p->h_status + k, h->d_worst, sizeof(int), cudaMemcpyDeviceToHost, C);
    // a warm-started sequence continues from this solve (a failed one shows
    // in its status)
    note_history(h, PSOLVE_OK);
    cudaStreamWaitEvent(C, p->phi_free, 0);
    cudaMemcpyAsync(p->phi_b, p->phi_dev, bytes, cudaMemcpyDeviceToDevice, C);
    cudaEventRecord(p->out_ready, C);
    if (k + 1 < n) {
      cudaStreamWaitEvent(p->up, p->rho_free, 0);
      cudaMemcpyAsync(p->rho_b, rho_host[k + 1], bytes, cudaMemcpyHostToDevice, p->up);
      cudaEventRecord(p->in_ready, p->up);
    }
    cudaStreamWaitEvent(p->down, p->out_ready, 0);
    cudaMemcpyAsync(phi_host[k], p->phi_b, bytes, cudaMemcpyDeviceToHost, p->down);
    cudaEventRecord(p->phi_free, p->down);
  }
  const cudaError_t e1 = cudaStreamSynchronize(p->up), e2 = cudaStreamSynchronize(C),
                    e3 = cudaStreamSynchronize(p->down);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || !cuda_ok("solve_host"))
    return fail(PSOLVE_ERR_CUDA, g_err.empty() ? "host pipeline failed" : g_err);
  if (first != PSOLVE_OK) return first;
  for (int k = 0; k < n; ++k) {
    const int c = status_code(p->h_status[k]);
    if (status) status[k] = c;
    if (c != PSOLVE_OK && first == PSOLVE_OK) first = c;
  }
  if (h->warm && status_code(p->h_status[n - 1]) == PSOLVE_ERR_NONFINITE) h->warm_hist = 0;
  if (first == PSOLVE_ERR_NONFINITE) return fail(first, "non-finite residual norm in a solve");
  if (first == PSOLVE_ERR_NOT_CONVERGED) return fail(first, "a mode did not reach the tolerance in a solve");
  return PSOLVE_OK;
}

extern "C" int psolve_solve_batched(psolve_t* hs, const double* const* rhos, double* const* phis,
                                    int n, double tol) {
  if (!hs || !rhos || !phis || n < 0) return fail(PSOLVE_ERR_ARG, "null argument");
  if (tol <= 0) tol = 1e-8;
  for (int k = 0; k < n; ++k) {
    if (!hs[k] || !rhos[k] || !phis[k] || rhos[k] == phis[k])
      return fail(PSOLVE_ERR_ARG, "invalid batch entry");
    if (!hs[k]->d.use_graph) return fail(PSOLVE_ERR_ARG, "batched solves need use_graph handles");
  }
  for (int k = 0; k < n; ++k) {
    int rc = enqueue_solve(hs[k], rhos[k], phis[k], tol);
    if (rc != PSOLVE_OK) return rc;
  }
  int first = PSOLVE_OK;
  for (int k = 0; k < n; ++k) {
    int rc = finish(hs[k]);
    note_history(hs[k], rc);
    if (rc != PSOLVE_OK && first == PSOLVE_OK) first = rc;
  }
  return first;
}

// ---- many problems in one captured graph -----------------------------------

struct psolve_batch_ctx {
  std::vector<psolve_t> hs;
  std::vector<cudaStream_t> branch;   // capture branches, one per problem
  std::vector<cudaEvent_t> done;      // recorded by the graph when a problem's potential is written
  cudaEvent_t start = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void batch_release(psolve_batch_ctx* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s : b->branch) if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->done) if (e) cudaEventDestroy(e);
  if (b->start) cudaEventDestroy(b->start);
  delete b;
}

extern "C" int psolve_batch_create(psolve_batch_t* out, psolve_t* hs, const double* const* rhos,
                                   double* const* phis, int n, double tol) {
  if (!out || !hs || !rhos || !phis || n < 1) return fail(PSOLVE_ERR_ARG, "null argument or n < 1");
  *out = nullptr;
  if (tol <= 0) tol = 1e-8;
  for (int k = 0; k < n; ++k) {
    if (!hs[k] || !rhos[k] || !phis[k] || rhos[k] == phis[k]) return fail(PSOLVE_ERR_ARG, "invalid batch entry");
    for (int q = 0; q < k; ++q)
      if (hs[q] == hs[k]) return fail(PSOLVE_ERR_ARG, "a handle appears twice in the batch");
  }
  psolve_batch_ctx* b = new psolve_batch_ctx();
  b->hs.assign(hs, hs + n);
  b->branch.assign(n, nullptr);
  b->done.assign(n, nullptr);
  cudaStream_t root = nullptr, body = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join(n, nullptr);
  int rc = 0;
  if (cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&b->start) != cudaSuccess)
    rc = -1;
  for (int k = 0; k < n && !rc; ++k)
    if (cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->done[k]) != cudaSuccess ||
        cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming) != cudaSuccess)
      rc = -1;
  cudaGraph_t graph = nullptr;
  if (!rc && cudaGraphCreate(&graph, 0) != cudaSuccess) rc = -1;
  if (!rc && cudaStreamBeginCaptureToGraph(root, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
                 cudaSuccess)
    rc = -1;
  if (!rc) {
    cudaEventRecord(fork, root);
    // each problem's whole solve on its own branch: independent problems
    // overlap on the GPU; a completion event per problem
    for (int k = 0; k < n && !rc; ++k) {
      psolve_t h = hs[k];
      const cudaStream_t saved = h->st;
      h->st = b->branch[k];
      cudaStreamWaitEvent(h->st, fork, 0);
      enqueue_front(h, rhos[k]);
      rc = add_while(h, graph, tol, body);
      if (!rc) {
        enqueue_middle(h);
        rc = add_while(h, graph, tol, body);
      }
      if (!rc) {
        enqueue_back(h, phis[k]);
        cudaEventRecordWithFlags(b->done[k], h->st, cudaEventRecordExternal);
        cudaEventRecord(join[k], h->st);
        cudaStreamWaitEvent(root, join[k], 0);
      }
      h->st = saved;
    }
    cudaGraph_t g2;
    if (cudaStreamEndCapture(root, &g2) != cudaSuccess) rc = -1;
  }
  if (!rc && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) rc = -1;
  if (graph) cudaGraphDestroy(graph);
  if (body) cudaStreamDestroy(body);
  if (root) cudaStreamDestroy(root);
  if (fork) cudaEventDestroy(fork);
  for (cudaEvent_t e : join) if (e) cudaEventDestroy(e);
  const cudaError_t le = cudaGetLastError();
  if (rc || le != cudaSuccess) {
    batch_release(b);
    return fail(PSOLVE_ERR_CUDA, std::string("batch capture failed: ") + cudaGetErrorString(le));
  }
  *out = b;
  return PSOLVE_OK;
}

extern "C" int psolve_batch_run(psolve_batch_t b, void* stream, float* latency_ms) {
  if (!b) return fail(PSOLVE_ERR_ARG, "null batch");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEventRecord(b->start, st);
  if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return fail(PSOLVE_ERR_CUDA, "batch graph launch");
  if (cudaStreamSynchronize(st) != cudaSuccess || !cuda_ok("batch run"))
    return fail(PSOLVE_ERR_CUDA, g_err.empty() ? "batch run failed" : g_err);
  int first = PSOLVE_OK;
  for (size_t k = 0; k < b->hs.size(); ++k) {
    psolve_t h = b->hs[k];
    int rc = PSOLVE_OK;
    if (*h->h_worst == -5) rc = fail(PSOLVE_ERR_NONFINITE, "non-finite residual norm");
    else if (*h->h_worst == -4) rc = fail(PSOLVE_ERR_NOT_CONVERGED, "a mode did not reach the tolerance");
    note_history(h, rc);
    if (rc != PSOLVE_OK && first == PSOLVE_OK) first = rc;
    if (latency_ms && cudaEventElapsedTime(&latency_ms[k], b->start, b->done[k]) != cudaSuccess)
      return fail(PSOLVE_ERR_CUDA, "batch latency");
  }
  return first;
}

extern "C" void psolve_batch_destroy(psolve_batch_t b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_release(b);
}

// ---- smoothing schedule and autotuner ---------------------------------------

extern "C" int psolve_get_schedule(psolve_t h, psolve_schedule* s) {
  if (!h || !s) return fail(PSOLVE_ERR_ARG, "null argument");
  const MGOptions& o = h->mg.opt;
  *s = psolve_schedule{};
  s->nu_pre = o.nu1;
  s->nu_post = o.nu2;
  s->n_sor = o.n_sor;
  s->lines_r = o.tiles.lines_r;
  s->cols_t = o.tiles.cols_t;
  s->nu_pre_fused = o.nu1f;
  s->nu_post_fused = o.nu2f;
  s->tail_planes = h->mg.tail_cap;
  return PSOLVE_OK;
}

static bool schedule_ok(const psolve_schedule& s, std::string& why) {
  if (s.nu_pre < 1 || s.nu_pre > 8 || s.nu_post < 1 || s.nu_post > 8) why = "nu_pre and nu_post must be 1..8";
  else if (s.n_sor < 1 || s.n_sor > 8) why = "n_sor must be 1..8";
  else if (s.lines_r != 4 && s.lines_r != 8) why = "lines_r must be 4 or 8";
  else if (s.cols_t != 0 && s.cols_t != 8 && s.cols_t != 16 && s.cols_t != 32) why = "cols_t must be 0, 8, 16 or 32";
  else if (s.nu_pre_fused < 0 || s.nu_pre_fused > 8 || s.nu_post_fused < 0 || s.nu_post_fused > 8)
    why = "nu_pre_fused and nu_post_fused must be 0..8";
  else if (s.tail_planes < -1) why = "tail_planes must be -1, 0 or positive";
  else return true;
  return false;
}

static void install_schedule(psolve_t h, const psolve_schedule& s) {
  Tiles t;
  t.lines_r = s.lines_r;
  t.cols_t = s.cols_t;
  h->mg.tail_cap = s.tail_planes;
  h->mg.set_schedule(s.nu_pre, s.nu_post, s.n_sor, t, s.nu_pre_fused, s.nu_post_fused);
  h->d.nu_pre = s.nu_pre;
  h->d.nu_post = s.nu_post;
  h->d.n_sor = s.n_sor;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
}

extern "C" int psolve_set_schedule(psolve_t h, const psolve_schedule* s) {
  if (!h || !s) return fail(PSOLVE_ERR_ARG, "null argument");
  std::string why;
  if (!schedule_ok(*s, why)) return fail(PSOLVE_ERR_ARG, "psolve_set_schedule: " + why);
  install_schedule(h, *s);
  return PSOLVE_OK;
}

static std::mutex g_tune_mu;
static std::vector<std::pair<std::string, psolve_schedule>> g_tune;   // process cache

static std::string tune_key(const psolve_desc& d) {
  char b[320];
  std::snprintf(b, sizeof b, "g%d:nr%d:nt%d:np%d:sp%d:r%.17g:%.17g:t%.17g:%.17g:p%d", d.geometry,
                d.n_r, d.n_tz, d.n_phi, d.spacing, d.r_in, d.r_out, d.t_min, d.t_max, d.precision);
  return b;
}

static const psolve_schedule* tune_find(const std::string& key) {
  for (auto it = g_tune.rbegin(); it != g_tune.rend(); ++it)
    if (it->first == key) return &it->second;
  return nullptr;
}

// The last valid line of `key` in the cache file, if any.
static bool tune_file_read(const char* path, const std::string& key, psolve_schedule& out) {
  FILE* fp = std::fopen(path, "r");
  if (!fp) return false;
  bool found = false;
  char line[512], k[384];
  while (std::fgets(line, sizeof line, fp)) {
    psolve_schedule s{};
    if (std::sscanf(line, "%383s %d %d %d %d %d %d %d %lf %d", k, &s.nu_pre, &s.nu_post, &s.n_sor,
                    &s.lines_r, &s.cols_t, &s.nu_pre_fused, &s.nu_post_fused, &s.ms, &s.tail_planes) != 10)
      continue;
    std::string why;
    if (key == k && schedule_ok(s, why)) {
      out = s;
      found = true;
    }
  }
  std::fclose(fp);
  return found;
}

static void tune_file_append(const char* path, const std::string& key, const psolve_schedule& s) {
  FILE* fp = std::fopen(path, "a");
  if (!fp) return;
  std::fprintf(fp, "%s %d %d %d %d %d %d %d %.4f %d\n", key.c_str(), s.nu_pre, s.nu_post, s.n_sor,
               s.lines_r, s.cols_t, s.nu_pre_fused, s.nu_post_fused, s.ms, s.tail_planes);
  std::fclose(fp);
}

// Median of three timed solves after one untimed solve; PSOLVE_OK or the
// failing solve's code.
static int time_solves(psolve_t h, const double* rho, double* phi, double tol, cudaEvent_t e0,
                       cudaEvent_t e1, double& ms) {
  int rc = enqueue_solve(h, rho, phi, tol);
  if (rc == PSOLVE_OK) rc = finish(h);
  if (rc != PSOLVE_OK) return rc;
  float t[3];
  for (int k = 0; k < 3; ++k) {
    cudaEventRecord(e0, h->st);
    rc = enqueue_solve(h, rho, phi, tol);
    cudaEventRecord(e1, h->st);
    if (rc == PSOLVE_OK) rc = finish(h);
    if (rc != PSOLVE_OK) return rc;
    if (cudaEventElapsedTime(&t[k], e0, e1) != cudaSuccess) return fail(PSOLVE_ERR_CUDA, "autotune timing");
  }
  const float lo = std::fmin(t[0], std::fmin(t[1], t[2])), hi = std::fmax(t[0], std::fmax(t[1], t[2]));
  ms = double(t[0] + t[1] + t[2] - lo - hi);
  return PSOLVE_OK;
}

extern "C" int psolve_autotune(psolve_t h, const double* rho, double* phi, double tol,
                               psolve_schedule* out) {
  if (!h || !rho || !phi) return fail(PSOLVE_ERR_ARG, "null argument");
  if (rho == phi) return fail(PSOLVE_ERR_ARG, "phi must not alias rho");
  if (tol <= 0) tol = 1e-8;
  const std::string key = tune_key(h->d);
  const char* path = std::getenv("PSOLVE_TUNE_CACHE");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  psolve_schedule best{};
  const psolve_schedule* hit = tune_find(key);
  if (hit || (path && *path && tune_file_read(path, key, best))) {
    if (hit) best = *hit;
    else g_tune.emplace_back(key, best);
    install_schedule(h, best);
    best.candidates = 0;
    best.cached = 1;
    if (out) *out = best;
    return PSOLVE_OK;
  }
  psolve_schedule cur{};
  psolve_get_schedule(h, &cur);
  const int warm = h->warm;
  h->warm = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // stage 1: schedules, the current one first
  std::vector<psolve_schedule> cand{cur};
  for (int a = 1; a <= 3; ++a)
    for (int b = 1; b <= a; ++b)
      for (int c = 1; c <= 3; ++c) {
        psolve_schedule s = cur;
        s.nu_pre = a;
        s.nu_post = b;
        s.n_sor = c;
        s.nu_pre_fused = s.nu_post_fused = 0;
        if (a != cur.nu_pre || b != cur.nu_post || c != cur.n_sor) cand.push_back(s);
      }
  int n_timed = 0, rc0 = PSOLVE_OK;
  best = cur;
  best.ms = -1;
  for (size_t k = 0; k < cand.size(); ++k) {
    double ms = 0;
    install_schedule(h, cand[k]);
    const int rc = time_solves(h, rho, phi, tol, e0, e1, ms);
    if (k == 0) rc0 = rc;
    if (rc != PSOLVE_OK) {
      if (k == 0) break;   // the current schedule fails: keep it and report
      continue;
    }
    ++n_timed;
    if (best.ms < 0 || ms < best.ms) { best = cand[k]; best.ms = ms; }
  }
  if (rc0 == PSOLVE_OK) {
    // stage 2: tile shapes with the chosen schedule (distinct launches only)
    const size_t vb = h->d.precision ? 8 : 16;
    std::vector<int> widths;
    for (int want : {8, 16, 32}) {
      const int w = smooth_tile_cols(h->d.n_r, h->d.n_tz, vb, want);
      bool seen = false;
      for (int x : widths) seen = seen || x == w;
      if (!seen) widths.push_back(w);
    }
    const int cur_w = smooth_tile_cols(h->d.n_r, h->d.n_tz, vb, best.cols_t);
    for (int lines : {8, 4})
      for (int w : widths) {
        if (lines == best.lines_r && w == cur_w) continue;   // timed in stage 1
        psolve_schedule s = best;
        s.lines_r = lines;
        s.cols_t = w;
        double ms = 0;
        install_schedule(h, s);
        if (time_solves(h, rho, phi, tol, e0, e1, ms) != PSOLVE_OK) continue;
        ++n_timed;
        if (ms < best.ms) { best = s; best.ms = ms; }
      }
    // stage 3: the fused levels' own smoothing counts
    if (h->mg.vs.nlev > 1) {   // the fused kernel smooths at least one level
      const int a0 = best.nu_pre_fused > 0 ? best.nu_pre_fused : best.nu_pre;
      const int b0 = best.nu_post_fused > 0 ? best.nu_post_fused : best.nu_post;
      const psolve_schedule base = best;
      for (int a = 1; a <= 3; ++a)
        for (int b = 1; b <= a; ++b) {
          if (a == a0 && b == b0) continue;
          psolve_schedule s = base;
          s.nu_pre_fused = a;
          s.nu_post_fused = b;
          double ms = 0;
          install_schedule(h, s);
          if (time_solves(h, rho, phi, tol, e0, e1, ms) != PSOLVE_OK) continue;
          ++n_timed;
          if (ms < best.ms) { best = s; best.ms = ms; }
        }
    }
    // stage 4: the cluster-resident tail off against on
    {
      psolve_schedule s = best;
      s.tail_planes = best.tail_planes == 0 ? -1 : 0;
      install_schedule(h, s);
      double ms = 0;
      if (h->mg.tail_planes > 0 || s.tail_planes == 0) {
        if (time_solves(h, rho, phi, tol, e0, e1, ms) == PSOLVE_OK) {
          ++n_timed;
          if (ms < best.ms) { best = s; best.ms = ms; }
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->warm = warm;
  if (rc0 != PSOLVE_OK) {
    install_schedule(h, cur);
    return rc0;
  }
  install_schedule(h, best);
  best.candidates = n_timed;
  best.cached = 0;
  g_tune.emplace_back(key, best);
  if (path && *path) tune_file_append(path, key, best);
  if (out) *out = best;
  return PSOLVE_OK;
}

extern "C" int psolve_get_stats(psolve_t h, psolve_stats* s) {
  if (!h || !s) return fail(PSOLVE_ERR_ARG, "null argument");
  cudaStreamSynchronize(h->st);
  const int M = h->M;
  s->n_modes = M;
  s->setup_ms = h->setup_ms;
  const int P = h->P;   // the residual covers every density's planes
  std::vector<double2> nf(P), nr(P);
  for (int pass = 0; pass < 2; ++pass) {
    SolveStats& q = pass ? h->sf : h->sp;
    int it = 0;
    cudaMemcpy(&it, q.iter, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(nf.data(), q.nf2, sizeof(double2) * P, cudaMemcpyDeviceToHost);
    cudaMemcpy(nr.data(), q.nr2, sizeof(double2) * P, cudaMemcpyDeviceToHost);
    double a = 0, b = 0;
    for (int m = 0; m < P; ++m) { a += nr[m].x + nr[m].y; b += nf[m].x + nf[m].y; }
    const double rel = b > 0 ? std::sqrt(a / b) : 0.0;
    int* cyc = pass ? s->cycles_phi : s->cycles_psi;
    if (cyc) cudaMemcpy(cyc, q.cycles, sizeof(int) * M, cudaMemcpyDeviceToHost);
    if (pass) { s->iterations_phi = it - 1; s->rel_residual_phi = rel; }
    else { s->iterations_psi = it - 1; s->rel_residual_psi = rel; }
  }
  if (s->status) {
    std::vector<int> a(M), b(M);
    cudaMemcpy(a.data(), h->sp.status, sizeof(int) * M, cudaMemcpyDeviceToHost);
    cudaMemcpy(b.data(), h->sf.status, sizeof(int) * M, cudaMemcpyDeviceToHost);
    for (int m = 0; m < M; ++m) {
      int w = PSOLVE_OK;
      if (a[m] == -5 || b[m] == -5) w = PSOLVE_ERR_NONFINITE;
      else if (a[m] != 0 || b[m] != 0) w = PSOLVE_ERR_NOT_CONVERGED;
      s->status[m] = w;
    }
  }
  return cuda_ok("stats") ? PSOLVE_OK : PSOLVE_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// stage entry points
// ---------------------------------------------------------------------------
extern "C" int psolve_stage_forward(psolve_t h, const double* rho, double* f_hat) {
  if (!h || !rho || !f_hat) return fail(PSOLVE_ERR_ARG, "null argument");
  launch_fft_forward(rho, reinterpret_cast<double2*>(f_hat), h->d.n_r, h->d.n_tz, h->d.n_phi,
                     4.0 * kPi * h->d.G / h->d.n_phi, h->tw, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("forward") ? PSOLVE_OK
                                                                             : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_stage_forward_rows(psolve_t h, const double* rho_rows, int n_rows,
                                         double* f_hat_rows) {
  if (!h || !rho_rows || !f_hat_rows) return fail(PSOLVE_ERR_ARG, "null argument");
  if (n_rows < 1 || n_rows > h->d.n_r) return fail(PSOLVE_ERR_ARG, "n_rows must lie in 1..n_r");
  launch_fft_forward(rho_rows, reinterpret_cast<double2*>(f_hat_rows), n_rows, h->d.n_tz, h->d.n_phi,
                     4.0 * kPi * h->d.G / h->d.n_phi, h->tw, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("forward_rows") ? PSOLVE_OK
                                                                                  : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_stage_inverse_rows(psolve_t h, const double* phi_hat_rows, int n_rows,
                                         double* phi_rows) {
  if (!h || !phi_hat_rows || !phi_rows) return fail(PSOLVE_ERR_ARG, "null argument");
  if (n_rows < 1 || n_rows > h->d.n_r) return fail(PSOLVE_ERR_ARG, "n_rows must lie in 1..n_r");
  launch_fft_inverse(reinterpret_cast<const double2*>(phi_hat_rows), phi_rows, n_rows, h->d.n_tz,
                     h->d.n_phi, h->tw, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("inverse_rows") ? PSOLVE_OK
                                                                                  : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_solve_modes(psolve_t h, const int* modes_host, int n, const double* f_hat,
                                  double* phi_hat, double tol) {
  if (!h || (n > 0 && (!modes_host || !f_hat || !phi_hat))) return fail(PSOLVE_ERR_ARG, "null argument");
  if (n < 0 || n > h->M) return fail(PSOLVE_ERR_ARG, "n must lie in 0..n_modes");
  if (n > 0 && f_hat == phi_hat) return fail(PSOLVE_ERR_ARG, "phi_hat must not alias f_hat");
  std::vector<char> seen(h->M, 0);
  for (int k = 0; k < n; ++k) {
    const int m = modes_host[k];
    if (m < 0 || m >= h->M || seen[m]) return fail(PSOLVE_ERR_ARG, "modes must be distinct and in 0..n_modes-1");
    seen[m] = 1;
  }
  if (tol <= 0) tol = 1e-8;
  const size_t plane = size_t(h->d.n_r) * h->d.n_tz;
  const int warm = h->warm;
  h->warm = 0;   // the history belongs to whole-problem solves
  // the listed modes' right-hand sides in their planes, zero elsewhere: a
  // zero plane meets the criterion at its first residual and retires
  cudaMemsetAsync(h->f, 0, plane_bytes(h), h->st);
  for (int k = 0; k < n; ++k)
    cudaMemcpyAsync(h->f + size_t(modes_host[k]) * plane, reinterpret_cast<const double2*>(f_hat) + k * plane,
                    plane * sizeof(double2), cudaMemcpyDeviceToDevice, h->st);
  cudaMemsetAsync(h->u, 0, plane_bytes(h), h->st);
  h->mg.zero_guess = 1;
  h->mg.init_loop(h->st);
  std::string err;
  int rc = PSOLVE_OK;
  if (h->mg.eager_solve(h->f, h->u, tol, h->st, err) != 0) rc = fail(PSOLVE_ERR_CUDA, err);
  if (rc == PSOLVE_OK) {
    enqueue_middle(h);
    if (h->mg.eager_solve(h->f, h->u, tol, h->st, err) != 0) rc = fail(PSOLVE_ERR_CUDA, err);
  }
  h->warm = warm;
  if (rc != PSOLVE_OK) return rc;
  snapshot(h, h->sf);
  for (int k = 0; k < n; ++k)
    cudaMemcpyAsync(reinterpret_cast<double2*>(phi_hat) + k * plane, h->u + size_t(modes_host[k]) * plane,
                    plane * sizeof(double2), cudaMemcpyDeviceToDevice, h->st);
  k_worst<<<1, 256, 0, h->st>>>(h->sp.status, h->sf.status, h->P, h->d_worst);
  cudaMemcpyAsync(h->h_worst, h->d_worst, sizeof(int), cudaMemcpyDeviceToHost, h->st);
  return finish(h);
}

extern "C" int psolve_stage_inverse(psolve_t h, const double* phi_hat, double* phi) {
  if (!h || !phi_hat || !phi) return fail(PSOLVE_ERR_ARG, "null argument");
  launch_fft_inverse(reinterpret_cast<const double2*>(phi_hat), phi, h->d.n_r, h->d.n_tz,
                     h->d.n_phi, h->tw, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("inverse") ? PSOLVE_OK
                                                                             : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_stage_mg_solve(psolve_t h, const double* f_hat, double* u_hat, double tol,
                                     int warm, int* cycles_host) {
  if (!h || !f_hat || !u_hat) return fail(PSOLVE_ERR_ARG, "null argument");
  if (tol <= 0) tol = 1e-8;
  const size_t bytes = sizeof(double2) * size_t(h->M) * h->d.n_r * h->d.n_tz;
  if (!warm) cudaMemsetAsync(u_hat, 0, bytes, h->st);
  h->mg.zero_guess = warm ? 0 : 1;
  std::string err;
  if (h->mg.eager_solve(reinterpret_cast<const double2*>(f_hat), reinterpret_cast<double2*>(u_hat),
                        tol, h->st, err) != 0)
    return fail(PSOLVE_ERR_CUDA, err);
  if (cycles_host)
    cudaMemcpyAsync(cycles_host, h->mg.d_cycles, sizeof(int) * h->M, cudaMemcpyDeviceToHost, h->st);
  if (cudaStreamSynchronize(h->st) != cudaSuccess || !cuda_ok("mg_solve")) return PSOLVE_ERR_CUDA;
  std::vector<int> st(h->M);
  cudaMemcpy(st.data(), h->mg.d_status, sizeof(int) * h->M, cudaMemcpyDeviceToHost);
  for (int v : st)
    if (v == -5) return fail(PSOLVE_ERR_NONFINITE, "non-finite residual");
  for (int v : st)
    if (v != 0) return fail(PSOLVE_ERR_NOT_CONVERGED, "a mode did not converge");
  return PSOLVE_OK;
}

// Stage helpers operate on all M planes: a full active list.
static void full_batch(psolve_t h) {
  launch_init_active(h->mg.d_act, h->mg.d_nact, h->M, h->mg.S, h->st);
}

static int check_level(psolve_t h, int level, int precision, bool need_next) {
  if (level < 0 || level >= int(h->mg.lv.size()) || (need_next && level + 1 >= int(h->mg.lv.size())))
    return fail(PSOLVE_ERR_ARG, "level out of range");
  if (precision != (h->d.precision == PSOLVE_MIXED ? 1 : 0))
    return fail(PSOLVE_ERR_ARG, "stage precision must match the handle (0 FP64, 1 mixed/FP32)");
  return PSOLVE_OK;
}

extern "C" int psolve_stage_smooth(psolve_t h, int level, int precision, void* e, const void* f,
                                   int cycles) {
  if (!h || !e || !f) return fail(PSOLVE_ERR_ARG, "null argument");
  int rc = check_level(h, level, precision, false);
  if (rc) return rc;
  full_batch(h);
  h->mg.smooth(level, e, f, cycles, false, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("smooth") ? PSOLVE_OK
                                                                            : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_stage_restrict(psolve_t h, int level, int precision, const void* e,
                                     const void* f, void* coarse) {
  if (!h || !e || !f || !coarse) return fail(PSOLVE_ERR_ARG, "null argument");
  int rc = check_level(h, level, precision, true);
  if (rc) return rc;
  full_batch(h);
  h->mg.restrict_(level, e, f, coarse, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("restrict") ? PSOLVE_OK
                                                                              : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_stage_prolong(psolve_t h, int level, int precision, void* e,
                                    const void* coarse) {
  if (!h || !e || !coarse) return fail(PSOLVE_ERR_ARG, "null argument");
  int rc = check_level(h, level, precision, true);
  if (rc) return rc;
  full_batch(h);
  h->mg.prolong(level, e, coarse, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("prolong") ? PSOLVE_OK
                                                                             : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_stage_residual(psolve_t h, int precision, const double* f, const double* u,
                                     void* r) {
  if (!h || !f || !u || !r) return fail(PSOLVE_ERR_ARG, "null argument");
  int rc = check_level(h, 0, precision, false);
  if (rc) return rc;
  full_batch(h);
  h->mg.residual_to(reinterpret_cast<const double2*>(f), reinterpret_cast<const double2*>(u), r,
                    h->st);
  return cuda_ok("residual") ? PSOLVE_OK : PSOLVE_ERR_CUDA;   // asynchronous
}

extern "C" int psolve_get_fused_level(psolve_t h, int* level) {
  if (!h || !level) return fail(PSOLVE_ERR_ARG, "null argument");
  *level = h->mg.first;
  return PSOLVE_OK;
}

extern "C" int psolve_stage_vcycle(psolve_t h, int level, int precision, const void* f, void* e) {
  if (!h || !f || !e) return fail(PSOLVE_ERR_ARG, "null argument");
  int rc = check_level(h, level, precision, false);
  if (rc) return rc;
  if (level != h->mg.first)
    return fail(PSOLVE_ERR_ARG, "the fused V-cycle starts at level " + std::to_string(h->mg.first));
  full_batch(h);
  if (precision)
    launch_vsmem<float>(h->mg.vs, h->mg.batch, static_cast<const float2*>(f), static_cast<float2*>(e), h->st);
  else
    launch_vsmem<double>(h->mg.vs, h->mg.batch, static_cast<const double2*>(f), static_cast<double2*>(e),
                         h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("vcycle") ? PSOLVE_OK
                                                                            : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_stage_screening(psolve_t h, const double* psi_hat, double* sigma) {
  if (!h || !psi_hat || !sigma) return fail(PSOLVE_ERR_ARG, "null argument");
  launch_screening(h->bdev, reinterpret_cast<const double2*>(psi_hat),
                   reinterpret_cast<double2*>(sigma), h->M, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("screening") ? PSOLVE_OK
                                                                               : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_stage_boundary(psolve_t h, const double* sigma, double* theta) {
  if (!h || !sigma || !theta) return fail(PSOLVE_ERR_ARG, "null argument");
  launch_boundary_potential(h->gt, reinterpret_cast<const double2*>(sigma),
                            reinterpret_cast<double2*>(theta), h->M, h->nb, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("boundary") ? PSOLVE_OK
                                                                              : PSOLVE_ERR_CUDA;
}

extern "C" int psolve_get_dgf(psolve_t h, double* dst) {
  if (!h || !dst) return fail(PSOLVE_ERR_ARG, "null argument");
  cudaMemcpyAsync(dst, h->gt, sizeof(double) * size_t(h->M) * h->nb * h->nb,
                  cudaMemcpyDeviceToDevice, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("dgf") ? PSOLVE_OK
                                                                         : PSOLVE_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Allocation-free smoothing step (psolve_stage_smooth_static)
//
// For callers that must not allocate device memory when they run a step: a
// host code that has handed all remaining device memory to its own pool
// after creating the handle, or that cannot afford the device-wide
// synchronisation cudaMalloc / cudaFree may imply.  The step's working
// memory -- the active-plane list and the ping-pong plane buffer of the
// radial -> polar passes -- lives in the file-scope array below instead of
// the handle's workspaces; the handle contributes only read-only tables.
// Every GPU that loads this library holds the array until the process exits.
// Calls share it and it keeps the last call's contents, so calls whose work
// overlaps on one GPU (different streams, threads or handles) race.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_scratch[PSOLVE_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_dev[kMaxDevices] = {};   // device address of g_static_scratch, per device

// In host code g_static_scratch names a host-side stand-in; the device
// address is looked up once per device, with that device current.
int static_scratch(int handle_device, void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PSOLVE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != handle_device)
    return fail(PSOLVE_ERR_ARG, "the handle's device (" + std::to_string(handle_device) +
                                    ") must be current, not device " + std::to_string(dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PSOLVE_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(PSOLVE_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") +
                                       cudaGetErrorString(e));
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return PSOLVE_OK;
}

__global__ void k_static_active(int* act, int* nact, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) act[k] = k;
  if (blockIdx.x == 0 && threadIdx.x == 0) *nact = n;
}
}  // namespace

extern "C" int psolve_stage_smooth_static(psolve_t h, int level, int precision, void* e,
                                          const void* f, int cycles) {
  if (!h || !e || !f) return fail(PSOLVE_ERR_ARG, "null argument");
  if (cycles < 0) return fail(PSOLVE_ERR_ARG, "cycles must be >= 0");
  int rc = check_level(h, level, precision, false);
  if (rc) return rc;
  const LevelDev& L = h->mg.lv[level];
  const size_t list_bytes = (sizeof(int) * (size_t(h->M) + 1) + 255) / 256 * 256;
  const size_t plane_bytes =
      size_t(h->M) * L.nr * L.nt * (precision ? sizeof(float2) : sizeof(double2));
  if (list_bytes + plane_bytes > PSOLVE_STATIC_SCRATCH_BYTES)
    return fail(PSOLVE_ERR_ARG,
                "psolve_stage_smooth_static: this level needs " +
                    std::to_string(list_bytes + plane_bytes) +
                    " bytes of scratch, above the static limit of " +
                    std::to_string(size_t(PSOLVE_STATIC_SCRATCH_BYTES)) +
                    " bytes; use psolve_stage_smooth");
  unsigned char* base = nullptr;
  rc = static_scratch(h->device, reinterpret_cast<void**>(&base));
  if (rc) return rc;
  int* act = reinterpret_cast<int*>(base);
  // The active list is rewritten on every call (the array holds the last
  // call's list).  The plane buffer needs no clearing: each cycle's radial
  // pass writes every cell of it that the polar pass then reads.
  k_static_active<<<(h->M + 255) / 256, 256, 0, h->st>>>(act, act + h->M, h->M);
  Batch B = h->mg.batch;
  B.act = act;
  B.nact = act + h->M;
  if (precision)
    launch_smooth<float>(L, B, static_cast<float2*>(e), static_cast<const float2*>(f),
                         reinterpret_cast<float2*>(base + list_bytes), cycles, h->mg.opt.n_sor,
                         false, h->mg.opt.tiles, h->st);
  else
    launch_smooth<double>(L, B, static_cast<double2*>(e), static_cast<const double2*>(f),
                          reinterpret_cast<double2*>(base + list_bytes), cycles, h->mg.opt.n_sor,
                          false, h->mg.opt.tiles, h->st);
  return cudaStreamSynchronize(h->st) == cudaSuccess && cuda_ok("smooth_static") ? PSOLVE_OK
                                                                                   : PSOLVE_ERR_CUDA;
}
