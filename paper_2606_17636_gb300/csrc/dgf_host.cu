// Host orchestration of the discrete Green's function tables (Sec. 4.2):
// the extended-domain construction for logarithmic radial grids with
// r_out / r_in >= 100 (batched multigrid over source x mode planes, the
// inner face carrying the closed-form radial derivative as a flux) and the
// auxiliary-window construction otherwise ((2 n_pad + 1)^2 windows, n_pad =
// 16, closed-form Dirichlet ring, exact window solves; closed form for
// targets outside the window).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dgf.h"

namespace ps {

static const int kPad = 16;
static const double kTol = 1e-12;
static const double kPi = 3.14159265358979323846;

bool uses_extended(const Law& rl, int n_r) {
  return rl.spacing == LOGS && rl.hi / rl.lo >= 100.0 && n_r >= 32;
}

template <typename X>
static X* up(Arena& A, const std::vector<X>& v) {
  X* d = static_cast<X*>(A.get(std::max<size_t>(1, v.size()) * sizeof(X)));
  if (d && !v.empty()) cudaMemcpy(d, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice);
  return d;
}

static int kind_r(int geometry) { return geometry == SPH ? 0 : 1; }
static int kind_t(int geometry) { return geometry == SPH ? 2 : 3; }

static bool green(Arena& A, int geometry, int N, int M, double G, int deriv,
                  const std::vector<double>& xt, const std::vector<double>& yt,
                  const std::vector<double>& xs, const std::vector<double>& ys, const double* cosk,
                  double* out, long mstride, long pstride, const double* scale, long scale_mod,
                  cudaStream_t st) {
  if (xt.empty()) return true;
  GreenArgs g{};
  g.geometry = geometry; g.N = N; g.M = M; g.deriv = deriv; g.G = G;
  g.npairs = long(xt.size());
  g.xt = up(A, xt); g.yt = up(A, yt); g.xs = up(A, xs); g.ys = up(A, ys);
  if (!g.xt || !g.yt || !g.xs || !g.ys) return false;
  g.cosk = cosk; g.out = out; g.mstride = mstride; g.pstride = pstride;
  g.scale = scale; g.scale_mod = scale_mod;
  launch_green(g, st);
  return true;
}

static bool build_extended(const PlaneGeo& g, const Law& rlaw, const Law& tlaw,
                           const std::vector<BPoint>& bp, double* gt, Arena& A, const double* cosk,
                           cudaStream_t st, std::string& err) {
  const int nr = g.r.n, nt = g.t.n, nb = int(bp.size()), N = g.n_phi, M = N / 2 + 1;
  const int o_r = nr - 16;
  const bool bounded = g.geometry == CYL || g.has_lower() || g.has_upper();
  const int o_t = bounded ? nt / 2 : 0;
  PlaneGeo ext;
  ext.geometry = g.geometry; ext.n_phi = N; ext.G = g.G;
  ext.r = axis_from_law(kind_r(g.geometry), rlaw, 1 - o_r, nr + 16);
  ext.t = axis_from_law(kind_t(g.geometry), tlaw, 1 - o_t, nt + o_t);
  ext.build();
  const int nre = ext.r.n, nte = ext.t.n;
  std::vector<int> src(nb);
  std::vector<double> sx(nb), sy(nb), dV(nb);
  for (int s = 0; s < nb; ++s) {
    const int i = bp[s].i + o_r, j = bp[s].j + o_t;
    src[s] = (j - 1) * nre + (i - 1);
    sx[s] = ext.r.x[i];
    sy[s] = ext.t.x[j];
    dV[s] = bp[s].dV;
  }
  // closed-form data, layout [ghost][source][m]
  auto pairs = [&](const std::vector<double>& gx, const std::vector<double>& gy,
                   std::vector<double>& xt, std::vector<double>& yt, std::vector<double>& xs,
                   std::vector<double>& ys) {
    for (size_t q = 0; q < gx.size(); ++q)
      for (int s = 0; s < nb; ++s) {
        xt.push_back(gx[q]); yt.push_back(gy[q]); xs.push_back(sx[s]); ys.push_back(sy[s]);
      }
  };
  std::vector<double> gx, gy, xt, yt, xs, ys;
  for (int j = 1; j <= nte; ++j) { gx.push_back(ext.r.x[nre + 1]); gy.push_back(ext.t.x[j]); }
  pairs(gx, gy, xt, yt, xs, ys);
  double* gout = static_cast<double*>(A.get(sizeof(double) * size_t(nte) * nb * M));
  if (!gout || !green(A, g.geometry, N, M, g.G, 0, xt, yt, xs, ys, cosk, gout, 1, M, nullptr, 1, st)) {
    err = "out of device memory (DGF)";
    return false;
  }
  double *glo = nullptr, *ghi = nullptr;
  for (int side = 0; side < 2; ++side) {
    const bool has = side == 0 ? ext.has_lower() : ext.has_upper();
    if (!has) continue;
    gx.clear(); gy.clear(); xt.clear(); yt.clear(); xs.clear(); ys.clear();
    const int jg = side == 0 ? 0 : nte + 1;
    for (int i = 1; i <= nre; ++i) { gx.push_back(ext.r.x[i]); gy.push_back(ext.t.x[jg]); }
    pairs(gx, gy, xt, yt, xs, ys);
    double* dst = static_cast<double*>(A.get(sizeof(double) * size_t(nre) * nb * M));
    if (!dst || !green(A, g.geometry, N, M, g.G, 0, xt, yt, xs, ys, cosk, dst, 1, M, nullptr, 1, st)) {
      err = "out of device memory (DGF)";
      return false;
    }
    (side == 0 ? glo : ghi) = dst;
  }
  gx.clear(); gy.clear(); xt.clear(); yt.clear(); xs.clear(); ys.clear();
  for (int j = 1; j <= nte; ++j) { gx.push_back(ext.r.F[1]); gy.push_back(ext.t.x[j]); }
  pairs(gx, gy, xt, yt, xs, ys);
  double* dval = static_cast<double*>(A.get(sizeof(double) * size_t(nte) * nb * M));
  if (!dval || !green(A, g.geometry, N, M, g.G, 1, xt, yt, xs, ys, cosk, dval, 1, M, nullptr, 1, st)) {
    err = "out of device memory (DGF)";
    return false;
  }
  ExtArgs ea{};
  ea.nr = nre; ea.nt = nte; ea.nb = nb; ea.npairs = (nb + 1) / 2; ea.M = M;
  ea.four_pi_G = 4.0 * kPi * g.G;
  ea.aE_out = ext.aE[nre];
  ea.aS_lo = ext.aS[1];
  ea.aN_hi = ext.aN[nte];
  const double F1 = ext.r.F[1], F2 = ext.r.F[2];
  ea.cN = g.geometry == SPH ? 3.0 * F1 * F1 / (F2 * F2 * F2 - F1 * F1 * F1)
                            : 2.0 * F1 / (F2 * F2 - F1 * F1);
  ea.src_cell = up(A, src);
  ea.dV = up(A, dV);
  ea.P = up(A, ext.P);
  ea.gout = gout; ea.glo = glo; ea.ghi = ghi; ea.dval = dval;
  // batched solve in chunks of planes
  const long total = long(M) * ea.npairs;
  const size_t cells = size_t(nre) * nte;
  const size_t per_plane = cells * (2 * sizeof(double2) + 2 * sizeof(float2) * 4 / 3 + 16) + 4096;
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  long chunk = long(std::min<size_t>(size_t(total), std::max<size_t>(1, (freeb / 3) / per_plane)));
  chunk = std::min<long>(chunk, 16384);
  std::vector<int> modes(M), slot(chunk);
  for (int m = 0; m < M; ++m) modes[m] = m;
  for (long p = 0; p < chunk; ++p) slot[p] = int(p / ea.npairs);
  MGSolver mg;
  MGOptions o;
  o.precision = 1;
  o.max_cycles = 200;
  o.stagnation = 1;
  if (!mg.init(A, ext, true, modes, slot, int(chunk), o, err)) return false;
  double2* u = static_cast<double2*>(A.get(sizeof(double2) * cells * chunk));
  double2* f = static_cast<double2*>(A.get(sizeof(double2) * cells * chunk));
  if (!u || !f) { err = "out of device memory (DGF planes)"; return false; }
  for (long p0 = 0; p0 < total; p0 += chunk) {
    const int np = int(std::min<long>(chunk, total - p0));
    for (int p = 0; p < np; ++p) slot[p] = int((p0 + p) / ea.npairs);
    for (int p = np; p < chunk; ++p) slot[p] = 0;
    cudaMemcpyAsync(mg.d_slot, slot.data(), sizeof(int) * chunk, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(u, 0, sizeof(double2) * cells * chunk, st);
    cudaMemsetAsync(f, 0, sizeof(double2) * cells * chunk, st);
    launch_ext_rhs(ea, f, int(p0), np, st);
    mg.batch.max_planes = np;
    mg.max_planes = np;
    if (mg.eager_solve(f, u, 1e-13, st, err) != 0) return false;
    launch_ext_extract(ea, u, gt, int(p0), np, st);
  }
  cudaStreamSynchronize(st);
  if (mg.h_cont) cudaFreeHost(mg.h_cont);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { err = std::string("extended-domain DGF: ") + cudaGetErrorString(e); return false; }
  return true;
}

// Cells c_first..c_last of a law kept in the auxiliary windows: radial cells
// stop at r = 0, polar cells at the poles; a clipped face must be such a
// zero-area face.
static bool big_range(const Law& L, int kind, int n, long& c0, long& c1, std::string& err) {
  c0 = 1 - (kPad + 1);
  c1 = n + kPad + 1;
  if (kind == 0 || kind == 1) {
    while (L.face(c0 - 1) < -kTol) ++c0;
    if (c0 > 1 - (kPad + 1) && std::fabs(L.face(c0 - 1)) > kTol) {
      err = "auxiliary DGF window crosses r = 0 away from a cell face (use r_in = 0 or r_in >= 17 cells)";
      return false;
    }
  } else if (kind == 2) {
    while (L.face(c0 - 1) < -kTol) ++c0;
    while (L.face(c1) > kPi + kTol) --c1;
    if ((c0 > 1 - (kPad + 1) && std::fabs(L.face(c0 - 1)) > kTol) ||
        (c1 < n + kPad + 1 && std::fabs(L.face(c1) - kPi) > kTol)) {
      err = "auxiliary DGF window crosses a pole away from a cell face";
      return false;
    }
  }
  return true;
}

static bool build_aux(const PlaneGeo& g, const Law& rlaw, const Law& tlaw,
                      const std::vector<BPoint>& bp, double* gt, Arena& A, const double* cosk,
                      cudaStream_t st, std::string& err) {
  const int nr = g.r.n, nt = g.t.n, nb = int(bp.size()), N = g.n_phi, M = N / 2 + 1;
  long r0, r1, t0, t1;
  if (!big_range(rlaw, kind_r(g.geometry), nr, r0, r1, err)) return false;
  if (!big_range(tlaw, kind_t(g.geometry), nt, t0, t1, err)) return false;
  PlaneGeo big;
  big.geometry = g.geometry; big.n_phi = N; big.G = g.G;
  big.r = axis_from_law(kind_r(g.geometry), rlaw, r0, r1);
  big.t = axis_from_law(kind_t(g.geometry), tlaw, t0, t1);
  big.build();
  auto bi = [&](long c) { return int(c - r0 + 1); };   // original -> big index
  auto bj = [&](long c) { return int(c - t0 + 1); };
  // far field: closed form for every (t, s), scaled by dV_s; near pairs are
  // replaced by the window solutions below
  std::vector<double> px(nb), py(nb), dV(nb);
  std::vector<int> ti(nb), tj(nb);
  for (int s = 0; s < nb; ++s) {
    ti[s] = bi(bp[s].i);
    tj[s] = bj(bp[s].j);
    px[s] = big.r.x[ti[s]];
    py[s] = big.t.x[tj[s]];
    dV[s] = bp[s].dV;
  }
  double* d_dV = up(A, dV);
  {
    std::vector<double> xt, yt, xs, ys;
    xt.reserve(size_t(nb) * nb);
    for (int t = 0; t < nb; ++t)
      for (int s = 0; s < nb; ++s) {
        xt.push_back(px[t]); yt.push_back(py[t]); xs.push_back(px[s]); ys.push_back(py[s]);
      }
    if (!green(A, g.geometry, N, M, g.G, 0, xt, yt, xs, ys, cosk, gt, long(nb) * nb, 1, d_dV, nb, st)) {
      err = "out of device memory (DGF far field)";
      return false;
    }
  }
  // windows, ring points and targets
  const int ring_max = 4 * (2 * kPad + 1);
  std::vector<AuxWin> win(nb);
  std::vector<int> tlist;
  std::vector<double> xt, yt, xs, ys;
  xt.reserve(size_t(nb) * ring_max);
  int max_cells = 0;
  auto sin_face = [&](double th) {
    return (std::fabs(th) < kTol || std::fabs(th - kPi) < kTol) ? 0.0 : std::sin(th);
  };
  for (int s = 0; s < nb; ++s) {
    AuxWin w{};
    w.is = ti[s];
    w.js = tj[s];
    w.i0 = std::max(w.is - kPad, 1);
    w.i1 = std::min(w.is + kPad, big.r.n);
    w.j0 = std::max(w.js - kPad, 1);
    w.j1 = std::min(w.js + kPad, big.t.n);
    const int wr = w.i1 - w.i0 + 1, wt = w.j1 - w.j0 + 1;
    max_cells = std::max(max_cells, wr * wt);
    int k = 0;
    auto add = [&](double x, double y) {
      xt.push_back(x); yt.push_back(y); xs.push_back(px[s]); ys.push_back(py[s]);
      ++k;
    };
    w.ring_r = k;
    for (int j = w.j0; j <= w.j1; ++j) add(big.r.x[w.i1 + 1], big.t.x[j]);
    w.ring_l = -1;
    if (big.r.F[w.i0] > kTol) {   // inner face of the window has area
      w.ring_l = k;
      for (int j = w.j0; j <= w.j1; ++j) add(big.r.x[w.i0 - 1], big.t.x[j]);
    }
    const bool lo = g.geometry == CYL || sin_face(big.t.F[w.j0]) != 0.0;
    const bool hi = g.geometry == CYL || sin_face(big.t.F[w.j1 + 1]) != 0.0;
    w.ring_b = -1;
    if (lo) {
      w.ring_b = k;
      for (int i = w.i0; i <= w.i1; ++i) add(big.r.x[i], big.t.x[w.j0 - 1]);
    }
    w.ring_t = -1;
    if (hi) {
      w.ring_t = k;
      for (int i = w.i0; i <= w.i1; ++i) add(big.r.x[i], big.t.x[w.j1 + 1]);
    }
    while (k < ring_max) add(px[s] + 1.0, py[s]);   // padding, never read
    w.tfirst = int(tlist.size());
    for (int t = 0; t < nb; ++t)
      if (ti[t] >= w.i0 && ti[t] <= w.i1 && tj[t] >= w.j0 && tj[t] <= w.j1) tlist.push_back(t);
    w.ntarget = int(tlist.size()) - w.tfirst;
    win[s] = w;
  }
  double* ring = static_cast<double*>(A.get(sizeof(double) * size_t(nb) * ring_max * M));
  if (!ring || !green(A, g.geometry, N, M, g.G, 0, xt, yt, xs, ys, cosk, ring, 1, M, nullptr, 1, st)) {
    err = "out of device memory (DGF ring)";
    return false;
  }
  std::vector<double> rtab(size_t(RT_N) * (big.r.n + 2), 0.0), ttab(size_t(TT_N) * (big.t.n + 2), 0.0);
  for (int i = 0; i < big.r.n + 2; ++i) {
    const int NR = big.r.n + 2;
    rtab[RT_AE * NR + i] = big.aE[i];
    rtab[RT_AW * NR + i] = big.aW[i];
    rtab[RT_P * NR + i] = big.P[i];
    rtab[RT_Q * NR + i] = big.Q[i];
    rtab[RT_V * NR + i] = big.vr[i];
  }
  for (int j = 0; j < big.t.n + 2; ++j) {
    const int NT = big.t.n + 2;
    ttab[TT_AN * NT + j] = big.aN[j];
    ttab[TT_AS * NT + j] = big.aS[j];
    ttab[TT_T * NT + j] = big.T[j];
    ttab[TT_V * NT + j] = big.vt[j];
  }
  std::vector<double> s2(M);
  for (int m = 0; m < M; ++m) s2[m] = g.s2(m);
  AuxArgs a{};
  a.nb = nb; a.M = M; a.nr_big = big.r.n; a.nt_big = big.t.n; a.ring_max = ring_max;
  a.max_iter = 20000;
  a.four_pi_G = 4.0 * kPi * g.G;
  a.rt = up(A, rtab); a.tt = up(A, ttab); a.s2 = up(A, s2); a.dV = d_dV;
  a.win = up(A, win); a.ring = ring; a.tlist = up(A, tlist);
  a.tcell_i = up(A, ti); a.tcell_j = up(A, tj);
  a.gt = gt;
  a.fail = static_cast<int*>(A.get(sizeof(int)));
  if (!a.fail || !a.win || !a.tlist) { err = "out of device memory (DGF windows)"; return false; }
  cudaMemsetAsync(a.fail, 0, sizeof(int), st);
  launch_aux_cg(a, M * nb, max_cells, st);
  int fails = 0;
  cudaMemcpyAsync(&fails, a.fail, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (fails) { err = "auxiliary DGF window solves did not converge"; return false; }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { err = std::string("auxiliary DGF: ") + cudaGetErrorString(e); return false; }
  return true;
}

bool build_dgf(const PlaneGeo& g, const Law& rlaw, const Law& tlaw, const std::vector<BPoint>& bp,
               double* gt, Arena& A, cudaStream_t st, int& construction, std::string& err) {
  const int N = g.n_phi;
  std::vector<double> ck(N);
  for (int k = 0; k < N; ++k) ck[k] = std::cos(2.0 * kPi * double(k) / double(N));
  const double* cosk = up(A, ck);
  if (!cosk) { err = "out of device memory"; return false; }
  bool ok;
  // construction on entry: 0 the paper's rule, 1 auxiliary windows, 2 the
  // extended domain; on return 1 for the extended domain, 0 for windows
  const bool ext = construction == 2 || (construction == 0 && uses_extended(rlaw, g.r.n));
  if (ext) {
    construction = 1;
    ok = build_extended(g, rlaw, tlaw, bp, gt, A, cosk, st, err);
  } else {
    construction = 0;
    ok = build_aux(g, rlaw, tlaw, bp, gt, A, cosk, st, err);
  }
  if (ok && cudaStreamSynchronize(st) != cudaSuccess) {
    err = std::string("DGF construction: ") + cudaGetErrorString(cudaGetLastError());
    ok = false;
  }
  return ok;
}

}  // namespace ps
