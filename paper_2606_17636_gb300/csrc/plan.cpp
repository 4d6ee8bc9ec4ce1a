// Host-side plan: grid geometry (Sec. 2.1.1, 2.1.2), multigrid level tables
// (Sec. 3.1), per-line relaxation parameters (App. A) and coarsest-level
// inverses (Sec. 3.3, solved exactly).
#include "plan.h"

#include <algorithm>
#include <cstdio>

namespace ps {

static const double kPoleTol = 1e-12;
static const double kPi = 3.14159265358979323846;

void Axis::centres() {
  x.assign(n + 2, 0.0);
  for (int c = 0; c < n + 2; ++c) {
    double a = F[c], b = F[c + 1];
    switch (kind) {
      case 0:  // r, spherical: volume-weighted centroid, Eq. cell_centers_sph
        x[c] = 0.75 * (b * b * b * b - a * a * a * a) / (b * b * b - a * a * a);
        break;
      case 1:  // R, cylindrical
        x[c] = (2.0 / 3.0) * (b * b * b - a * a * a) / (b * b - a * a);
        break;
      case 2:  // theta
        x[c] = (std::sin(b) - std::sin(a) + a * std::cos(a) - b * std::cos(b)) /
               (std::cos(a) - std::cos(b));
        break;
      default:
        x[c] = 0.5 * (a + b);
    }
  }
}

Axis axis_from_law(int kind, const Law& L, long c_first, long c_last) {
  Axis a;
  a.kind = kind;
  a.spacing = L.spacing;
  a.n = int(c_last - c_first + 1);
  a.F.resize(a.n + 3);
  for (int q = 0; q < a.n + 3; ++q) a.F[q] = L.face(c_first - 2 + q);
  a.centres();
  return a;
}

Axis coarse_axis(const Axis& f) {
  Axis c;
  c.kind = f.kind;
  c.spacing = f.spacing;
  c.n = f.n / 2;
  c.F.resize(c.n + 3);
  for (int q = 0; q <= c.n; ++q) c.F[q + 1] = f.F[1 + 2 * q];
  if (f.spacing == LOGS && (f.kind == 0 || f.kind == 1)) {
    double qr = c.F[2] / c.F[1];
    c.F[0] = c.F[1] / qr;
    c.F[c.n + 2] = c.F[c.n + 1] * qr;
  } else {
    double d = c.F[2] - c.F[1];
    c.F[0] = c.F[1] - d;
    c.F[c.n + 2] = c.F[c.n + 1] + d;
  }
  c.centres();
  return c;
}

static double sin_face(double th) {
  if (std::fabs(th) < kPoleTol || std::fabs(th - kPi) < kPoleTol) return 0.0;
  return std::sin(th);
}

bool PlaneGeo::has_inner() const { return r.F[1] > 0.0; }
bool PlaneGeo::has_lower() const { return geometry == CYL || sin_face(t.F[1]) != 0.0; }
bool PlaneGeo::has_upper() const { return geometry == CYL || sin_face(t.F[t.n + 1]) != 0.0; }

double PlaneGeo::s2(int m) const {
  double s = std::sin(double(m) * kPi / double(n_phi)) / (kPi / double(n_phi));
  return s * s;
}

void PlaneGeo::build() {
  const int nr = r.n, nt = t.n;
  aE.assign(nr + 2, 0.0); aW.assign(nr + 2, 0.0);
  P.assign(nr + 2, 1.0); Q.assign(nr + 2, 0.0); vr.assign(nr + 2, 0.0);
  aN.assign(nt + 2, 0.0); aS.assign(nt + 2, 0.0);
  T.assign(nt + 2, 1.0); vt.assign(nt + 2, 0.0);
  for (int c = 0; c < nr + 2; ++c) {
    double lo = r.F[c], hi = r.F[c + 1];
    if (geometry == SPH) {  // nabla^2_r and R_i (Sec. 2.1.1)
      double v3 = hi * hi * hi - lo * lo * lo;
      if (c + 1 < nr + 2) aE[c] = 3.0 * hi * hi / v3 / (r.x[c + 1] - r.x[c]);
      if (c > 0) aW[c] = 3.0 * lo * lo / v3 / (r.x[c] - r.x[c - 1]);
      P[c] = Q[c] = 1.5 / r.x[c] * (hi * hi - lo * lo) / v3;
      vr[c] = v3 / 3.0;
    } else {  // nabla^2_R and W_i (Sec. 2.1.2)
      double v2 = hi * hi - lo * lo;
      if (c + 1 < nr + 2) aE[c] = 2.0 * hi / v2 / (r.x[c + 1] - r.x[c]);
      if (c > 0) aW[c] = 2.0 * lo / v2 / (r.x[c] - r.x[c - 1]);
      P[c] = 1.0;
      Q[c] = 2.0 / (r.x[c] * (hi + lo));
      vr[c] = v2 / 2.0;
    }
  }
  for (int c = 0; c < nt + 2; ++c) {
    double lo = t.F[c], hi = t.F[c + 1];
    if (geometry == SPH) {  // nabla^2_theta / R_i and T_j
      double vc = std::cos(lo) - std::cos(hi);
      if (c + 1 < nt + 2) aN[c] = sin_face(hi) / vc / (t.x[c + 1] - t.x[c]);
      if (c > 0) aS[c] = sin_face(lo) / vc / (t.x[c] - t.x[c - 1]);
      T[c] = (hi - lo) / (std::sin(t.x[c]) * vc);
      vt[c] = vc;
    } else {  // nabla^2_z
      double dz = hi - lo;
      if (c + 1 < nt + 2) aN[c] = 1.0 / dz / (t.x[c + 1] - t.x[c]);
      if (c > 0) aS[c] = 1.0 / dz / (t.x[c] - t.x[c - 1]);
      T[c] = 1.0;
      vt[c] = dz;
    }
  }
}

static bool invert(std::vector<double>& A, int n) {  // Gauss-Jordan, partial pivoting
  std::vector<double> I(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) I[size_t(i) * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int rr = col + 1; rr < n; ++rr)
      if (std::fabs(A[size_t(rr) * n + col]) > std::fabs(A[size_t(piv) * n + col])) piv = rr;
    if (A[size_t(piv) * n + col] == 0.0) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(A[size_t(piv) * n + k], A[size_t(col) * n + k]);
        std::swap(I[size_t(piv) * n + k], I[size_t(col) * n + k]);
      }
    double d = 1.0 / A[size_t(col) * n + col];
    for (int k = 0; k < n; ++k) { A[size_t(col) * n + k] *= d; I[size_t(col) * n + k] *= d; }
    for (int rr = 0; rr < n; ++rr) {
      if (rr == col) continue;
      double fct = A[size_t(rr) * n + col];
      if (fct == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[size_t(rr) * n + k] -= fct * A[size_t(col) * n + k];
        I[size_t(rr) * n + k] -= fct * I[size_t(col) * n + k];
      }
    }
  }
  A.swap(I);
  return true;
}

// Eigen-decomposition of a symmetric n x n matrix S (row-major, destroyed)
// by cyclic Jacobi rotations: S = U diag(lam) U^T, U orthogonal (columns).
static void jacobi_eig(std::vector<double>& S, int n, std::vector<double>& U,
                       std::vector<double>& lam) {
  U.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) U[size_t(i) * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < n; ++p) {
      dia += S[size_t(p) * n + p] * S[size_t(p) * n + p];
      for (int q = p + 1; q < n; ++q) off += S[size_t(p) * n + q] * S[size_t(p) * n + q];
    }
    if (off <= 1e-32 * dia) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double b = S[size_t(p) * n + q];
        if (std::fabs(b) < 1e-300) continue;
        // rotation by phi with cot(2 phi) = (S_qq - S_pp) / (2 S_pq) zeroes S_pq
        const double th = (S[size_t(q) * n + q] - S[size_t(p) * n + p]) / (2.0 * b);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double skp = S[size_t(k) * n + p], skq = S[size_t(k) * n + q];
          S[size_t(k) * n + p] = c * skp - sn * skq;
          S[size_t(k) * n + q] = sn * skp + c * skq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double spk = S[size_t(p) * n + k], sqk = S[size_t(q) * n + k];
          S[size_t(p) * n + k] = c * spk - sn * sqk;
          S[size_t(q) * n + k] = sn * spk + c * sqk;
        }
        for (int k = 0; k < n; ++k) {
          const double ukp = U[size_t(k) * n + p], ukq = U[size_t(k) * n + q];
          U[size_t(k) * n + p] = c * ukp - sn * ukq;
          U[size_t(k) * n + q] = sn * ukp + c * ukq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = S[size_t(i) * n + i];
}

// Mirror symmetry j <-> n-1-j of the symmetrised polar operator S and its
// weights w (relative 1e-12: the weights come from a running product over
// the polar faces).
static bool mirror_symmetric(const std::vector<double>& S, const std::vector<double>& w, int n) {
  auto near = [](double x, double y) { return std::fabs(x - y) <= 1e-12 * std::fmax(std::fabs(x), std::fabs(y)); };
  if (n % 2) return false;
  for (int j = 0; j < n; ++j) {
    if (!near(S[size_t(j) * n + j], S[size_t(n - 1 - j) * n + (n - 1 - j)])) return false;
    if (!near(w[j + 1], w[n - j])) return false;
    if (j + 1 < n && !near(S[size_t(j) * n + j + 1], S[size_t(n - 2 - j) * n + (n - 1 - j)])) return false;
  }
  return true;
}

// Separable factors of L_m on plane g (see Hierarchy::coarse_sep), written
// to out; sym selects the mirror-symmetric layout (the polar eigenvectors
// taken in the even / odd subspaces).  Returns false when the operator does
// not split this way (or is not mirror-symmetric, for sym) or the factors
// fail the residual check; *resid receives the check's relative residual.
static bool separable_factors(const PlaneGeo& g, int m, double* out, bool sym, double* resid) {
  const int nr = g.r.n, nt = g.t.n, h = nt / 2;
  const double s2 = g.s2(m);
  const bool sph = g.geometry == SPH;
  std::vector<double> dr(nr + 1), dt(nt + 1);
  for (int i = 1; i <= nr; ++i) dr[i] = -(g.aE[i] + g.aW[i]) - (sph ? 0.0 : s2 * g.Q[i] * g.T[1]);
  for (int j = 1; j <= nt; ++j) dt[j] = -(g.aN[j] + g.aS[j]) - (sph ? s2 * g.T[j] : 0.0);
  for (int j = 1; j <= nt; ++j)
    for (int i = 1; i <= nr; ++i) {
      const double d = g.diag(m, i, j), sp = dr[i] + g.P[i] * dt[j];
      if (std::fabs(d - sp) > 1e-12 * std::fabs(d)) return false;   // not separable
      if (!sph && (g.P[i] != 1.0 || g.T[j] != 1.0)) return false;
    }
  // W-symmetrised polar operator: off-diagonal sqrt(aN_j aS_{j+1}), weights w
  std::vector<double> S(size_t(nt) * nt, 0.0), w(nt + 1, 1.0), U, lam;
  for (int j = 1; j <= nt; ++j) S[size_t(j - 1) * nt + (j - 1)] = dt[j];
  for (int j = 1; j < nt; ++j) {
    if (!(g.aN[j] > 0.0 && g.aS[j + 1] > 0.0)) return false;
    const double e = std::sqrt(g.aN[j] * g.aS[j + 1]);
    S[size_t(j - 1) * nt + j] = S[size_t(j) * nt + (j - 1)] = e;
    w[j + 1] = w[j] * g.aN[j] / g.aS[j + 1];
  }
  if (sym) {
    // even / odd subspaces, basis (delta_j +- delta_{n-1-j}) / sqrt 2, j < h:
    // the top-left block of S with the middle coupling added (even) or
    // subtracted (odd); eigenvectors k < h even, k >= h odd
    if (!mirror_symmetric(S, w, nt)) return false;
    const double emid = S[size_t(h - 1) * nt + h];
    U.assign(size_t(nt) * nt, 0.0);
    lam.assign(nt, 0.0);
    for (int par = 0; par < 2; ++par) {
      std::vector<double> Sh(size_t(h) * h), Uh, lh;
      for (int x = 0; x < h; ++x)
        for (int y = 0; y < h; ++y) Sh[size_t(x) * h + y] = S[size_t(x) * nt + y];
      Sh[size_t(h - 1) * h + (h - 1)] += par ? -emid : emid;
      jacobi_eig(Sh, h, Uh, lh);
      for (int kk = 0; kk < h; ++kk) {
        const int k = par * h + kk;
        lam[k] = lh[kk];
        for (int j = 0; j < h; ++j) {
          const double v = Uh[size_t(j) * h + kk] * std::sqrt(0.5);
          U[size_t(j) * nt + k] = v;
          U[size_t(nt - 1 - j) * nt + k] = par ? -v : v;
        }
      }
    }
  } else {
    jacobi_eig(S, nt, U, lam);
  }
  // general layout: V [nt][nt], V^-1 [nt][nt]; mirror-symmetric layout: the
  // rows j < h of V [h][nt] and the columns j < h of V^-1 [nt][h]
  const int vr = sym ? h : nt;
  double* V = out;
  double* Vi = V + size_t(vr) * nt;
  double* invd = Vi + size_t(nt) * vr;
  double* cp = invd + size_t(nt) * nr;
  double* lid = cp + size_t(nt) * nr;
  std::vector<double> low(nr);
  for (int j = 0; j < vr; ++j)
    for (int k = 0; k < nt; ++k) {
      V[size_t(j) * nt + k] = U[size_t(j) * nt + k] / std::sqrt(w[j + 1]);
      Vi[size_t(k) * vr + j] = U[size_t(j) * nt + k] * std::sqrt(w[j + 1]);
    }
  for (int i = 1; i <= nr; ++i) low[i - 1] = i > 1 ? g.aW[i] : 0.0;
  for (int k = 0; k < nt; ++k) {
    double cprev = 0.0;
    for (int i = 1; i <= nr; ++i) {
      const double up = i < nr ? g.aE[i] : 0.0;
      const double den = dr[i] + lam[k] * g.P[i] - low[i - 1] * cprev;
      if (den == 0.0) return false;
      invd[size_t(k) * nr + i - 1] = 1.0 / den;
      cprev = up / den;
      cp[size_t(k) * nr + i - 1] = cprev;
      lid[size_t(k) * nr + i - 1] = low[i - 1] / den;
    }
  }
  // residual check of the factors on a fixed test vector, in the kernel's
  // form: z' = invd .* (V^-1 f), dp_i = z'_i - lid_i dp_{i-1}, back
  // substitution, x = V z (mirror-symmetric: sums and differences of the
  // mirrored rows in, even and odd parts out)
  std::vector<double> b(size_t(nr) * nt), z(size_t(nr) * nt), x(size_t(nr) * nt), fs(size_t(nr) * nt);
  for (size_t q = 0; q < b.size(); ++q) b[q] = std::sin(0.37 * double(q) + 1.0);
  if (sym) {
    for (int j = 0; j < h; ++j)
      for (int i = 0; i < nr; ++i) {
        const double u = b[size_t(j) * nr + i], v = b[size_t(nt - 1 - j) * nr + i];
        fs[size_t(j) * nr + i] = u + v;
        fs[size_t(h + j) * nr + i] = u - v;
      }
  } else {
    fs = b;
  }
  for (int k = 0; k < nt; ++k)
    for (int i = 0; i < nr; ++i) {
      const double* src = fs.data() + (sym && k >= h ? size_t(h) * nr : 0) + i;
      double a = 0.0;
      for (int j = 0; j < vr; ++j) a += Vi[size_t(k) * vr + j] * src[size_t(j) * nr];
      z[size_t(k) * nr + i] = a * invd[size_t(k) * nr + i];
    }
  for (int k = 0; k < nt; ++k) {
    double* zz = z.data() + size_t(k) * nr;
    double dp = zz[0];
    for (int i = 1; i < nr; ++i) { dp = zz[i] - lid[size_t(k) * nr + i] * dp; zz[i] = dp; }
    double xv = zz[nr - 1];
    for (int i = nr - 2; i >= 0; --i) { xv = zz[i] - cp[size_t(k) * nr + i] * xv; zz[i] = xv; }
  }
  for (int j = 0; j < vr; ++j)
    for (int i = 0; i < nr; ++i) {
      double ev = 0.0, od = 0.0;
      for (int k = 0; k < nt; ++k) {
        const double t = V[size_t(j) * nt + k] * z[size_t(k) * nr + i];
        if (sym && k >= h) od += t; else ev += t;
      }
      x[size_t(j) * nr + i] = ev + od;
      if (sym) x[size_t(nt - 1 - j) * nr + i] = ev - od;
    }
  double rn = 0.0, bn = 0.0;
  for (int j = 1; j <= nt; ++j)
    for (int i = 1; i <= nr; ++i) {
      const size_t q = size_t(j - 1) * nr + (i - 1);
      double ax = g.diag(m, i, j) * x[q];
      if (i < nr) ax += g.aE[i] * x[q + 1];
      if (i > 1) ax += g.aW[i] * x[q - 1];
      if (j < nt) ax += g.P[i] * g.aN[j] * x[q + nr];
      if (j > 1) ax += g.P[i] * g.aS[j] * x[q - nr];
      rn += (ax - b[q]) * (ax - b[q]);
      bn += b[q] * b[q];
    }
  *resid = std::sqrt(rn / bn);
  return rn <= 1e-20 * bn;   // 1e-10 relative: a sound factorisation (rounding only)
}

bool plan_hierarchy(const PlaneGeo& fine, bool neumann, const std::vector<int>& modes,
                    int coarsest_size, int precision, Hierarchy& H, std::string& err) {
  const bool try_large = coarsest_size == 2 || (coarsest_size == 0 && precision == 1);
  if (try_large) {
    if (!build_hierarchy(fine, neumann, modes, H, err, 32, 2048, true)) return false;
    const bool keep = H.sep_stride > 0 && (coarsest_size == 2 || H.lv.size() >= 2);
    if (keep) {
      H.large = 1;
      return true;
    }
  }
  H = Hierarchy();
  return build_hierarchy(fine, neumann, modes, H, err);
}

bool build_hierarchy(const PlaneGeo& fine, bool neumann, const std::vector<int>& modes,
                     Hierarchy& H, std::string& err, int min_side, int max_cells, bool sep_only) {
  H.lv.clear();
  PlaneGeo g = fine;
  g.build();
  while (true) {
    LevelHost L;
    L.g = g;
    if (neumann) L.g.aW[1] = 0.0;
    H.lv.push_back(L);
    // coarsen while the short side exceeds min_side cells, or exceeds 4 cells
    // while the plane has more than max_cells (the coarsest level is solved
    // directly)
    const int mn = std::min(g.r.n, g.t.n);
    if (!(mn > min_side || (mn > 4 && g.r.n * g.t.n > max_cells))) break;
    if (g.r.n % 2 || g.t.n % 2) { err = "grid sizes must be powers of two"; return false; }
    PlaneGeo c;
    c.geometry = g.geometry; c.n_phi = g.n_phi; c.G = g.G;
    c.r = coarse_axis(g.r);
    c.t = coarse_axis(g.t);
    c.build();
    g = c;
  }
  const int nlev = int(H.lv.size());
  const int M = int(modes.size());
  for (int l = 0; l < nlev; ++l) {
    LevelHost& L = H.lv[l];
    const PlaneGeo& p = L.g;
    const int nr = p.r.n, nt = p.t.n, NR = nr + 2, NT = nt + 2;
    L.rtab.assign(size_t(RT_N) * NR, 0.0);
    L.ttab.assign(size_t(TT_N) * NT, 0.0);
    for (int i = 0; i < NR; ++i) {
      L.rtab[RT_AE * NR + i] = p.aE[i];
      L.rtab[RT_AW * NR + i] = p.aW[i];
      L.rtab[RT_P * NR + i] = p.P[i];
      L.rtab[RT_Q * NR + i] = p.Q[i];
      L.rtab[RT_DR * NR + i] = -(p.aE[i] + p.aW[i]);
      L.rtab[RT_V * NR + i] = p.vr[i];
    }
    for (int j = 0; j < NT; ++j) {
      L.ttab[TT_AN * NT + j] = p.aN[j];
      L.ttab[TT_AS * NT + j] = p.aS[j];
      L.ttab[TT_T * NT + j] = p.T[j];
      L.ttab[TT_DT * NT + j] = -(p.aN[j] + p.aS[j]);
      L.ttab[TT_V * NT + j] = p.vt[j];
    }
    // restriction (Sec. 3.1): weight = overlap area of the fine cell in the
    // (r^2, theta) or (R, z) plane, normalised over the four children
    if (l + 1 < nlev) {
      auto ra = [&](int i) {
        double a = p.r.F[i], b = p.r.F[i + 1];
        return p.geometry == SPH ? std::fabs(b * b - a * a) : std::fabs(b - a);
      };
      auto tb = [&](int j) { return std::fabs(p.t.F[j + 1] - p.t.F[j]); };
      for (int i = 1; i <= nr; ++i) {
        int s = (i % 2) ? i + 1 : i - 1;
        L.rtab[RT_RW * NR + i] = ra(i) / (ra(i) + ra(s));
      }
      for (int j = 1; j <= nt; ++j) {
        int s = (j % 2) ? j + 1 : j - 1;
        L.ttab[TT_RW * NT + j] = tb(j) / (tb(j) + tb(s));
      }
      // prolongation weights: bilinear in (r^2, theta) or (R, z) between the
      // two coarse centres that bracket each fine centre
      const PlaneGeo& c = H.lv[l + 1].g;
      auto xi = [&](const Axis& a, int k) { return p.geometry == SPH ? a.x[k] * a.x[k] : a.x[k]; };
      for (int i = 1; i <= nr; ++i) {
        int I1 = (i % 2) ? (i + 1) / 2 - 1 : i / 2, I2 = I1 + 1;
        double den = std::fabs(xi(c.r, I2) - xi(c.r, I1));
        L.rtab[RT_P1 * NR + i] = std::fabs(xi(c.r, I2) - xi(p.r, i)) / den;
        L.rtab[RT_P2 * NR + i] = std::fabs(xi(c.r, I1) - xi(p.r, i)) / den;
      }
      for (int j = 1; j <= nt; ++j) {
        int J1 = (j % 2) ? (j + 1) / 2 - 1 : j / 2, J2 = J1 + 1;
        double den = std::fabs(c.t.x[J2] - c.t.x[J1]);
        L.ttab[TT_P1 * NT + j] = std::fabs(c.t.x[J2] - p.t.x[j]) / den;
        L.ttab[TT_P2 * NT + j] = std::fabs(c.t.x[J1] - p.t.x[j]) / den;
      }
    }
    // coarse-ghost rules used when this level is prolongated from
    if (neumann) L.gL = GH_EVEN;
    else if (!p.has_inner()) L.gL = (p.geometry == CYL) ? GH_PARITY : GH_EVEN;
    else L.gL = GH_ZERO;
    L.gR = GH_ZERO;
    L.gB = p.has_lower() ? GH_ZERO : GH_PARITY;
    L.gT = p.has_upper() ? GH_ZERO : GH_PARITY;
    // App. A relaxation parameters per line and mode: for a line of N cells
    // with neighbour couplings a_q, c_q and diagonal b_q,
    //   mu_1 = sum_q (a_q + c_q) cos(pi (x_q - x_{q-1}) / L) w_q / sum_q b_q w_q,
    //   w_q = sin^2(pi (x_q - x_0) / L), L = x_{N+1} - x_0,
    //   omega = 2 / (1 + sqrt(1 - mu_1^2)).
    // The weights and the off-diagonal sums do not depend on the mode, and
    // the diagonal is d0 - s_m^2 Q T with d0 its m = 0 value, so each line's
    // sums over the mode-independent parts are formed once and every mode
    // then costs O(1) per line.
    L.om_r.assign(size_t(M) * nt, 1.0);
    L.om_t.assign(size_t(M) * nr, 1.0);
    {
      auto weights = [](const std::vector<double>& x, int N, std::vector<double>& w,
                        std::vector<double>& c) {
        const double len = x[N + 1] - x[0];
        w.assign(N + 1, 0.0);
        c.assign(N + 1, 0.0);
        for (int q = 1; q <= N; ++q) {
          const double sn = std::sin(kPi * (x[q] - x[0]) / len);
          w[q] = sn * sn;
          c[q] = std::cos(kPi * (x[q] - x[q - 1]) / len);
        }
      };
      auto omega = [](double num, double den) {
        const double rho = std::min(std::fabs(num / den), 1.0);
        return 2.0 / (1.0 + std::sqrt(1.0 - rho * rho));
      };
      std::vector<double> wr, cr, wt, ct;
      weights(p.r.x, nr, wr, cr);
      weights(p.t.x, nt, wt, ct);
      // radial line j: num = sum_i (aW + aE) c_i w_i; den = D0r_j - s2 T_j sum_i Q_i w_i
      double numr = 0.0, qr = 0.0;
      for (int i = 1; i <= nr; ++i) {
        numr += (p.aW[i] + p.aE[i]) * cr[i] * wr[i];
        qr += p.Q[i] * wr[i];
      }
      std::vector<double> d0r(nt + 1, 0.0), numt(nr + 1, 0.0), d0t(nr + 1, 0.0);
      for (int j = 1; j <= nt; ++j)
        for (int i = 1; i <= nr; ++i) d0r[j] += p.diag(0, i, j) * wr[i];
      // polar line i: num = P_i sum_j (aS + aN) c_j w_j; den = D0t_i - s2 Q_i sum_j T_j w_j
      double st = 0.0, qt = 0.0;
      for (int j = 1; j <= nt; ++j) {
        st += (p.aS[j] + p.aN[j]) * ct[j] * wt[j];
        qt += p.T[j] * wt[j];
      }
      for (int i = 1; i <= nr; ++i) {
        numt[i] = p.P[i] * st;
        for (int j = 1; j <= nt; ++j) d0t[i] += p.diag(0, i, j) * wt[j];
      }
      for (int k = 0; k < M; ++k) {
        const double s2 = p.s2(modes[k]);
        for (int j = 1; j <= nt; ++j)
          L.om_r[size_t(k) * nt + j - 1] = omega(numr, d0r[j] - s2 * p.T[j] * qr);
        for (int i = 1; i <= nr; ++i)
          L.om_t[size_t(k) * nr + i - 1] = omega(numt[i], d0t[i] - s2 * p.Q[i] * qt);
      }
    }
  }
  // coarsest level: dense inverse of L_m (zero ghosts) per mode
  const LevelHost& C = H.lv.back();
  const int nr = C.g.r.n, nt = C.g.t.n, nc = nr * nt;
  H.nc = nc;
  if (nt <= 64) {
    // the mirror-symmetric layout first (half the transform work), else general
    for (int sym = 1; sym >= 0; --sym) {
      if (sym && nt % 2) continue;
      H.sep_stride = ((sym ? 1 : 2) * nt * nt + 3 * nt * nr + 1) / 2 * 2;
      H.coarse_sep.assign(size_t(M) * H.sep_stride, 0.0);
      bool ok = true;
      double worst = 0.0;
      for (int k = 0; k < M && ok; ++k) {
        double res = 0.0;
        ok = separable_factors(C.g, modes[k], H.coarse_sep.data() + size_t(k) * H.sep_stride, sym != 0,
                               &res);
        worst = std::fmax(worst, res);
      }
      if (ok) {
        H.sep_sym = sym;
        H.sep_check = worst;
        return true;
      }
    }
    H.coarse_sep.clear();
    H.sep_stride = 0;
    H.sep_sym = 0;
  }
  if (sep_only) return true;   // the caller takes another rule
  const bool blocks = nr <= 64;
  H.blk_n = blocks ? nr : 0;
  H.blk_nt = blocks ? nt : 0;
  const size_t bstride = size_t(nt) * nr * (nr + 2);
  if (blocks) H.coarse_blk.assign(size_t(M) * bstride, 0.0);
  else H.coarse_inv.assign(size_t(M) * nc * nc, 0.0);
  std::vector<double> A(size_t(nc) * nc), S(size_t(nr) * nr);
  for (int k = 0; k < M; ++k) {
    std::fill(A.begin(), A.end(), 0.0);
    int m = modes[k];
    for (int j = 1; j <= nt; ++j)
      for (int i = 1; i <= nr; ++i) {
        int row = (j - 1) * nr + (i - 1);
        A[size_t(row) * nc + row] = C.g.diag(m, i, j);
        if (i < nr) A[size_t(row) * nc + row + 1] = C.g.aE[i];
        if (i > 1) A[size_t(row) * nc + row - 1] = C.g.aW[i];
        if (j < nt) A[size_t(row) * nc + row + nr] = C.g.P[i] * C.g.aN[j];
        if (j > 1) A[size_t(row) * nc + row - nr] = C.g.P[i] * C.g.aS[j];
      }
    if (!blocks) {
      if (!invert(A, nc)) { err = "singular coarsest-level operator"; return false; }
      std::copy(A.begin(), A.end(), H.coarse_inv.begin() + size_t(k) * nc * nc);
      continue;
    }
    double* out = H.coarse_blk.data() + size_t(k) * bstride;
    double* bsub = out + size_t(nt) * nr * nr;
    double* csup = bsub + size_t(nt) * nr;
    auto a = [&](int J, int r, int J2, int r2) { return A[size_t(J * nr + r) * nc + J2 * nr + r2]; };
    for (int J = 0; J < nt; ++J) {
      for (int r = 0; r < nr; ++r) {
        bsub[J * nr + r] = J > 0 ? a(J, r, J - 1, r) : 0.0;
        csup[J * nr + r] = J + 1 < nt ? a(J, r, J + 1, r) : 0.0;
      }
      for (int r = 0; r < nr; ++r)
        for (int q = 0; q < nr; ++q) {
          double v = a(J, r, J, q);
          if (J > 0)
            v -= bsub[J * nr + r] * out[size_t(J - 1) * nr * nr + r * nr + q] * csup[(J - 1) * nr + q];
          S[size_t(r) * nr + q] = v;
        }
      if (!invert(S, nr)) { err = "singular coarsest-level operator"; return false; }
      std::copy(S.begin(), S.end(), out + size_t(J) * nr * nr);
    }
  }
  return true;
}

std::vector<BPoint> boundary_points(const PlaneGeo& g) {
  std::vector<BPoint> out;
  const int nr = g.r.n, nt = g.t.n;
  const double dphi = 2.0 * kPi / g.n_phi;
  const double inv4piG = 1.0 / (4.0 * kPi * g.G);
  auto dv = [&](int i, int j) { return g.vr[i] * g.vt[j] * dphi; };
  if (g.has_inner())
    for (int j = 1; j <= nt; ++j)
      out.push_back({'L', 0, j, 1, j, g.aE[0] * inv4piG, g.aW[1], dv(0, j)});
  for (int j = 1; j <= nt; ++j)
    out.push_back({'R', nr + 1, j, nr, j, g.aW[nr + 1] * inv4piG, g.aE[nr], dv(nr + 1, j)});
  if (g.has_lower())
    for (int i = 1; i <= nr; ++i)
      out.push_back({'B', i, 0, i, 1, g.P[i] * g.aN[0] * inv4piG, g.P[i] * g.aS[1], dv(i, 0)});
  if (g.has_upper())
    for (int i = 1; i <= nr; ++i)
      out.push_back({'T', i, nt + 1, i, nt, g.P[i] * g.aS[nt + 1] * inv4piG, g.P[i] * g.aN[nt],
                     dv(i, nt + 1)});
  return out;
}

}  // namespace ps
