// Host-side plan of a solver: grid geometry, multigrid level tables, per-line
// relaxation parameters, coarsest-level inverses and the boundary-point list.
// Everything here runs once in psolve_create; nothing here is on the solve path.
#pragma once
#include <cmath>
#include <string>
#include <vector>

namespace ps {

enum { SPH = 0, CYL = 1 };
enum { UNI = 0, LOGS = 1 };
enum { GH_ZERO = 0, GH_PARITY = 1, GH_EVEN = 2 };

// radial / polar table ids inside a level's packed table block
enum { RT_AE = 0, RT_AW, RT_P, RT_Q, RT_DR, RT_V, RT_RW, RT_P1, RT_P2, RT_N };
enum { TT_AN = 0, TT_AS, TT_T, TT_DT, TT_V, TT_RW, TT_P1, TT_P2, TT_N };

// Grid law of one axis: face k sits at lo + k (hi-lo)/n (uniform) or
// lo (hi/lo)^(k/n) (log).  Cell c spans faces c-1 .. c (cells 1..n inside).
struct Law {
  double lo = 0, hi = 1;
  int n = 1;
  int spacing = UNI;
  double face(long k) const {
    if (spacing == LOGS) return lo * std::pow(hi / lo, double(k) / double(n));
    return lo + double(k) * ((hi - lo) / double(n));
  }
};

// One axis: n cells plus one ghost each side; F[c] c = 0..n+2, x[c] c = 0..n+1.
struct Axis {
  int kind = 0;  // 0 r_sph, 1 r_cyl, 2 theta, 3 z
  int n = 0;
  int spacing = UNI;
  std::vector<double> F, x;
  void centres();
};
Axis axis_from_law(int kind, const Law& L, long c_first, long c_last);  // cells c_first..c_last
Axis coarse_axis(const Axis& a);

// 2-D plane tables (double), indices as in the paper: cell 1..n, ghosts 0, n+1.
struct PlaneGeo {
  int geometry = SPH;
  Axis r, t;
  int n_phi = 4;
  double G = 1.0;
  std::vector<double> aE, aW, P, Q, aN, aS, T, vr, vt;
  bool has_inner() const;
  bool has_lower() const;
  bool has_upper() const;
  void build();
  double s2(int m) const;
  double diag(int m, int i, int j) const {
    return -(aE[i] + aW[i]) - P[i] * (aN[j] + aS[j]) - s2(m) * Q[i] * T[j];
  }
};

struct LevelHost {
  PlaneGeo g;
  std::vector<double> rtab, ttab;   // packed RT_N x (nr+2), TT_N x (nt+2)
  std::vector<double> om_r, om_t;   // [M][nt], [M][nr]
  int gL = 0, gR = 0, gB = 0, gT = 0;
};

struct Hierarchy {
  std::vector<LevelHost> lv;
  int nc = 0;                       // cells of the coarsest level
  // Block factors of L_m on the coarsest level (blocks = polar rows J of
  // nb = nr cells, L_m block tridiagonal with diagonal couplings), per mode
  // slot: [nt][nb][nb] inverses of the Schur complements
  // S_0 = D_0, S_J = D_J - B_J S_{J-1}^{-1} C_{J-1}; then [nt][nb] sub-diagonal
  // couplings b_J (row J to J-1) and [nt][nb] super-diagonal couplings c_J
  // (row J to J+1).  Used when nb <= 64; otherwise coarse_inv holds the dense
  // inverse [M][nc][nc].
  std::vector<double> coarse_blk;
  std::vector<double> coarse_inv;
  int blk_n = 0, blk_nt = 0;
  // Separable factors (used when nt <= 64): on the coarsest level
  // L_m = L_r (x) I + D_r (x) L_t, with D_r = diag(P) and the s_m^2 term in
  // L_t (spherical, P = Q) or in L_r (cylindrical, P = T = 1).  Per slot:
  // V [nt][nt] and V^-1 [nt][nt] (L_t = V diag(lambda) V^-1), then per
  // eigenvalue k the Thomas factors of L_r + lambda_k D_r: 1/pivot [nt][nr],
  // upper/pivot [nt][nr] and lower/pivot [nt][nr] (the forward sweep is then
  // one FMA per cell: dp_i = z_i/pivot_i - (lower_i/pivot_i) dp_{i-1});
  // sep_stride doubles per slot.  sep_sym = 1: the polar operator is
  // mirror-symmetric (j <-> nt-1-j), eigenvectors k < nt/2 are even and
  // k >= nt/2 odd, and only the rows j < nt/2 of V ([nt/2][nt]) and the
  // columns j < nt/2 of V^-1 ([nt][nt/2]) are stored.
  std::vector<double> coarse_sep;
  int sep_stride = 0;
  int sep_sym = 0;
  double sep_check = -1.0;   // largest relative residual of the factors' check over the modes
  int large = 0;             // 1: built with the large coarsest-level rule
};

// Build levels: halve both sides while the short side exceeds min_side
// cells, or exceeds 4 cells while the plane has more than max_cells; neumann
// zeroes the inner radial face coefficient on every level.  modes: list of
// azimuthal mode numbers whose omega tables / coarse factors are needed
// (index = plane-mode slot).  sep_only: compute the coarsest level's factors
// only in the separable form (none when it does not apply).
bool build_hierarchy(const PlaneGeo& fine, bool neumann, const std::vector<int>& modes,
                     Hierarchy& H, std::string& err, int min_side = 16, int max_cells = 1024,
                     bool sep_only = false);

// The levels for a coarsest-size choice (0 automatic, 1 small, 2 large; see
// psolve_desc.coarsest_size) and precision (0 FP64, 1 mixed): the large rule
// (short side up to 32, up to 2048 cells) is kept only when its coarsest
// level has the separable form (and, automatic, for the mixed path with at
// least two levels); otherwise the small rule (16, 1024).
bool plan_hierarchy(const PlaneGeo& fine, bool neumann, const std::vector<int>& modes,
                    int coarsest_size, int precision, Hierarchy& H, std::string& err);


struct BPoint {
  char side;       // 'L','R','B','T'
  int i, j;        // ghost cell indices
  int ai, aj;      // adjacent domain cell
  double sigma_coef;   // screening-mass coefficient incl. 1/(4 pi G)
  double couple;       // coefficient of the ghost value in L at the adjacent cell
  double dV;           // 3-D volume of the ghost cell
};
std::vector<BPoint> boundary_points(const PlaneGeo& g);

}  // namespace ps
