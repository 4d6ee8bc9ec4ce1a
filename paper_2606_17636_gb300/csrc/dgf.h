// Device-side construction of the discrete Green's function tables (Sec. 4.2).
#pragma once
#include <string>
#include <vector>

#include "kernels.h"
#include "solver.h"

namespace ps {

struct GreenArgs {
  int geometry, N, M, deriv;
  double G;
  long npairs;
  const double *xt, *yt, *xs, *ys;   // field and source points per pair
  const double* cosk;                // cos(2 pi k / N), k < N
  double* out;
  long mstride, pstride;
  const double* scale;
  long scale_mod;
};
void launch_green(const GreenArgs& a, cudaStream_t st);

struct ExtArgs {
  int nr, nt, nb, npairs, M;
  double four_pi_G, aE_out, aS_lo, aN_hi, cN;
  const int* src_cell;   // [nb] extended cell (0-based j*nr + i) of each boundary point
  const double* dV;      // [nb] source-cell volumes
  const double* P;       // [nr+2] radial factor of the extended plane (0-based cell i -> P[i+1])
  const double* gout;    // [nt][nb][M] Dirichlet data at the outer radial ghosts
  const double* glo;     // [nr][nb][M] lower edge ghosts (nullptr: no data there)
  const double* ghi;     // [nr][nb][M] upper edge ghosts (nullptr: no data there)
  const double* dval;    // [nt][nb][M] radial derivative at the inner face
};
void launch_ext_rhs(const ExtArgs& a, double2* f, int p0, int np, cudaStream_t st);
void launch_ext_extract(const ExtArgs& a, const double2* u, double* gt, int p0, int np,
                        cudaStream_t st);

struct AuxWin {
  int i0, i1, j0, j1;        // window cells in big-plane indices (1-based)
  int is, js;                // source cell
  int ring_r, ring_l, ring_b, ring_t;   // offsets of the ring sides (-1 = no data)
  int tfirst, ntarget;       // targets inside the window: tlist[tfirst .. +ntarget)
};
struct AuxArgs {
  int nb, M, nr_big, nt_big, ring_max, max_iter;
  double four_pi_G;
  const double* rt;          // big-plane radial tables RT_N x (nr_big+2)
  const double* tt;          // big-plane polar tables TT_N x (nt_big+2)
  const double* s2;          // [M]
  const double* dV;          // [nb]
  const AuxWin* win;         // [nb]
  const double* ring;        // [nb*ring_max][M]
  const int* tlist;
  const int* tcell_i;        // [nb] big-plane cell of each boundary point
  const int* tcell_j;
  double* gt;
  int* fail;
};
void launch_aux_cg(const AuxArgs& a, int nprob, int max_cells, cudaStream_t st);

// Build the table gt[m][t][s] (device, M * nb * nb doubles) for the plane `g`
// whose boundary points are `bp`.  Scratch comes from a temporary arena.
// `construction`: in, 0 automatic (Sec. 4.2), 1 auxiliary windows, 2 the
// extended domain; out, 1 when the extended domain was used, else 0.
bool build_dgf(const PlaneGeo& g, const Law& rlaw, const Law& tlaw,
               const std::vector<BPoint>& bp, double* gt, Arena& scratch, cudaStream_t st,
               int& construction, std::string& err);

bool uses_extended(const Law& rlaw, int n_r);

}  // namespace ps
