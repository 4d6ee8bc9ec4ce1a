// Vacuum boundary treatment per Fourier mode (Sec. 4): screening mass
// (Eqs. charge_sph, charge_cyl), boundary potential as a DGF convolution
// (Eqs. theta_left..theta_top) and the Dirichlet data -Theta folded into the
// right-hand side of the second solve.
#include "kernels.h"

namespace ps {

// sigma[m][b] = coef_b * psi[m][adj_b]
__global__ void k_screening(BDev b, const double2* __restrict__ psi, double2* __restrict__ sigma,
                            int M) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * b.nb) return;
  const int m = idx / b.nb, t = idx - m * b.nb;
  const double2 v = psi[size_t(m) * b.plane_cells + b.adj[t]];
  const double c = b.sig[t];
  sigma[idx] = make_double2(c * v.x, c * v.y);
}

void launch_screening(const BDev& b, const double2* psi, double2* sigma, int M, cudaStream_t st) {
  const int n = M * b.nb;
  k_screening<<<(n + 255) / 256, 256, 0, st>>>(b, psi, sigma, M);
}

// theta[m][t] = sum_s gt[m][t][s] sigma[m][s]: one warp per (m, t) row; the
// table is the only large stream and is read once, coalesced.
__global__ void __launch_bounds__(256) k_boundary(const double* __restrict__ gt,
                                                  const double2* __restrict__ sigma,
                                                  double2* __restrict__ theta, int M, int nb) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= M * nb) return;
  const int m = warp / nb;
  const double* row = gt + size_t(warp) * nb;
  const double2* sg = sigma + size_t(m) * nb;
  double sx = 0.0, sy = 0.0;
  for (int s = lane; s < nb; s += 32) {
    const double g = __ldg(row + s);
    const double2 v = sg[s];
    sx += g * v.x;
    sy += g * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_down_sync(0xffffffffu, sx, o);
    sy += __shfl_down_sync(0xffffffffu, sy, o);
  }
  if (lane == 0) theta[warp] = make_double2(sx, sy);
}

void launch_boundary_potential(const double* gt, const double2* sigma, double2* theta, int M,
                               int nb, cudaStream_t st) {
  const long warps = long(M) * nb;
  k_boundary<<<unsigned((warps * 32 + 255) / 256), 256, 0, st>>>(gt, sigma, theta, M, nb);
}

// Several densities of one geometry (planes p = b M + m, b < nd): theta of
// every density at once, theta[bM+m][t] = sum_s gt[m][t][s] sigma[bM+m][s],
// so each table row is read once for up to ND densities (a [nb x nb] by
// [nb x 2 nd] product per mode).  One warp per (m, t) row.
template <int ND>
__global__ void __launch_bounds__(256) k_boundary_multi(const double* __restrict__ gt,
                                                        const double2* __restrict__ sigma,
                                                        double2* __restrict__ theta, int M, int nb,
                                                        int nd, int b0) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= M * nb) return;
  const int m = warp / nb, t = warp - m * nb;
  const int nb_here = nd - b0 < ND ? nd - b0 : ND;
  const double* row = gt + size_t(warp) * nb;
  double sx[ND], sy[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) sx[q] = sy[q] = 0.0;
  for (int s = lane; s < nb; s += 32) {
    const double g = __ldg(row + s);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      if (q < nb_here) {
        const double2 v = sigma[(size_t(b0 + q) * M + m) * nb + s];
        sx[q] += g * v.x;
        sy[q] += g * v.y;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      sx[q] += __shfl_down_sync(0xffffffffu, sx[q], o);
      sy[q] += __shfl_down_sync(0xffffffffu, sy[q], o);
    }
    if (lane == 0 && q < nb_here) theta[(size_t(b0 + q) * M + m) * nb + t] = make_double2(sx[q], sy[q]);
  }
}

void launch_boundary_potential_multi(const double* gt, const double2* sigma, double2* theta, int M,
                                     int nb, int nd, cudaStream_t st) {
  const long warps = long(M) * nb;
  for (int b0 = 0; b0 < nd; b0 += 8)
    k_boundary_multi<8><<<unsigned((warps * 32 + 255) / 256), 256, 0, st>>>(gt, sigma, theta, M, nb, nd, b0);
}

// f[m][cell] += cpl_b * theta[m][b] for the (at most two) ghosts of a cell:
// L_m u = f with ghost u = -Theta  <=>  L_m(ghost 0) u = f + cpl * Theta.
__global__ void k_rhs_ghosts(BDev b, double2* __restrict__ f, const double2* __restrict__ theta,
                             int M) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * b.ncell) return;
  const int m = idx / b.ncell, k = idx - m * b.ncell;
  double2 v = f[size_t(m) * b.plane_cells + b.cell[k]];
  for (int q = 0; q < 2; ++q) {
    const int t = b.cbp[2 * k + q];
    if (t < 0) continue;
    const double2 th = theta[size_t(m) * b.nb + t];
    v.x += b.cpl[t] * th.x;
    v.y += b.cpl[t] * th.y;
  }
  f[size_t(m) * b.plane_cells + b.cell[k]] = v;
}

void launch_rhs_ghosts(const BDev& b, double2* f, const double2* theta, int M, cudaStream_t st) {
  const int n = M * b.ncell;
  k_rhs_ghosts<<<(n + 255) / 256, 256, 0, st>>>(b, f, theta, M);
}

}  // namespace ps
