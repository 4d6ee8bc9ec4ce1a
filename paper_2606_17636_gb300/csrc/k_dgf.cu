// Discrete Green's function tables on the device (Sec. 4.2).
#include "kernels.h"
#include "dgf.h"

namespace ps {

// G^m (deriv = 0) or dG^m/dr (deriv = 1) of -G/|x - x'| for a list of point
// pairs (Eqs. DGF_bc_sph, DGF_bc_cyl and their radial derivatives), all
// modes m = 0..M-1, one warp per pair.  out[m * mstride + pair * pstride],
// multiplied by scale[pair % scale_mod] when scale != nullptr.
__global__ void __launch_bounds__(256) k_green(GreenArgs a) {
  extern __shared__ double gsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long pair = long(blockIdx.x) * (blockDim.x >> 5) + warp;
  double* v = gsm + size_t(warp) * a.N;
  if (pair >= a.npairs) return;
  const double xt = a.xt[pair], yt = a.yt[pair], xs = a.xs[pair], ys = a.ys[pair];
  bool bad = false;
  for (int k = lane; k < a.N; k += 32) {
    const double c = a.cosk[k];
    double d2, num = 1.0;
    if (a.geometry == SPH) {
      const double ct = cos(yt), st = sin(yt), cs = cos(ys), ss = sin(ys);
      d2 = xt * xt + xs * xs - 2.0 * xt * xs * (ct * cs + st * ss * c);
      if (a.deriv) num = (xt - xs * ct * cs) - xs * st * ss * c;
    } else {
      d2 = xt * xt + xs * xs - 2.0 * xt * xs * c + (yt - ys) * (yt - ys);
      if (a.deriv) num = xt - xs * c;
    }
    if (!(d2 > 0.0)) bad = true;
    const double id = 1.0 / sqrt(d2);
    v[k] = a.deriv ? a.G * num * id * id * id : -a.G * id;
  }
  bad = __any_sync(0xffffffffu, bad);
  __syncwarp();
  const double sc = a.scale ? a.scale[pair % a.scale_mod] : 1.0;
  for (int m = lane; m < a.M; m += 32) {
    double s = 0.0;
    if (!bad)
      for (int k = 0; k < a.N; ++k) s += a.cosk[(long(m) * k) & (a.N - 1)] * v[k];
    a.out[long(m) * a.mstride + pair * a.pstride] = bad ? 0.0 : s * sc;
  }
}

void launch_green(const GreenArgs& a, cudaStream_t st) {
  if (a.npairs == 0) return;
  const long blocks = (a.npairs + 7) / 8;
  static bool attr = false;
  if (!attr) {   // 8 warps x N doubles: 64 KB at the largest N = 1024
    cudaFuncSetAttribute(k_green, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * 1024 * int(sizeof(double)));
    attr = true;
  }
  k_green<<<unsigned(blocks), 256, 8 * a.N * sizeof(double), st>>>(a);
}

// ---------------------------------------------------------------------------
// Extended domain: right-hand sides of the (source pair, mode) planes and the
// extraction of the table.  Plane p = slot * npairs + q holds sources 2q
// (real part) and 2q+1 (imaginary part) for the mode in `slot`.
// ---------------------------------------------------------------------------
__global__ void k_ext_rhs(ExtArgs a, double2* __restrict__ f, int p0, int np) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  const long cells = long(a.nr) * a.nt;
  if (idx >= long(np) * cells) return;
  const int pl = int(idx / cells);
  const int c = int(idx - long(pl) * cells);
  const int p = p0 + pl;
  const int slot = p / a.npairs, q = p - slot * a.npairs;
  const int j = c / a.nr, i = c - j * a.nr;   // 0-based extended cell
  double v[2] = {0.0, 0.0};
  for (int h = 0; h < 2; ++h) {
    const int s = 2 * q + h;
    if (s >= a.nb) continue;
    if (a.src_cell[s] == c) v[h] += a.four_pi_G / a.dV[s];
    // outer radial Dirichlet ghost (Eq. DGF_bc_*) enters cell nr-1
    if (i == a.nr - 1) v[h] -= a.aE_out * a.gout[(long(j) * a.nb + s) * a.M + slot];
    // bounded t edges (P is indexed by the 1-based cell)
    if (a.glo && j == 0) v[h] -= a.P[i + 1] * a.aS_lo * a.glo[(long(i) * a.nb + s) * a.M + slot];
    if (a.ghi && j == a.nt - 1) v[h] -= a.P[i + 1] * a.aN_hi * a.ghi[(long(i) * a.nb + s) * a.M + slot];
    // inner radial Neumann flux: + (A/dV) dG/dr at the inner face
    if (i == 0) v[h] += a.cN * a.dval[(long(j) * a.nb + s) * a.M + slot];
  }
  f[long(p - p0) * cells + c] = make_double2(v[0], v[1]);
}

__global__ void k_ext_extract(ExtArgs a, const double2* __restrict__ u, double* __restrict__ gt,
                              int p0, int np) {
  const long idx = long(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= long(np) * 2 * a.nb) return;
  const int pl = int(idx / (2 * a.nb));
  const int rem = int(idx - long(pl) * 2 * a.nb);
  const int h = rem / a.nb, t = rem - h * a.nb;
  const int p = p0 + pl;
  const int slot = p / a.npairs, q = p - slot * a.npairs;
  const int s = 2 * q + h;
  if (s >= a.nb) return;
  const double2 v = u[long(pl) * a.nr * a.nt + a.src_cell[t]];
  gt[(long(slot) * a.nb + t) * a.nb + s] = (h ? v.y : v.x) * a.dV[s];
}

void launch_ext_rhs(const ExtArgs& a, double2* f, int p0, int np, cudaStream_t st) {
  const long n = long(np) * a.nr * a.nt;
  k_ext_rhs<<<unsigned((n + 255) / 256), 256, 0, st>>>(a, f, p0, np);
}
void launch_ext_extract(const ExtArgs& a, const double2* u, double* gt, int p0, int np,
                        cudaStream_t st) {
  const long n = long(np) * 2 * a.nb;
  k_ext_extract<<<unsigned((n + 255) / 256), 256, 0, st>>>(a, u, gt, p0, np);
}

// ---------------------------------------------------------------------------
// Auxiliary windows: one block solves one (source, mode) window problem with
// Jacobi-preconditioned conjugate gradients on the symmetric positive form
// -dV L_m (the operator is volume-symmetric), FP64, to a relative residual
// of 1e-14, and writes the window values at the targets inside the window.
// ---------------------------------------------------------------------------
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) s += sh[w];
  return s;
}

__global__ void __launch_bounds__(256) k_aux_cg(AuxArgs a) {
  extern __shared__ double asm_[];
  __shared__ double red[8];
  const int prob = blockIdx.x;          // = slot * nb + s
  const int slot = prob / a.nb, s = prob - slot * a.nb;
  const AuxWin w = a.win[s];
  const int wr = w.i1 - w.i0 + 1, wt = w.j1 - w.j0 + 1, n = wr * wt;
  double* x = asm_;
  double* r = x + n;
  double* pp = r + n;
  double* ap = pp + n;
  double* dinv = ap + n;
  const double s2 = a.s2[slot];
  const int NR = a.nr_big + 2, NT = a.nt_big + 2;
  auto AE = [&](int i) { return a.rt[RT_AE * NR + i]; };
  auto AW = [&](int i) { return a.rt[RT_AW * NR + i]; };
  auto PP = [&](int i) { return a.rt[RT_P * NR + i]; };
  auto QQ = [&](int i) { return a.rt[RT_Q * NR + i]; };
  auto VR = [&](int i) { return a.rt[RT_V * NR + i]; };
  auto AN = [&](int j) { return a.tt[TT_AN * NT + j]; };
  auto AS = [&](int j) { return a.tt[TT_AS * NT + j]; };
  auto TT = [&](int j) { return a.tt[TT_T * NT + j]; };
  auto VT = [&](int j) { return a.tt[TT_V * NT + j]; };
  const double* ring = a.ring + (long(s) * a.ring_max) * a.M;   // [k][M]
  // right-hand side b = -dV (4 pi G delta / dV_s - ghost terms); x = 0
  double rr0 = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const int jj = c / wr, ii = c - jj * wr;
    const int i = w.i0 + ii, j = w.j0 + jj;
    const double dv = VR(i) * VT(j);
    double rhs = (i == w.is && j == w.js) ? a.four_pi_G / a.dV[s] : 0.0;
    // Dirichlet ring values sit in the order R side, L side, B side, T side
    if (ii == wr - 1) rhs -= AE(i) * ring[long(w.ring_r + jj) * a.M + slot];
    if (ii == 0 && w.ring_l >= 0) rhs -= AW(i) * ring[long(w.ring_l + jj) * a.M + slot];
    if (jj == 0 && w.ring_b >= 0) rhs -= PP(i) * AS(j) * ring[long(w.ring_b + ii) * a.M + slot];
    if (jj == wt - 1 && w.ring_t >= 0) rhs -= PP(i) * AN(j) * ring[long(w.ring_t + ii) * a.M + slot];
    const double b = -dv * rhs;
    const double diag = dv * ((AE(i) + AW(i)) + PP(i) * (AN(j) + AS(j)) + s2 * QQ(i) * TT(j));
    dinv[c] = 1.0 / diag;
    x[c] = 0.0;
    r[c] = b;
    pp[c] = b * dinv[c];
    rr0 += b * b * dinv[c];
  }
  double rz = block_sum(rr0, red);
  const double stop = rz * 1e-28;
  int it = 0;
  for (; it < a.max_iter && rz > stop; ++it) {
    double pap = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int jj = c / wr, ii = c - jj * wr;
      const int i = w.i0 + ii, j = w.j0 + jj;
      const double dv = VR(i) * VT(j);
      const double pc = pp[c];
      double lp = -(AE(i) + AW(i) + PP(i) * (AN(j) + AS(j)) + s2 * QQ(i) * TT(j)) * pc;
      if (ii + 1 < wr) lp += AE(i) * pp[c + 1];
      if (ii > 0) lp += AW(i) * pp[c - 1];
      if (jj + 1 < wt) lp += PP(i) * AN(j) * pp[c + wr];
      if (jj > 0) lp += PP(i) * AS(j) * pp[c - wr];
      ap[c] = -dv * lp;
      pap += pc * ap[c];
    }
    pap = block_sum(pap, red);
    const double alpha = rz / pap;
    double rzn = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      x[c] += alpha * pp[c];
      r[c] -= alpha * ap[c];
      rzn += r[c] * r[c] * dinv[c];
    }
    rzn = block_sum(rzn, red);
    const double beta = rzn / rz;
    rz = rzn;
    for (int c = threadIdx.x; c < n; c += blockDim.x) pp[c] = r[c] * dinv[c] + beta * pp[c];
    __syncthreads();
  }
  if (threadIdx.x == 0 && it >= a.max_iter && a.fail) atomicAdd(a.fail, 1);
  // targets inside the window
  for (int k = threadIdx.x; k < w.ntarget; k += blockDim.x) {
    const int t = a.tlist[w.tfirst + k];
    const int i = a.tcell_i[t], j = a.tcell_j[t];
    const int c = (j - w.j0) * wr + (i - w.i0);
    a.gt[(long(slot) * a.nb + t) * a.nb + s] = x[c] * a.dV[s];
  }
}

void launch_aux_cg(const AuxArgs& a, int nprob, int max_cells, cudaStream_t st) {
  const size_t sm = size_t(5) * max_cells * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_aux_cg, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    attr = true;
  }
  k_aux_cg<<<nprob, 256, sm, st>>>(a);
}

}  // namespace ps
