// Discrete Green's function tables on the device (Sec. 4.2).
#include "kernels.h"
#include "dgf.h"

namespace ps {

// G^m (deriv = 0) or dG^m/dr (deriv = 1) of -G/|x - x'| for a list of point
// pairs (Eqs. DGF_bc_sph, DGF_bc_cyl and their radial derivatives), all
// modes m = 0..M-1.  The kernel of a pair depends on phi - phi' only through
// cos(2 pi k / N), so its samples v[k] are real and even in k and their DFT
// is real: G^m = sum_k v[k] cos(2 pi m k / N).  A warp takes two pairs a, b,
// packs z[k] = v_a[k] + i v_b[k] and computes the length-N DFT of z by a
// radix-2 FFT in its shared memory (bit-reversed input order): then
// G_a^m = Re Z[m] and G_b^m = Im Z[m].  out[m * mstride + pair * pstride],
// multiplied by scale[pair % scale_mod] when scale != nullptr.
__device__ __forceinline__ double green_sample(const GreenArgs& a, long pair, double c, bool& bad) {
  const double xt = a.xt[pair], yt = a.yt[pair], xs = a.xs[pair], ys = a.ys[pair];
  double d2, num = 1.0;
  if (a.geometry == SPH) {
    const double ct = cos(yt), st = sin(yt), cs = cos(ys), ss = sin(ys);
    d2 = xt * xt + xs * xs - 2.0 * xt * xs * (ct * cs + st * ss * c);
    if (a.deriv) num = (xt - xs * ct * cs) - xs * st * ss * c;
  } else {
    d2 = xt * xt + xs * xs - 2.0 * xt * xs * c + (yt - ys) * (yt - ys);
    if (a.deriv) num = xt - xs * c;
  }
  if (!(d2 > 0.0)) {
    bad = true;
    return 0.0;
  }
  const double id = 1.0 / sqrt(d2);
  return a.deriv ? a.G * num * id * id * id : -a.G * id;
}

__global__ void __launch_bounds__(128) k_green(GreenArgs a, int lg) {
  extern __shared__ double2 gz[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = a.N;
  const long pa = (long(blockIdx.x) * (blockDim.x >> 5) + warp) * 2, pb = pa + 1;
  if (pa >= a.npairs) return;
  const bool has_b = pb < a.npairs;
  double2* z = gz + size_t(warp) * N;
  bool bad_a = false, bad_b = false;
  for (int k = lane; k < N; k += 32) {
    const double c = a.cosk[k];
    const double va = green_sample(a, pa, c, bad_a);
    const double vb = has_b ? green_sample(a, pb, c, bad_b) : 0.0;
    const int kr = lg ? int(__brev(unsigned(k)) >> (32 - lg)) : 0;
    z[kr] = make_double2(va, vb);
  }
  bad_a = __any_sync(0xffffffffu, bad_a);
  bad_b = __any_sync(0xffffffffu, bad_b);
  __syncwarp();
  // decimation in time: butterflies of span `half`, twiddle e^{-2 pi i t / N}
  // with sin(2 pi t / N) = cos(2 pi (t - N/4) / N)
  for (int half = 1; half < N; half <<= 1) {
    const int step = N / (2 * half);
    for (int j = lane; j < N / 2; j += 32) {
      const int pos = j & (half - 1);
      const int i0 = ((j - pos) << 1) + pos, i1 = i0 + half;
      const int t = pos * step;
      const double wr = a.cosk[t];
      const double wi = t ? -a.cosk[(t + 3 * (N >> 2)) & (N - 1)] : 0.0;
      const double2 u = z[i0], v = z[i1];
      const double vr = v.x * wr - v.y * wi, vi = v.x * wi + v.y * wr;
      z[i0] = make_double2(u.x + vr, u.y + vi);
      z[i1] = make_double2(u.x - vr, u.y - vi);
    }
    __syncwarp();
  }
  const double sa = a.scale ? a.scale[pa % a.scale_mod] : 1.0;
  const double sb = (a.scale && has_b) ? a.scale[pb % a.scale_mod] : 1.0;
  for (int m = lane; m < a.M; m += 32) {
    const double2 v = z[m];
    a.out[long(m) * a.mstride + pa * a.pstride] = bad_a ? 0.0 : v.x * sa;
    if (has_b) a.out[long(m) * a.mstride + pb * a.pstride] = bad_b ? 0.0 : v.y * sb;
  }
}

void launch_green(const GreenArgs& a, cudaStream_t st) {
  if (a.npairs == 0) return;
  int lg = 0;
  while ((1 << lg) < a.N) ++lg;
  const long blocks = (a.npairs + 7) / 8;   // 4 warps x 2 pairs
  static bool attr = false;
  if (!attr) {   // 4 warps x N complex doubles: 64 KB at the largest N = 1024
    cudaFuncSetAttribute(k_green, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 1024 * int(sizeof(double2)));
    attr = true;
  }
  k_green<<<unsigned(blocks), 128, 4 * a.N * sizeof(double2), st>>>(a, lg);
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
// Auxiliary windows: one block solves one (source, mode) window problem on
// the symmetric positive form -dV L_m (the operator is volume-symmetric) to a
// relative residual of 1e-14 (Jacobi-preconditioned norm), and writes the
// window values at the targets inside the window.  Mixed-precision iterative
// refinement: the solution x and the defect r = b - A x are FP64; each
// correction A d = r is solved by Jacobi-preconditioned conjugate gradients
// in FP32 (coefficients staged once per block as FP32) until its own
// preconditioned residual falls by 1e-8, then x += d and the FP64 defect is
// formed again.  GB300's FP32 rate is about 64 times its FP64 rate, so the
// FP64 work is a few stencil passes per window instead of one per CG step.
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

__device__ float block_sumf(float v, float* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) s += sh[w];
  return s;
}

// FP32 coefficients of one window cell of -dV L_m: east, west, north, south
// neighbours and the diagonal (A c = diag c - sum nb c_nb)
struct AuxCoef {
  float e, w, n, s, d;
};

__global__ void __launch_bounds__(256) k_aux_cg(AuxArgs a) {
  extern __shared__ double asm_[];
  __shared__ double red[8];
  __shared__ float redf[8];
  const int prob = blockIdx.x;          // = slot * nb + s
  const int slot = prob / a.nb, s = prob - slot * a.nb;
  const AuxWin w = a.win[s];
  const int wr = w.i1 - w.i0 + 1, wt = w.j1 - w.j0 + 1, n = wr * wt;
  double* x = asm_;                     // FP64 solution
  double* b = x + n;                    // FP64 right-hand side
  double* r64 = b + n;                  // FP64 defect
  float* d = reinterpret_cast<float*>(r64 + n);   // FP32 correction
  float* r = d + n;
  float* pp = r + n;
  float* ap = pp + n;
  float* dinv = ap + n;
  AuxCoef* cf = reinterpret_cast<AuxCoef*>(dinv + n + (n & 1));   // 8-byte aligned
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
  double rz = 0.0;
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
    const double bc = -dv * rhs;
    const double diag = dv * ((AE(i) + AW(i)) + PP(i) * (AN(j) + AS(j)) + s2 * QQ(i) * TT(j));
    AuxCoef q;
    q.e = ii + 1 < wr ? float(dv * AE(i)) : 0.f;
    q.w = ii > 0 ? float(dv * AW(i)) : 0.f;
    q.n = jj + 1 < wt ? float(dv * PP(i) * AN(j)) : 0.f;
    q.s = jj > 0 ? float(dv * PP(i) * AS(j)) : 0.f;
    q.d = float(diag);
    cf[c] = q;
    dinv[c] = float(1.0 / diag);
    x[c] = 0.0;
    b[c] = bc;
    r64[c] = bc;
    rz += bc * bc / diag;
  }
  rz = block_sum(rz, red);
  const double stop = rz * 1e-28;
  int it = 0;
  for (int outer = 0; outer < 12 && rz > stop; ++outer) {
    // FP32 conjugate gradients on A d = r64, d = 0
    float rzf = 0.f;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const float rc = float(r64[c]);
      r[c] = rc;
      d[c] = 0.f;
      pp[c] = rc * dinv[c];
      rzf += rc * rc * dinv[c];
    }
    rzf = block_sumf(rzf, redf);
    const float inner_stop = rzf * 1e-8f;
    for (; it < a.max_iter && rzf > inner_stop; ++it) {
      float pap = 0.f;
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const AuxCoef q = cf[c];
        const int ii = c % wr;
        float v = q.d * pp[c];
        if (ii + 1 < wr) v -= q.e * pp[c + 1];
        if (ii > 0) v -= q.w * pp[c - 1];
        if (c + wr < n) v -= q.n * pp[c + wr];
        if (c >= wr) v -= q.s * pp[c - wr];
        ap[c] = v;
        pap += pp[c] * v;
      }
      pap = block_sumf(pap, redf);
      const float alpha = rzf / pap;
      float rzn = 0.f;
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        d[c] += alpha * pp[c];
        const float rc = r[c] - alpha * ap[c];
        r[c] = rc;
        rzn += rc * rc * dinv[c];
      }
      rzn = block_sumf(rzn, redf);
      const float beta = rzn / rzf;
      rzf = rzn;
      for (int c = threadIdx.x; c < n; c += blockDim.x) pp[c] = r[c] * dinv[c] + beta * pp[c];
      __syncthreads();
    }
    // x += d; FP64 defect r64 = b - A x with the FP64 coefficients
    for (int c = threadIdx.x; c < n; c += blockDim.x) x[c] += double(d[c]);
    __syncthreads();
    double rzd = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int jj = c / wr, ii = c - jj * wr;
      const int i = w.i0 + ii, j = w.j0 + jj;
      const double dv = VR(i) * VT(j);
      double lx = -(AE(i) + AW(i) + PP(i) * (AN(j) + AS(j)) + s2 * QQ(i) * TT(j)) * x[c];
      if (ii + 1 < wr) lx += AE(i) * x[c + 1];
      if (ii > 0) lx += AW(i) * x[c - 1];
      if (jj + 1 < wt) lx += PP(i) * AN(j) * x[c + wr];
      if (jj > 0) lx += PP(i) * AS(j) * x[c - wr];
      const double rc = b[c] + dv * lx;
      r64[c] = rc;
      rzd += rc * rc * double(dinv[c]);
    }
    rz = block_sum(rzd, red);
  }
  if (threadIdx.x == 0 && (rz > stop || !(rz == rz)) && a.fail) atomicAdd(a.fail, 1);
  // targets inside the window
  for (int k = threadIdx.x; k < w.ntarget; k += blockDim.x) {
    const int t = a.tlist[w.tfirst + k];
    const int i = a.tcell_i[t], j = a.tcell_j[t];
    const int c = (j - w.j0) * wr + (i - w.i0);
    a.gt[(long(slot) * a.nb + t) * a.nb + s] = x[c] * a.dV[s];
  }
}

void launch_aux_cg(const AuxArgs& a, int nprob, int max_cells, cudaStream_t st) {
  // FP64 x, b, r; FP32 d, r, p, Ap, 1/diag; five FP32 coefficients per cell
  const size_t sm = size_t(max_cells) * (3 * sizeof(double) + 5 * sizeof(float) + sizeof(AuxCoef)) + 8;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_aux_cg, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr = true;
  }
  k_aux_cg<<<nprob, 256, sm, st>>>(a);
}

}  // namespace ps
