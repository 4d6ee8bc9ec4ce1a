// Cluster-resident multigrid iterations for the last few active mode planes.
//
// App. B: the low modes (m = 0 above all) need many more V-cycles than the
// rest, so the end of every solve iterates on one or a few planes.  The
// level-wide kernels then leave most of the GPU idle and pay a launch per
// step.  Here each remaining plane gets one thread-block cluster (C CTAs,
// one per SM) that keeps the whole plane's multigrid state in distributed
// shared memory and loops on the device until the plane meets the App. B
// criterion: FP64 residual and norms, the FP32 V-cycle of Sec. 3 on every
// level (Algorithm 1's alternating zebra line relaxation, area-weighted
// restriction, the exact FP64 coarsest solve, bilinear prolongation), and
// the FP64 update.
//
// Decomposition: on every level the CTA of rank c owns rows [c s, (c+1) s)
// of the (r, theta) / (R, z) plane.  Radial lines lie inside one CTA.  A
// polar line crosses all CTAs; each CTA relaxes the segment of it that
// covers its own rows plus h = 2 n_sor rows of its neighbours on each side
// (halo rows, copied in).  n_sor even-odd SOR sweeps move information at
// most 2 n_sor cells along the line, so the values the CTA keeps -- its own
// rows -- are exactly those of a relaxation of the whole line.  After every
// colour step each CTA writes its boundary rows into its neighbours' halo
// buffers (distributed shared memory stores) and the cluster synchronises
// once; the halo buffers alternate between steps, so a CTA still reading its
// halo never sees a neighbour's newer rows.  Prolongation is computed by each
// CTA for its halo rows too (it holds the coarse rows they need), so the
// halo stays current without an exchange.
//
// The arithmetic of every cell is that of the level-wide and shared-memory
// kernels (the same line-relaxation helpers, restriction, prolongation,
// coarsest-solve and residual expressions).
#include <cooperative_groups.h>

#include <cstdio>

#include "lines.cuh"

namespace cg = cooperative_groups;

namespace ps {

namespace {

typedef float2 V;
constexpr int kTailThreads = 256;
enum { TS_ACTIVE = 1, TS_OK = 0, TS_STAGNATED = 2, TS_NOTCONV = -4, TS_NONFINITE = -5 };

struct __align__(16) D4 {
  double x, y, z, w;
};

__device__ __forceinline__ V vz() { return make_float2(0.f, 0.f); }

// Row r (relative to the CTA's first row, -h <= r < s + h) of a level's error.
__device__ __forceinline__ V* erow(unsigned char* sm, const TailLevel& t, int h, int cur, int r) {
  V* b = reinterpret_cast<V*>(sm);
  const int nr = t.L.nr;
  if (r < 0) return b + (cur ? t.eh1 : t.eh0) + (r + h) * nr;
  if (r >= t.s) return b + (cur ? t.eh1 : t.eh0) + (h + r - t.s) * nr;
  return b + t.eo + r * nr;
}
__device__ __forceinline__ V* frow(unsigned char* sm, const TailLevel& t, int h, int r) {
  return reinterpret_cast<V*>(sm) + t.fo + (r + h) * t.L.nr;
}

// Copies the CTA's own rows (row r at src + r nr, r < s) into the halo slots
// of every CTA of the cluster whose halo (h rows on each side) covers them.
// Target rank + d receives rows r >= d s - h at its top slot r - d s + h
// (top slots at top_off); target rank - d receives rows r < h - (d - 1) s at
// its bottom slot r + (d - 1) s (bottom slots at bot_off).
__device__ void push_halo(cg::cluster_group& cl, unsigned char* sm, const V* src, int s, int nr,
                          int h, int top_off, int bot_off, int rank, int C) {
  const int chunks = nr >> 1;   // two cells per 16-byte store
  V* base = reinterpret_cast<V*>(sm);
  for (int d = 1; (d - 1) * s < h; ++d) {
    for (int side = 0; side < 2; ++side) {
      const int tgt = side ? rank - d : rank + d;
      if (tgt < 0 || tgt >= C) continue;
      const int r0 = side ? 0 : max(0, d * s - h);
      const int r1 = side ? min(s, h - (d - 1) * s) : s;
      if (r1 <= r0) continue;
      V* tb = cl.map_shared_rank(base, tgt);
      const int n = (r1 - r0) * chunks;
      for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int q = idx / chunks, c = idx - q * chunks, rr = r0 + q;
        const int slot = side ? bot_off + (rr + (d - 1) * s) * nr : top_off + (rr - d * s + h) * nr;
        *reinterpret_cast<float4*>(tb + slot + 2 * c) = *reinterpret_cast<const float4*>(src + rr * nr + 2 * c);
      }
    }
  }
}

// Radial lines of colour `color` among the CTA's own rows, one warp per line
// (Sec. 3.2; the helpers of the level-wide pass).
template <int CPL>
__device__ void t_rlines(const LevelDev& L, unsigned char* sm, const TailLevel& t, int h, int cur,
                         int j0, float s2, int n_sor, int color) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nr = L.nr, nt = L.nt;
  RLineTabs<float, CPL> tabs;
  ld_rtabs<float, CPL>(tabs, L, L.rf);
  for (int r = 2 * warp + color; r < t.s; r += 2 * nw) {
    const int j = j0 + r;
    V ev[CPL], g[CPL], un[CPL], us[CPL];
    ld_line<V, CPL>(ev, erow(sm, t, h, cur, r), lane, nr);
    ld_line<V, CPL>(g, frow(sm, t, h, r), lane, nr);
    if (j + 1 < nt) {
      ld_line<V, CPL>(un, erow(sm, t, h, cur, r + 1), lane, nr);
    } else {
#pragma unroll
      for (int c = 0; c < CPL; ++c) un[c] = vz();
    }
    if (j > 0) {
      ld_line<V, CPL>(us, erow(sm, t, h, cur, r - 1), lane, nr);
    } else {
#pragma unroll
      for (int c = 0; c < CPL; ++c) us[c] = vz();
    }
    relax_r<float, CPL>(L, tabs, L.tf, s2, L.omr_f[j], j, g, un, us, n_sor, ev);
    st_line<V, CPL>(erow(sm, t, h, cur, r), ev, lane, nr);
  }
}

// Polar lines of colour `color`: one thread per column relaxes the segment
// of rows [rlo, rhi) (own rows and up to h halo rows each side, clipped to
// the plane) with the even-odd SOR sweeps of the line smoother, and keeps
// the own rows.  LM >= rhi - rlo.
template <int LM>
__device__ void t_tcols(const LevelDev& L, unsigned char* sm, const TailLevel& t, int h, int cur,
                        int j0, float s2, int n_sor, int color) {
  const int nr = L.nr, nt = L.nt, NR = nr + 2, NT = nt + 2;
  const float* rt = L.rf;
  const float* tt = L.tf;
  const int rlo = max(-h, -j0), rhi = min(t.s + h, nt - j0), n = rhi - rlo;
  const int par0 = (j0 + rlo) & 1;
  for (int col = threadIdx.x; 2 * col + color < nr; col += blockDim.x) {
    const int i = 2 * col + color;
    const float P = rt[RT_P * NR + i + 1], aE = rt[RT_AE * NR + i + 1], aW = rt[RT_AW * NR + i + 1];
    const float dr = rt[RT_DR * NR + i + 1], Qi = rt[RT_Q * NR + i + 1];
    const float w = L.omt_f[i], w1 = 1.0f - w;
    V x[LM], g[LM];
    float up[LM], dn[LM], id[LM];
#pragma unroll
    for (int k = 0; k < LM; ++k) {
      x[k] = g[k] = vz();
      up[k] = dn[k] = id[k] = 0.f;
      if (k < n) {
        const int r = rlo + k, jj = j0 + r + 1;
        const V* er = erow(sm, t, h, cur, r);
        x[k] = er[i];
        const V ue = (i + 1 < nr) ? er[i + 1] : vz();
        const V uw = (i > 0) ? er[i - 1] : vz();
        const V fv = frow(sm, t, h, r)[i];
        g[k].x = fv.x - aE * ue.x - aW * uw.x;
        g[k].y = fv.y - aE * ue.y - aW * uw.y;
        id[k] = rcp_diag(dr + P * tt[TT_DT * NT + jj] - s2 * Qi * tt[TT_T * NT + jj]);
        up[k] = P * tt[TT_AN * NT + jj];
        dn[k] = P * tt[TT_AS * NT + jj];
      }
    }
    for (int it = 0; it < n_sor; ++it) {
#pragma unroll
      for (int par = 0; par < 2; ++par) {
#pragma unroll
        for (int k = 0; k < LM; ++k) {
          if (k < n && ((k + par0) & 1) == par) {
            const V em = k > 0 ? x[k > 0 ? k - 1 : 0] : vz();
            const V ep = k + 1 < n ? x[k + 1 < LM ? k + 1 : k] : vz();
            const float tx = (g[k].x - up[k] * ep.x - dn[k] * em.x) * id[k];
            const float ty = (g[k].y - up[k] * ep.y - dn[k] * em.y) * id[k];
            x[k].x = w1 * x[k].x + w * tx;
            x[k].y = w1 * x[k].y + w * ty;
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < LM; ++k) {
      const int r = rlo + k;
      if (k < n && r >= 0 && r < t.s) erow(sm, t, h, cur, r)[i] = x[k];
    }
  }
}

__device__ void t_rstep(const LevelDev& L, unsigned char* sm, const TailLevel& t, int h, int cur,
                        int j0, float s2, int n_sor, int color) {
  switch (L.nr <= 32 ? 1 : L.nr >> 5) {
    case 1: t_rlines<1>(L, sm, t, h, cur, j0, s2, n_sor, color); break;
    case 2: t_rlines<2>(L, sm, t, h, cur, j0, s2, n_sor, color); break;
    case 4: t_rlines<4>(L, sm, t, h, cur, j0, s2, n_sor, color); break;
    default: t_rlines<8>(L, sm, t, h, cur, j0, s2, n_sor, color); break;
  }
}

__device__ void t_tstep(const LevelDev& L, unsigned char* sm, const TailLevel& t, int h, int cur,
                        int j0, float s2, int n_sor, int color) {
  const int n = t.s + 2 * h;
  if (n <= 8) t_tcols<8>(L, sm, t, h, cur, j0, s2, n_sor, color);
  else if (n <= 12) t_tcols<12>(L, sm, t, h, cur, j0, s2, n_sor, color);
  else if (n <= 16) t_tcols<16>(L, sm, t, h, cur, j0, s2, n_sor, color);
  else t_tcols<24>(L, sm, t, h, cur, j0, s2, n_sor, color);
}

// `cycles` smoothing cycles of one level: radial colours 0, 1, polar colours
// 0, 1; after each step the boundary rows go to the neighbours' other halo
// buffer and the cluster synchronises.
__device__ void t_smooth(cg::cluster_group& cl, const LevelDev& L, unsigned char* sm,
                         const TailLevel& t, int h, int& cur, int rank, int C, float s2, int n_sor,
                         int cycles) {
  const int j0 = rank * t.s;
  for (int cyc = 0; cyc < cycles; ++cyc)
    for (int dir = 0; dir < 2; ++dir)
      for (int color = 0; color < 2; ++color) {
        if (dir == 0) t_rstep(L, sm, t, h, cur, j0, s2, n_sor, color);
        else t_tstep(L, sm, t, h, cur, j0, s2, n_sor, color);
        __syncthreads();
        const int nb = cur ? t.eh0 : t.eh1;
        push_halo(cl, sm, reinterpret_cast<V*>(sm) + t.eo, t.s, L.nr, h, nb, nb + h * L.nr, rank, C);
        cl.sync();
        cur ^= 1;
      }
}

// Coarse right-hand side of the CTA's own coarse rows: the area-weighted
// restriction of the defect f - L e (Sec. 3.1), with the expression of the
// other restriction kernels.
__device__ void t_restrict(const LevelDev& L, const LevelDev& Cl, unsigned char* sm,
                           const TailLevel& tf, const TailLevel& tc, int h, int cur, int rank,
                           float s2, V* out) {
  const int nr = L.nr, nt = L.nt, NR = nr + 2, NT = nt + 2;
  const float* rt = L.rf;
  const float* tt = L.tf;
  const int j0 = rank * tf.s;
  const int n = tc.s * Cl.nr;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int R = idx / Cl.nr, I = idx - R * Cl.nr;
    float ax = 0.f, ay = 0.f;
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int i = 2 * I + a, rr = 2 * R + b, j = j0 + rr;
        const V* er = erow(sm, tf, h, cur, rr);
        const V c = er[i];
        const V E = (i + 1 < nr) ? er[i + 1] : vz();
        const V W = (i > 0) ? er[i - 1] : vz();
        const V N = (j + 1 < nt) ? erow(sm, tf, h, cur, rr + 1)[i] : vz();
        const V S = (j > 0) ? erow(sm, tf, h, cur, rr - 1)[i] : vz();
        const float aE = rt[RT_AE * NR + i + 1], aW = rt[RT_AW * NR + i + 1], P = rt[RT_P * NR + i + 1];
        const float aN = P * tt[TT_AN * NT + j + 1], aS = P * tt[TT_AS * NT + j + 1];
        const float d = rt[RT_DR * NR + i + 1] + P * tt[TT_DT * NT + j + 1] -
                        s2 * rt[RT_Q * NR + i + 1] * tt[TT_T * NT + j + 1];
        const V fv = frow(sm, tf, h, rr)[i];
        const float rx = fv.x - (aE * E.x + aW * W.x + aN * N.x + aS * S.x + d * c.x);
        const float ry = fv.y - (aE * E.y + aW * W.y + aN * N.y + aS * S.y + d * c.y);
        const float wgt = rt[RT_RW * NR + i + 1] * tt[TT_RW * NT + j + 1];
        ax += wgt * rx;
        ay += wgt * ry;
      }
    out[R * Cl.nr + I] = make_float2(ax, ay);
  }
}

// Coarse-grid value at 1-based coarse indices (I, J) with the ghost rules of
// the coarse level (zero next to a Dirichlet side, (-1)^m times the
// neighbour across a pole or the axis, the neighbour itself across a
// Neumann face or the origin).
__device__ __forceinline__ V t_cval(const LevelDev& Cl, unsigned char* sm, const TailLevel& tc,
                                    int h, int cur, int j0c, int I, int J, int m) {
  float fac = 1.f;
  const float sgn = (m & 1) ? -1.f : 1.f;
  int Ic = I, Jc = J;
  if (I == 0) { if (Cl.gL == GH_ZERO) return vz(); Ic = 1; if (Cl.gL == GH_PARITY) fac *= sgn; }
  if (I == Cl.nr + 1) { if (Cl.gR == GH_ZERO) return vz(); Ic = Cl.nr; if (Cl.gR == GH_PARITY) fac *= sgn; }
  if (J == 0) { if (Cl.gB == GH_ZERO) return vz(); Jc = 1; if (Cl.gB == GH_PARITY) fac *= sgn; }
  if (J == Cl.nt + 1) { if (Cl.gT == GH_ZERO) return vz(); Jc = Cl.nt; if (Cl.gT == GH_PARITY) fac *= sgn; }
  const V v = erow(sm, tc, h, cur, Jc - 1 - j0c)[Ic - 1];
  return make_float2(fac * v.x, fac * v.y);
}

// e += P e_coarse on the fine rows [rlo, rhi) (own rows and halo rows,
// clipped to the plane), bilinear in (r^2, theta) / (R, z) (Sec. 3.1).
__device__ void t_prolong(const LevelDev& L, const LevelDev& Cl, unsigned char* sm,
                          const TailLevel& tf, const TailLevel& tc, int h, int curf, int curc,
                          int rank, int m) {
  const int nr = L.nr, nt = L.nt, NR = nr + 2, NT = nt + 2;
  const float* rt = L.rf;
  const float* tt = L.tf;
  const int j0 = rank * tf.s, j0c = rank * tc.s;
  const int rlo = max(-h, -j0), rhi = min(tf.s + h, nt - j0);
  const int n = (rhi - rlo) * nr;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int q = idx / nr, i = idx - q * nr, r = rlo + q, j = j0 + r;
    const int i1 = i + 1, j1 = j + 1;
    const int I1 = (i1 & 1) ? (i1 + 1) / 2 - 1 : i1 / 2, J1 = (j1 & 1) ? (j1 + 1) / 2 - 1 : j1 / 2;
    const float p1 = rt[RT_P1 * NR + i1], p2 = rt[RT_P2 * NR + i1];
    const float q1 = tt[TT_P1 * NT + j1], q2 = tt[TT_P2 * NT + j1];
    const V a = t_cval(Cl, sm, tc, h, curc, j0c, I1, J1, m);
    const V b = t_cval(Cl, sm, tc, h, curc, j0c, I1 + 1, J1, m);
    const V c = t_cval(Cl, sm, tc, h, curc, j0c, I1, J1 + 1, m);
    const V d = t_cval(Cl, sm, tc, h, curc, j0c, I1 + 1, J1 + 1, m);
    V* e = erow(sm, tf, h, curf, r) + i;
    V u = *e;
    u.x += p1 * q1 * a.x + p2 * q1 * b.x + p1 * q2 * c.x + p2 * q2 * d.x;
    u.y += p1 * q1 * a.y + p2 * q1 * b.y + p1 * q2 * c.y + p2 * q2 * d.y;
    *e = u;
  }
}

// Exact FP64 solve of the coarsest level (separable form L_m = L_r (x) I +
// D_r (x) L_t, L_t = V diag(lambda) V^-1): the CTA of rank c transforms and
// Thomas-solves its own eigenvalues k, every CTA receives all of z, and each
// back-transforms its own rows and the coarse halo rows its prolongation
// reads.  G: the gathered coarse right-hand side [nt][nr] (all rows).
__device__ void t_coarsest(cg::cluster_group& cl, const TailArgs& a, const LevelDev& Lc,
                           unsigned char* sm, const TailLevel& tc, int h, int cur, int rank,
                           int slot) {
  const int nr = Lc.nr, nt = Lc.nt, nc = nr * nt, C = a.C, sc = tc.s, k0 = rank * sc;
  const V* G = reinterpret_cast<const V*>(sm + a.g_off);
  double2* Z = reinterpret_cast<double2*>(sm + a.z_off);    // [nt][nr], both components
  double2* zl = reinterpret_cast<double2*>(sm + a.zl_off);  // [sc][nr], own eigenvalues
  const double* Fq = a.sep + size_t(slot) * a.sep_stride;
  const int hh = nt / 2, vr = a.sep_sym ? hh : nt;
  const double* Vm = Fq;
  const double* Vi = Vm + vr * nt;
  const double* invd = Vi + nt * vr;
  const double* cp = invd + nt * nr;
  const double* lid = cp + nt * nr;
  (void)nc;
  // z_k = (1/pivot) (V^-1 f)_k for the own k (mirror-symmetric: sums of
  // mirrored rows for even eigenvectors, differences for odd ones)
  for (int q = threadIdx.x; q < 2 * sc * nr; q += blockDim.x) {
    const int c = q / (sc * nr), rq = q - c * sc * nr, kk = rq / nr, i = rq - kk * nr, k = k0 + kk;
    double acc = 0.0;
    for (int j = 0; j < vr; ++j) {
      double fj;
      if (a.sep_sym) {
        const V u = G[j * nr + i], v = G[(nt - 1 - j) * nr + i];
        const double ux = c ? u.y : u.x, vx = c ? v.y : v.x;
        fj = k < hh ? ux + vx : ux - vx;
      } else {
        const V u = G[j * nr + i];
        fj = double(c ? u.y : u.x);
      }
      acc += Vi[k * vr + j] * fj;
    }
    const double zv = acc * invd[k * nr + i];
    if (c) zl[kk * nr + i].y = zv;
    else zl[kk * nr + i].x = zv;
  }
  __syncthreads();
  // Thomas sweeps, one FMA per step each way (2 sc independent systems on
  // the first warp)
  for (int q = threadIdx.x < 32 ? int(threadIdx.x) : 2 * sc; q < 2 * sc; q += 32) {
    const int c = q / sc, kk = q - c * sc, k = k0 + kk;
    double* zz = reinterpret_cast<double*>(zl + kk * nr) + c;   // stride 2
    const double* lk = lid + k * nr;
    const double* ck = cp + k * nr;
    double dp = zz[0];
    for (int i = 1; i < nr; ++i) {
      dp = fma(-lk[i], dp, zz[2 * i]);
      zz[2 * i] = dp;
    }
    double xv = dp;
    for (int i = nr - 2; i >= 0; --i) {
      xv = fma(-ck[i], xv, zz[2 * i]);
      zz[2 * i] = xv;
    }
  }
  __syncthreads();
  // every CTA receives the own z rows
  {
    const int n = sc * nr;
    for (int tgt = 0; tgt < C; ++tgt) {
      double2* zt = cl.map_shared_rank(Z, tgt);
      for (int q = threadIdx.x; q < n; q += blockDim.x) zt[k0 * nr + q] = zl[q];
    }
  }
  cl.sync();
  // e rows [j0c - hb, j0c + sc + hb) within the plane: own rows and the
  // coarse halo the prolongation reads
  const int hb = h / 2 + 1, j0c = rank * sc;
  const int jlo = max(0, j0c - hb), jhi = min(nt, j0c + sc + hb);
  for (int q = threadIdx.x; q < (jhi - jlo) * nr; q += blockDim.x) {
    const int j = jlo + q / nr, i = q - (q / nr) * nr;
    float ex, ey;
    if (a.sep_sym) {
      const int jj = j < hh ? j : nt - 1 - j;
      double Ex = 0.0, Ey = 0.0, Ox = 0.0, Oy = 0.0;
      for (int k = 0; k < hh; ++k) {
        const double vk = Vm[jj * nt + k];
        Ex += vk * Z[k * nr + i].x;
        Ey += vk * Z[k * nr + i].y;
      }
      for (int k = hh; k < nt; ++k) {
        const double vk = Vm[jj * nt + k];
        Ox += vk * Z[k * nr + i].x;
        Oy += vk * Z[k * nr + i].y;
      }
      ex = j < hh ? float(Ex + Ox) : float(Ex - Ox);
      ey = j < hh ? float(Ey + Oy) : float(Ey - Oy);
    } else {
      double ax = 0.0, ay = 0.0;
      for (int k = 0; k < nt; ++k) {
        const double vk = Vm[j * nt + k];
        ax += vk * Z[k * nr + i].x;
        ay += vk * Z[k * nr + i].y;
      }
      ex = float(ax);
      ey = float(ay);
    }
    erow(sm, tc, h, cur, j - j0c)[i] = make_float2(ex, ey);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kTailThreads, 1)
    k_tail(TailArgs a, Batch B, RetireState S, const double2* __restrict__ fg, double2* __restrict__ ug) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ LevelDev sL[8];
  __shared__ D4 red[kTailThreads / 32];
  cg::cluster_group cl = cg::this_cluster();
  const int C = a.C, rank = int(cl.block_rank());
  const int q = int(blockIdx.x) / C;
  if (q >= *B.nact) return;   // uniform over the cluster: no CTA of it synchronises
  const int p = B.act[q];
  const int slot = B.slot ? B.slot[p] : p;
  const int m = B.mode[slot];
  const float s2 = B.s2f[slot];
  const double s2d = B.s2d[slot];
  const int h = a.h, K = a.nlev;
  // this slot's FP32 tables of every level, staged once
  {
    float* tb = reinterpret_cast<float*>(sm + a.tab_off);
    const float4* src = reinterpret_cast<const float4*>(a.tabs + size_t(slot) * a.tab_stride);
    float4* dst = reinterpret_cast<float4*>(tb);
    for (int k = threadIdx.x; k < a.tab_stride / 4; k += blockDim.x) cp_async_v(dst + k, src + k, true);
    if (threadIdx.x < K) {
      const TailLevel& t = a.lv[threadIdx.x];
      LevelDev d = t.L;
      const int NR = d.nr + 2, NT = d.nt + 2;
      d.rf = tb + t.tab;
      d.tf = d.rf + RT_N * NR;
      d.omr_f = d.tf + TT_N * NT;
      d.omt_f = d.omr_f + d.nt;
      sL[threadIdx.x] = d;
    }
  }
  // FP64 solution rows -1 .. s0 of level 0 (own rows and one halo row each side)
  const TailLevel& t0 = a.lv[0];
  const int nr0 = t0.L.nr, nt0 = t0.L.nt, s0 = t0.s, j00 = rank * s0, n0 = nr0 * nt0;
  const size_t base = size_t(p) * n0;
  double2* U = reinterpret_cast<double2*>(sm + a.u_off);
  for (int idx = threadIdx.x; idx < (s0 + 2) * nr0; idx += blockDim.x) {
    const int j = j00 - 1 + idx / nr0, i = idx - (idx / nr0) * nr0;
    U[idx] = (j >= 0 && j < nt0) ? ug[base + size_t(j) * nr0 + i] : make_double2(0.0, 0.0);
  }
  cp_async_wait_all();
  // every CTA of the cluster has started before any writes into a peer's
  // shared memory
  cl.sync();
  int cur[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) cur[l] = 0;
  int it = *S.iter;
  double px = S.nr2[p].x, py = S.nr2[p].y;
  const double2 nf = S.nf2[p];
  const double floor2 = 1e-28 * (*S.fmax2);
  const double tol2 = a.tol * a.tol;
  D4* part = reinterpret_cast<D4*>(sm + a.part_off);
  const double* rd0 = t0.L.rd;
  const int NR0 = nr0 + 2, NT0 = nt0 + 2;
  for (;;) {
    // FP64 residual of the own rows (the defect expression of the
    // level-wide residual kernel), stored as the FP32 right-hand side of
    // level 0; volume-weighted squares accumulated in FP32 per thread
    float ax = 0.f, ay = 0.f;
    {
      const LevelDev& L0 = sL[0];
      V* f0 = frow(sm, t0, h, 0);
      for (int idx = threadIdx.x; idx < s0 * nr0; idx += blockDim.x) {
        const int r = idx / nr0, i = idx - r * nr0, j = j00 + r;
        const double2* ur = U + (r + 1) * nr0;
        const double2 c = ur[i];
        const double2 E = (i + 1 < nr0) ? ur[i + 1] : make_double2(0.0, 0.0);
        const double2 W = (i > 0) ? ur[i - 1] : make_double2(0.0, 0.0);
        const double2 N = (j + 1 < nt0) ? ur[i + nr0] : make_double2(0.0, 0.0);
        const double2 Sv = (j > 0) ? ur[i - nr0] : make_double2(0.0, 0.0);
        const size_t cq = size_t(j) * nr0 + i;
        const double aE = rd0[RT_AE * NR0 + i + 1], aW = rd0[RT_AW * NR0 + i + 1];
        const double aN = a.ctab[cq], aS = a.ctab[n0 + cq];
        const double d = fma(-s2d, a.ctab[3 * size_t(n0) + cq], a.ctab[2 * size_t(n0) + cq]);
        const double2 fv = fg[base + cq];
        const double rx = fv.x - (aE * E.x + aW * W.x + aN * N.x + aS * Sv.x + d * c.x);
        const double ry = fv.y - (aE * E.y + aW * W.y + aN * N.y + aS * Sv.y + d * c.y);
        const V ro = make_float2(float(rx), float(ry));
        f0[idx] = ro;
        const float dv = L0.rf[RT_V * NR0 + i + 1] * L0.tf[TT_V * NT0 + j + 1];
        ax += dv * ro.x * ro.x;
        ay += dv * ro.y * ro.y;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_down_sync(0xffffffffu, ax, o);
      ay += __shfl_down_sync(0xffffffffu, ay, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = D4{ax, ay, 0.0, 0.0};
    __syncthreads();
    if (threadIdx.x < C) {   // the CTA's partial to every CTA of the cluster
      D4 tsum{0.0, 0.0, 0.0, 0.0};
      for (int w = 0; w < int(blockDim.x >> 5); ++w) { tsum.x += red[w].x; tsum.y += red[w].y; }
      *cl.map_shared_rank(part + rank, int(threadIdx.x)) = tsum;
    }
    push_halo(cl, sm, frow(sm, t0, h, 0), s0, nr0, h, t0.fo, t0.fo + (h + s0) * nr0, rank, C);
    cl.sync();
    // App. B criterion, evaluated identically by every thread of the cluster
    double sx = 0.0, sy = 0.0;
    for (int c = 0; c < C; ++c) { sx += part[c].x; sy += part[c].y; }
    int st = TS_ACTIVE;
    if (!isfinite(sx) || !isfinite(sy)) st = TS_NONFINITE;
    else if (sx <= tol2 * fmax(nf.x, floor2) && sy <= tol2 * fmax(nf.y, floor2)) st = TS_OK;
    else if (it >= a.max_cycles) st = TS_NOTCONV;
    else if (a.stagnation && it >= 3 && sx + sy > 0.81 * (px + py)) st = TS_STAGNATED;
    px = sx;
    py = sy;
    if (rank == 0 && threadIdx.x == 0) {
      S.nr2[p] = make_double2(sx, sy);
      S.cycles[p] = it;
      S.status[p] = st;
    }
    if (st != TS_ACTIVE) break;
    // one V-cycle on L e = r from e = 0
    for (int l = 0; l < K - 1; ++l) {
      const TailLevel& t = a.lv[l];
      const LevelDev L = sL[l];
      {
        V* eo = reinterpret_cast<V*>(sm) + t.eo;
        V* eh = reinterpret_cast<V*>(sm) + (cur[l] ? t.eh1 : t.eh0);
        for (int k = threadIdx.x; k < t.s * L.nr; k += blockDim.x) eo[k] = vz();
        for (int k = threadIdx.x; k < 2 * h * L.nr; k += blockDim.x) eh[k] = vz();
      }
      __syncthreads();
      t_smooth(cl, L, sm, t, h, cur[l], rank, C, s2, a.n_sor, t.nu1);
      const TailLevel& tc = a.lv[l + 1];
      const LevelDev Lq = sL[l + 1];
      if (l + 1 < K - 1) {
        V* fo = frow(sm, tc, h, 0);
        t_restrict(L, Lq, sm, t, tc, h, cur[l], rank, s2, fo);
        __syncthreads();
        push_halo(cl, sm, fo, tc.s, Lq.nr, h, tc.fo, tc.fo + (h + tc.s) * Lq.nr, rank, C);
        // the coarse level's first step reads only its own rows; the
        // synchronisation after that step publishes these halo rows
      } else {
        V* G = reinterpret_cast<V*>(sm + a.g_off);
        V* own = G + rank * tc.s * Lq.nr;
        t_restrict(L, Lq, sm, t, tc, h, cur[l], rank, s2, own);
        __syncthreads();
        const int n = tc.s * Lq.nr;
        for (int tgt = 0; tgt < C; ++tgt) {
          if (tgt == rank) continue;
          V* gt = cl.map_shared_rank(G, tgt);
          for (int k = threadIdx.x; k < n; k += blockDim.x) gt[rank * n + k] = own[k];
        }
        cl.sync();
      }
    }
    t_coarsest(cl, a, sL[K - 1], sm, a.lv[K - 1], h, cur[K - 1], rank, slot);
    for (int l = K - 2; l >= 0; --l) {
      const TailLevel& t = a.lv[l];
      const LevelDev L = sL[l];
      t_prolong(L, sL[l + 1], sm, t, a.lv[l + 1], h, cur[l], cur[l + 1], rank, m);
      __syncthreads();
      t_smooth(cl, L, sm, t, h, cur[l], rank, C, s2, a.n_sor, t.nu2);
    }
    // u += e on the own rows and the two halo rows (the halo rows of e are
    // current, so every copy of a row gets the owner's values)
    for (int idx = threadIdx.x; idx < (s0 + 2) * nr0; idx += blockDim.x) {
      const int r = idx / nr0 - 1, i = idx - (idx / nr0) * nr0, j = j00 + r;
      if (j < 0 || j >= nt0) continue;
      const V v = erow(sm, t0, h, cur[0], r)[i];
      double2 x = U[idx];
      x.x += double(v.x);
      x.y += double(v.y);
      U[idx] = x;
    }
    __syncthreads();
    ++it;
  }
  for (int idx = threadIdx.x; idx < s0 * nr0; idx += blockDim.x)
    ug[base + size_t(j00) * nr0 + idx] = U[nr0 + idx];
  if (rank == 0 && threadIdx.x == 0) {
    // the solve's iteration count is the largest over the planes; the last
    // cluster to finish folds it into the counter and clears the scratch
    atomicMax(a.titer, it + 1);
    __threadfence();
    if (atomicAdd(a.tdone, 1) == *B.nact - 1) {
      __threadfence();
      const int tmax = atomicAdd(a.titer, 0);
      if (tmax > *S.iter) *S.iter = tmax;
      *a.titer = 0;
      *a.tdone = 0;
    }
  }
  cl.sync();   // no CTA leaves while a peer could still address its shared memory
}

}  // namespace

// The kernel's attributes are process-wide: opt in once to the largest
// dynamic shared memory its static usage leaves, so that no handle's set-up
// lowers the limit below another handle's launch size.
static int tail_attributes() {
  static const int max_dyn = [] {   // thread-safe one-time set-up
    int got = 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_tail) == cudaSuccess) {
      const int want = int(227 * 1024 - fa.sharedSizeBytes);
      if (cudaFuncSetAttribute(k_tail, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
          cudaFuncSetAttribute(k_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, want) == cudaSuccess)
        got = want;
    }
    cudaGetLastError();
    return got;
  }();
  return max_dyn;
}

int tail_max_clusters(const TailArgs& a) {
  if (int(a.smem_bytes) > tail_attributes()) return 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(a.C);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(unsigned(a.C));
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = a.smem_bytes;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_tail, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

void launch_tail(const TailArgs& a, const Batch& B, const RetireState& S, const double2* f,
                 double2* u, int clusters, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(a.C);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(unsigned(a.C * clusters));
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = a.smem_bytes;
  cfg.stream = st;
  cudaLaunchKernelEx(&cfg, k_tail, a, B, S, f, u);
}

}  // namespace ps
