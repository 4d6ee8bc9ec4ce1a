// The lower part of a V-cycle (Sec. 3) in one kernel: one block per mode
// plane keeps the error and right-hand side of every level from `first`
// down to the coarsest in shared memory and runs smoothing (the same
// alternating zebra line relaxation), defect restriction, the coarsest
// exact solve, prolongation and post-smoothing with block barriers instead
// of kernel boundaries.  Input f[first] and output e[first] live in global
// memory.  The coarsest level is solved directly: in FP64 by the FP64
// kernel; a separable coarsest level in FP32 by the FP32 kernel, with factors
// computed in FP64 on the host (coarsest_f32c).
//
// Shared-memory layout of a level (nr x nt, unpadded rows): cell (j, i) sits
// at j * nr + (i ^ h(j)).  The row swizzle h(j) < min(16, nr) follows the
// rows a half-warp holds in a polar line (pairs of rows or single rows):
// (j >> 1) or j, doubled for FP32 planes so that the two cells of an aligned
// pair (16 bytes, one bank group) stay together.  Row-wise vector accesses of
// radial lines and the column accesses of polar lines (pairs of columns for
// FP32) are then free of bank conflicts.
#include <cstdio>
#include <type_traits>

#include "lines.cuh"

namespace ps {

#define R_(id, i) rt[(id) * (L.nr + 2) + (i)]
#define T_(id, j) tt[(id) * (L.nt + 2) + (j)]

template <typename T>
__device__ __forceinline__ int vswz(const LevelDev& L, int j) {
  const int mask = (L.nr < 16 ? L.nr : 16) - 1;
  const int x = L.nt > 32 ? j >> 1 : j;
  if constexpr (sizeof(T) == 4) return (x << 1) & mask;
  else return x & mask;
}
template <typename T>
__device__ __forceinline__ int vslot(const LevelDev& L, int j, int i) {
  return j * L.nr + (i ^ vswz<T>(L, j));
}

template <typename T, int CPL>
__device__ void s_rlines(const LevelDev& L, vec2_t<T>* e, const vec2_t<T>* f, T s2, int n_sor,
                         int color) {
  typedef vec2_t<T> V;
  const int nr = L.nr, nt = L.nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const T* rt = rt_<T>(L);
  const T* tt = tt_<T>(L);
  const T* om = omr_<T>(L);
  // the same for every radial line of the level: loaded once (FP32; the
  // FP64 kernel reloads them per line to stay within its registers)
  RLineTabs<T, CPL> tabs;
  if constexpr (sizeof(T) == 4) ld_rtabs<T, CPL>(tabs, L, rt);
  for (int line = warp; 2 * line + color < nt; line += nw) {
    const int j = 2 * line + color;
    const int sj = vswz<T>(L, j);
    V ev[CPL], g[CPL], un[CPL], us[CPL];
    ld_line_swz<V, CPL>(ev, e + j * nr, sj, lane, nr);
    ld_line_swz<V, CPL>(g, f + j * nr, sj, lane, nr);
    if (j + 1 < nt) {
      ld_line_swz<V, CPL>(un, e + (j + 1) * nr, vswz<T>(L, j + 1), lane, nr);
    } else {
#pragma unroll
      for (int c = 0; c < CPL; ++c) un[c] = z2<V>();
    }
    if (j > 0) {
      ld_line_swz<V, CPL>(us, e + (j - 1) * nr, vswz<T>(L, j - 1), lane, nr);
    } else {
#pragma unroll
      for (int c = 0; c < CPL; ++c) us[c] = z2<V>();
    }
    if constexpr (sizeof(T) == 4) relax_r<T, CPL>(L, tabs, tt, s2, om[j], j, g, un, us, n_sor, ev);
    else relax_r<T, CPL>(L, rt, tt, s2, om[j], j, g, un, us, n_sor, ev);
    st_line_swz<V, CPL>(e + j * nr, sj, ev, lane, nr);
  }
}

template <typename T, int CPL>
__device__ void s_tcols(const LevelDev& L, vec2_t<T>* e, const vec2_t<T>* f, T s2, int n_sor,
                        int color) {
  typedef vec2_t<T> V;
  const int nr = L.nr, nt = L.nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const T* rt = rt_<T>(L);
  const T* tt = tt_<T>(L);
  const T* om = omt_<T>(L);
  const bool on = CPL > 1 || lane < nt;
  TLineTabs<T, CPL> tabs;   // the same for every polar line of the level (FP32: loaded once)
  if constexpr (sizeof(T) == 4) ld_ttabs<T, CPL>(tabs, L, tt);
  for (int col = warp; 2 * col + color < nr; col += nw) {
    const int i = 2 * col + color;
    V ev[CPL], g[CPL], ue[CPL], uw[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      ev[c] = g[c] = ue[c] = uw[c] = z2<V>();
      if (on) {
        const int j = lcell<CPL>(lane, c), row = j * nr, s = vswz<T>(L, j);
        ev[c] = e[row + (i ^ s)];
        g[c] = f[row + (i ^ s)];
        if (i > 0) uw[c] = e[row + ((i - 1) ^ s)];
        if (i + 1 < nr) ue[c] = e[row + ((i + 1) ^ s)];
      }
    }
    if constexpr (sizeof(T) == 4) relax_t<T, CPL>(L, rt, tabs, s2, om[i], i, g, ue, uw, n_sor, ev);
    else relax_t<T, CPL>(L, rt, tt, s2, om[i], i, g, ue, uw, n_sor, ev);
    if (on) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = lcell<CPL>(lane, c);
        e[j * nr + (i ^ vswz<T>(L, j))] = ev[c];
      }
    }
  }
}

// ---- FP32 band smoothing ----------------------------------------------------
// Both colours of one direction as a band per warp: warp w owns lines
// w B .. w B + B - 1 (B = lines / warps, even).  It relaxes the band's even
// (first-colour) lines, then its odd lines but the last, keeping every line
// it touches in registers; the last odd line needs the first even line of the
// band above, so it waits for a block barrier.  The band's first even line is
// stored before that barrier (the band below needs it for its last odd line).
// Each line relaxation receives exactly the operands of the line-by-line
// schedule (the lines of one colour are independent), so the results are
// bitwise the same; a line is loaded once per half-cycle instead of up to
// three times, and polar columns move as 16-byte pairs.

// Row j of an FP32 level held as the lane's cells (even swizzle s: pairs stay
// whole).
template <int CPL>
__device__ __forceinline__ void b_ld_row(float2 (&d)[CPL], const float2* row, int s, int lane) {
  if constexpr (CPL == 1) {
    d[0] = row[lane ^ s];
  } else {
#pragma unroll
    for (int q = 0; q < CPL / 2; ++q) ld_pair(d[2 * q], d[2 * q + 1], row + ((2 * lane + 64 * q) ^ s));
  }
}
template <int CPL>
__device__ __forceinline__ void b_st_row(float2* row, int s, const float2 (&d)[CPL], int lane) {
  if constexpr (CPL == 1) {
    row[lane ^ s] = d[0];
  } else {
#pragma unroll
    for (int q = 0; q < CPL / 2; ++q) st_pair(row + ((2 * lane + 64 * q) ^ s), d[2 * q], d[2 * q + 1]);
  }
}
template <int CPL>
__device__ __forceinline__ void b_zero(float2 (&d)[CPL]) {
#pragma unroll
  for (int c = 0; c < CPL; ++c) d[c] = make_float2(0.f, 0.f);
}

// Radial lines (rows), nr = 32 CPL, nt = B * warps.  Order: even row j0,
// then per k the even row j0 + 2k and the odd row j0 + 2k - 1 below it, each
// row stored once final; the last odd row after the barrier.  The rows move
// through a window of registers in a loop, so the code holds four line
// relaxations whatever B (the instruction cache is the kernel's limit).
template <int CPL, int B>
__device__ __forceinline__ void band_r(const LevelDev& L, float2* e, const float2* f, float s2,
                                       int n_sor) {
  const int nr = L.nr, nt = L.nt, lane = threadIdx.x & 31;
  const int j0 = (threadIdx.x >> 5) * B;
  const float* tt = L.tf;
  const float* om = L.omr_f;
  RLineTabs<float, CPL> tabs;
  ld_rtabs<float, CPL>(tabs, L, L.rf);
  auto ld = [&](float2 (&d)[CPL], const float2* a, int j) { b_ld_row<CPL>(d, a + j * nr, vswz<float>(L, j), lane); };
  auto relax = [&](int j, float2 (&un)[CPL], float2 (&us)[CPL], float2 (&ev)[CPL]) {
    float2 g[CPL];
    ld(g, f, j);
    relax_r<float, CPL>(L, tabs, tt, s2, om[j], j, g, un, us, n_sor, ev);
    b_st_row<CPL>(e + j * nr, vswz<float>(L, j), ev, lane);
  };
  // P: the even row j0 + 2k - 2 (relaxed), Q: the odd row j0 + 2k - 1
  float2 M[CPL], P[CPL], Q[CPL];
  if (j0 > 0) ld(M, e, j0 - 1);
  else b_zero<CPL>(M);
  ld(P, e, j0);
  ld(Q, e, j0 + 1);
  relax(j0, Q, M, P);
  if constexpr (B > 2) {
#pragma unroll 1
    for (int k = 1; k < B / 2; ++k) {
      float2 R[CPL], S[CPL];
      ld(R, e, j0 + 2 * k);
      ld(S, e, j0 + 2 * k + 1);
      relax(j0 + 2 * k, S, Q, R);
      relax(j0 + 2 * k - 1, R, P, Q);
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        P[c] = R[c];
        Q[c] = S[c];
      }
    }
  }
  __syncthreads();
  float2 A[CPL];
  if (j0 + B < nt) ld(A, e, j0 + B);
  else b_zero<CPL>(A);
  relax(j0 + B - 1, A, P, Q);
}

// Polar lines (columns), nt = 32 CPL, nr = B * warps; the lane's cells are the
// rows lcell(lane, c).  Same order and window as the rows; the two columns of
// a pair are stored together once both are final (column i0 alone when
// B = 2: the band to the left reads it after the barrier).
template <int CPL, int B>
__device__ __forceinline__ void band_t(const LevelDev& L, float2* e, const float2* f, float s2,
                                       int n_sor) {
  const int nr = L.nr, lane = threadIdx.x & 31;
  const int i0 = (threadIdx.x >> 5) * B;
  const float* rt = L.rf;
  const float* om = L.omt_f;
  TLineTabs<float, CPL> tabs;
  ld_ttabs<float, CPL>(tabs, L, L.tf);
  int base[CPL], sw[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int j = lcell<CPL>(lane, c);
    base[c] = j * nr;
    sw[c] = vswz<float>(L, j);
  }
  auto ld_col = [&](float2 (&d)[CPL], int i) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) d[c] = e[base[c] + (i ^ sw[c])];
  };
  auto ld_pr = [&](float2 (&x)[CPL], float2 (&y)[CPL], const float2* a, int i) {   // columns i, i + 1
#pragma unroll
    for (int c = 0; c < CPL; ++c) ld_pair(x[c], y[c], a + base[c] + (i ^ sw[c]));
  };
  auto st_pr = [&](const float2 (&x)[CPL], const float2 (&y)[CPL], int i) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) st_pair(e + base[c] + (i ^ sw[c]), x[c], y[c]);
  };
  auto relax = [&](int i, float2 (&g)[CPL], float2 (&ue)[CPL], float2 (&uw)[CPL], float2 (&ev)[CPL]) {
    relax_t<float, CPL>(L, rt, tabs, s2, om[i], i, g, ue, uw, n_sor, ev);
  };
  // P, Q: the columns i0 + 2k - 2 (relaxed) and i0 + 2k - 1; gQ: Q's right-hand side
  float2 M[CPL], P[CPL], Q[CPL], gP[CPL], gQ[CPL];
  if (i0 > 0) ld_col(M, i0 - 1);
  else b_zero<CPL>(M);
  ld_pr(P, Q, e, i0);
  ld_pr(gP, gQ, f, i0);
  relax(i0, gP, Q, M, P);
  if constexpr (B == 2) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) e[base[c] + (i0 ^ sw[c])] = P[c];
  } else {
#pragma unroll 1
    for (int k = 1; k < B / 2; ++k) {
      const int i = i0 + 2 * k;
      float2 R[CPL], S[CPL], gR[CPL], gS[CPL];
      ld_pr(R, S, e, i);
      ld_pr(gR, gS, f, i);
      relax(i, gR, S, Q, R);
      relax(i - 1, gQ, R, P, Q);
      st_pr(P, Q, i - 2);
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        P[c] = R[c];
        Q[c] = S[c];
        gQ[c] = gS[c];
      }
    }
  }
  __syncthreads();
  float2 A[CPL];
  if (i0 + B < nr) ld_col(A, i0 + B);
  else b_zero<CPL>(A);
  relax(i0 + B - 1, gQ, A, P, Q);
  if constexpr (B == 2) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) e[base[c] + ((i0 + 1) ^ sw[c])] = Q[c];
  } else {
    st_pr(P, Q, i0 + B - 2);
  }
}

// Lines of n = 32, 64 or 128 cells (lanes x CPL) in bands of B = m / 16 lines
// for m = 32, 64 or 128 lines, with B CPL <= 16 (registers): the band kind
// (CPL, B) as 3 * log2(CPL) + log2(B / 2), or -1 when the level takes the
// line-by-line schedule.
__device__ __forceinline__ int band_kind(int n, int m, int nw) {
  if (nw != 16 || (n != 32 && n != 64 && n != 128) || (m != 32 && m != 64 && m != 128)) return -1;
  const int cpl = n / 32, b = m / 16;
  if (cpl * b > 16) return -1;
  return 3 * (cpl == 1 ? 0 : cpl == 2 ? 1 : 2) + (b == 2 ? 0 : b == 4 ? 1 : 2);
}

__device__ __forceinline__ void band_r_any(int kind, const LevelDev& L, float2* e, const float2* f,
                                           float s2, int n_sor) {
  switch (kind) {
    case 0: band_r<1, 2>(L, e, f, s2, n_sor); break;
    case 1: band_r<1, 4>(L, e, f, s2, n_sor); break;
    case 2: band_r<1, 8>(L, e, f, s2, n_sor); break;
    case 3: band_r<2, 2>(L, e, f, s2, n_sor); break;
    case 4: band_r<2, 4>(L, e, f, s2, n_sor); break;
    case 5: band_r<2, 8>(L, e, f, s2, n_sor); break;
    case 6: band_r<4, 2>(L, e, f, s2, n_sor); break;
    default: band_r<4, 4>(L, e, f, s2, n_sor); break;
  }
}
__device__ __forceinline__ void band_t_any(int kind, const LevelDev& L, float2* e, const float2* f,
                                           float s2, int n_sor) {
  switch (kind) {
    case 0: band_t<1, 2>(L, e, f, s2, n_sor); break;
    case 1: band_t<1, 4>(L, e, f, s2, n_sor); break;
    case 2: band_t<1, 8>(L, e, f, s2, n_sor); break;
    case 3: band_t<2, 2>(L, e, f, s2, n_sor); break;
    case 4: band_t<2, 4>(L, e, f, s2, n_sor); break;
    case 5: band_t<2, 8>(L, e, f, s2, n_sor); break;
    case 6: band_t<4, 2>(L, e, f, s2, n_sor); break;
    default: band_t<4, 4>(L, e, f, s2, n_sor); break;
  }
}

// `cycles` alternating-line smoothing cycles of a level held in shared memory
// (L's table and omega pointers point at shared-memory copies; the omega
// rows are those of this block's mode).
template <typename T>
__device__ __noinline__ void s_smooth(const LevelDev& L, vec2_t<T>* e, const vec2_t<T>* f, T s2, int cycles,
                         int n_sor) {
  const int cr = L.nr <= 32 ? 1 : L.nr / 32, ct = L.nt <= 32 ? 1 : L.nt / 32;
  if constexpr (sizeof(T) == 4) {
    const int nw = blockDim.x >> 5;
    const int kr = band_kind(L.nr, L.nt, nw), kt = band_kind(L.nt, L.nr, nw);
    if (kr >= 0 && kt >= 0) {
      for (int cyc = 0; cyc < cycles; ++cyc) {
        band_r_any(kr, L, e, f, s2, n_sor);
        __syncthreads();
        band_t_any(kt, L, e, f, s2, n_sor);
        __syncthreads();
      }
      return;
    }
  }
  for (int cyc = 0; cyc < cycles; ++cyc) {
    for (int color = 0; color < 2; ++color) {
      if (cr == 1) s_rlines<T, 1>(L, e, f, s2, n_sor, color);
      else if (cr == 2) s_rlines<T, 2>(L, e, f, s2, n_sor, color);
      else s_rlines<T, 4>(L, e, f, s2, n_sor, color);
      __syncthreads();
    }
    for (int color = 0; color < 2; ++color) {
      if (ct == 1) s_tcols<T, 1>(L, e, f, s2, n_sor, color);
      else if (ct == 2) s_tcols<T, 2>(L, e, f, s2, n_sor, color);
      else s_tcols<T, 4>(L, e, f, s2, n_sor, color);
      __syncthreads();
    }
  }
}

template <typename T>
__device__ void s_restrict(const LevelDev& L, const LevelDev& C, const vec2_t<T>* e,
                           const vec2_t<T>* f, vec2_t<T>* fc, T s2) {
  typedef vec2_t<T> V;
  const int nr = L.nr, nt = L.nt;
  const T* rt = rt_<T>(L);
  const T* tt = tt_<T>(L);
  for (RowWalk w(threadIdx.x, blockDim.x, C.nr); w.j < C.nt; w.next()) {
    const int J = w.j, I = w.c;
    T ax = 0, ay = 0;
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int i = 2 * I + a, j = 2 * J + b;
        const V c = e[vslot<T>(L, j, i)];
        const V E = (i + 1 < nr) ? e[vslot<T>(L, j, i + 1)] : V{0, 0};
        const V W = (i > 0) ? e[vslot<T>(L, j, i - 1)] : V{0, 0};
        const V N = (j + 1 < nt) ? e[vslot<T>(L, j + 1, i)] : V{0, 0};
        const V S = (j > 0) ? e[vslot<T>(L, j - 1, i)] : V{0, 0};
        const T aE = R_(RT_AE, i + 1), aW = R_(RT_AW, i + 1), P = R_(RT_P, i + 1);
        const T aN = P * T_(TT_AN, j + 1), aS = P * T_(TT_AS, j + 1);
        const T d = fmac(-(s2 * R_(RT_Q, i + 1)), T_(TT_T, j + 1), fmac(P, T_(TT_DT, j + 1), R_(RT_DR, i + 1)));
        const V fv = f[vslot<T>(L, j, i)];
        const T rx = fv.x - fmac(d, c.x, fmac(aS, S.x, fmac(aN, N.x, fmac(aW, W.x, aE * E.x))));
        const T ry = fv.y - fmac(d, c.y, fmac(aS, S.y, fmac(aN, N.y, fmac(aW, W.y, aE * E.y))));
        const T wgt = R_(RT_RW, i + 1) * T_(TT_RW, j + 1);
        ax = fmac(wgt, rx, ax);
        ay = fmac(wgt, ry, ay);
      }
    fc[vslot<T>(C, J, I)] = V{ax, ay};
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ vec2_t<T> s_cval(const LevelDev& C, const vec2_t<T>* ec, int I, int J, int m) {
  typedef vec2_t<T> V;
  T fac = T(1);
  const T sgn = (m & 1) ? T(-1) : T(1);
  int Ic = I, Jc = J;
  if (I == 0) { if (C.gL == GH_ZERO) return V{0, 0}; Ic = 1; if (C.gL == GH_PARITY) fac *= sgn; }
  if (I == C.nr + 1) { if (C.gR == GH_ZERO) return V{0, 0}; Ic = C.nr; if (C.gR == GH_PARITY) fac *= sgn; }
  if (J == 0) { if (C.gB == GH_ZERO) return V{0, 0}; Jc = 1; if (C.gB == GH_PARITY) fac *= sgn; }
  if (J == C.nt + 1) { if (C.gT == GH_ZERO) return V{0, 0}; Jc = C.nt; if (C.gT == GH_PARITY) fac *= sgn; }
  const V v = ec[vslot<T>(C, Jc - 1, Ic - 1)];
  return V{fac * v.x, fac * v.y};
}

// e += P ec (bilinear, Sec. 3.1): one thread per coarse cell (I, J) updates
// its four children (2I + a, 2J + b) from the 3 x 3 coarse neighbourhood;
// child a uses coarse columns I - 1 + a, I + a, child b rows J - 1 + b, J + b.
template <typename T>
__device__ void s_prolong(const LevelDev& L, const LevelDev& C, vec2_t<T>* e, const vec2_t<T>* ec, int m) {
  typedef vec2_t<T> V;
  const T* rt = rt_<T>(L);
  const T* tt = tt_<T>(L);
  for (RowWalk w(threadIdx.x, blockDim.x, C.nr); w.j < C.nt; w.next()) {
    const int J = w.j, I = w.c;
    V cv[3][3];   // coarse (I - 1 + u, J - 1 + v), 1-based index I + u, J + v
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int u = 0; u < 3; ++u) cv[v][u] = s_cval<T>(C, ec, I + u, J + v, m);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int j = 2 * J + b;
      const T q1 = T_(TT_P1, j + 1), q2 = T_(TT_P2, j + 1);
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int i = 2 * I + a;
        const T p1 = R_(RT_P1, i + 1), p2 = R_(RT_P2, i + 1);
        const V A = cv[b][a], Bv = cv[b][a + 1], Cv = cv[b + 1][a], D = cv[b + 1][a + 1];
        V u = e[vslot<T>(L, j, i)];
        const T w11 = p1 * q1, w21 = p2 * q1, w12 = p1 * q2, w22 = p2 * q2;
        u.x += fmac(w22, D.x, fmac(w12, Cv.x, fmac(w21, Bv.x, w11 * A.x)));
        u.y += fmac(w22, D.y, fmac(w12, Cv.y, fmac(w21, Bv.y, w11 * A.y)));
        e[vslot<T>(L, j, i)] = u;
      }
    }
  }
  __syncthreads();
}

// ---- FP32 restriction and prolongation with vector accesses ---------------
// The same formulas, operands and order of operations as s_restrict and
// s_prolong (so the same results); a coarse cell's two fine columns
// 2I, 2I + 1 form an aligned pair (one 16-byte access per fine row, even
// swizzle), and so do the table entries of two neighbouring cells (one
// 8-byte access).  Needs an even number of fine columns and rows.

__device__ __forceinline__ float2 tab2(const float* t, int id, int n, int i) {   // entries of cells i, i + 1
  return *reinterpret_cast<const float2*>(t + id * (n + 2) + i + 1);
}

__device__ void s_restrict_f32(const LevelDev& L, const LevelDev& C, const float2* e, const float2* f,
                               float2* fc, float s2) {
  const int nr = L.nr, nt = L.nt;
  const float* rt = L.rf;
  const float* tt = L.tf;
  const float2 z = make_float2(0.f, 0.f);
  for (RowWalk w(threadIdx.x, blockDim.x, C.nr); w.j < C.nt; w.next()) {
    const int J = w.j, I = w.c, i0 = 2 * I, j0 = 2 * J;
    // e on rows j0 - 1 .. j0 + 2 at columns i0, i0 + 1; the W and E neighbours on rows j0, j0 + 1
    float2 r[4][2], W[2], E[2], fv[2][2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 - 1 + q;
      if (j >= 0 && j < nt) ld_pair(r[q][0], r[q][1], e + vslot<float>(L, j, i0));
      else r[q][0] = r[q][1] = z;
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int j = j0 + b;
      W[b] = i0 > 0 ? e[vslot<float>(L, j, i0 - 1)] : z;
      E[b] = i0 + 2 < nr ? e[vslot<float>(L, j, i0 + 2)] : z;
      ld_pair(fv[b][0], fv[b][1], f + vslot<float>(L, j, i0));
    }
    const float2 AE = tab2(rt, RT_AE, nr, i0), AW = tab2(rt, RT_AW, nr, i0), PP = tab2(rt, RT_P, nr, i0);
    const float2 DR = tab2(rt, RT_DR, nr, i0), QQ = tab2(rt, RT_Q, nr, i0), RW = tab2(rt, RT_RW, nr, i0);
    const float2 AN = tab2(tt, TT_AN, nt, j0), AS = tab2(tt, TT_AS, nt, j0), DT = tab2(tt, TT_DT, nt, j0);
    const float2 TT2 = tab2(tt, TT_T, nt, j0), TW = tab2(tt, TT_RW, nt, j0);
    float ax = 0, ay = 0;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const float2 c = r[b + 1][a];
        const float2 Ev = a ? E[b] : r[b + 1][1];
        const float2 Wv = a ? r[b + 1][0] : W[b];
        const float2 N = r[b + 2][a], S = r[b][a];
        const float aE = a ? AE.y : AE.x, aW = a ? AW.y : AW.x, P = a ? PP.y : PP.x;
        const float aN = P * (b ? AN.y : AN.x), aS = P * (b ? AS.y : AS.x);
        const float d = fmac(-(s2 * (a ? QQ.y : QQ.x)), b ? TT2.y : TT2.x, fmac(P, b ? DT.y : DT.x, a ? DR.y : DR.x));
        const float rx = fv[b][a].x - fmac(d, c.x, fmac(aS, S.x, fmac(aN, N.x, fmac(aW, Wv.x, aE * Ev.x))));
        const float ry = fv[b][a].y - fmac(d, c.y, fmac(aS, S.y, fmac(aN, N.y, fmac(aW, Wv.y, aE * Ev.y))));
        const float wgt = (a ? RW.y : RW.x) * (b ? TW.y : TW.x);
        ax = fmac(wgt, rx, ax);
        ay = fmac(wgt, ry, ay);
      }
    fc[vslot<float>(C, J, I)] = make_float2(ax, ay);
  }
  __syncthreads();
}

__device__ void s_prolong_f32(const LevelDev& L, const LevelDev& C, float2* e, const float2* ec, int m) {
  const float* rt = L.rf;
  const float* tt = L.tf;
  const int nr = L.nr, nt = L.nt;
  // each task: coarse column I, coarse rows J0 .. J0 + S - 1 (neighbourhood
  // rows J0 - 1 .. J0 + S loaded once); the ghost rules of s_cval chosen per
  // column and row without branching (the same values: zero, the mirrored
  // cell, or its negative for odd m across a parity face, twice negated
  // across two)
  constexpr int S = 4;
  const bool odd = (m & 1) != 0;
  const int strips = (C.nt + S - 1) / S;
  for (int t = threadIdx.x; t < C.nr * strips; t += blockDim.x) {
    const int I = t % C.nr, J0 = (t / C.nr) * S;
    int ic[3];
    bool zc[3], nc[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {   // 1-based coarse column I + u
      const int x = I + u, rule = x == 0 ? C.gL : (x == C.nr + 1 ? C.gR : -1);
      ic[u] = min(max(x, 1), C.nr) - 1;
      zc[u] = rule == GH_ZERO;
      nc[u] = rule == GH_PARITY && odd;
    }
    float2 r[S + 2][3];   // 1-based coarse rows J0 .. J0 + S + 1
#pragma unroll
    for (int v = 0; v < S + 2; ++v) {
      const int y = J0 + v, rule = y == 0 ? C.gB : (y == C.nt + 1 ? C.gT : -1);
      const int jc = min(max(y, 1), C.nt) - 1;
      const bool zr = rule == GH_ZERO, nrw = rule == GH_PARITY && odd;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const float2 x = ec[vslot<float>(C, jc, ic[u])];
        r[v][u] = (zc[u] || zr) ? make_float2(0.f, 0.f) : ((nc[u] != nrw) ? make_float2(-x.x, -x.y) : x);
      }
    }
    const int i0 = 2 * I;
    const float2 P1 = tab2(rt, RT_P1, nr, i0), P2 = tab2(rt, RT_P2, nr, i0);
#pragma unroll
    for (int q = 0; q < S; ++q) {
      const int J = J0 + q;
      if (J >= C.nt) break;
      const float2 Q1 = tab2(tt, TT_P1, nt, 2 * J), Q2 = tab2(tt, TT_P2, nt, 2 * J);
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int j = 2 * J + b;
        const float q1 = b ? Q1.y : Q1.x, q2 = b ? Q2.y : Q2.x;
        float2 uu[2];
        float2* row = e + vslot<float>(L, j, i0);
        ld_pair(uu[0], uu[1], row);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const float p1 = a ? P1.y : P1.x, p2 = a ? P2.y : P2.x;
          const float2 A = r[q + b][a], Bv = r[q + b][a + 1], Cv = r[q + b + 1][a], D = r[q + b + 1][a + 1];
          const float w11 = p1 * q1, w21 = p2 * q1, w12 = p1 * q2, w22 = p2 * q2;
          uu[a].x += fmac(w22, D.x, fmac(w12, Cv.x, fmac(w21, Bv.x, w11 * A.x)));
          uu[a].y += fmac(w22, D.y, fmac(w12, Cv.y, fmac(w21, Bv.y, w11 * A.y)));
        }
        st_pair(row, uu[0], uu[1]);
      }
    }
  }
  __syncthreads();
}

// ---- separable coarsest level of the FP32 V-cycle --------------------------
// L_m = L_r (x) I + D_r (x) L_t with L_t = V diag(lambda) V^-1 (Sec. 3.3
// allows any direct solver).  The FP32 V-cycle solves it in FP32 throughout,
// with factors computed in FP64 on the host and rounded once: a coarse
// correction only needs the solve of an operator close to the coarse one
// (the rounding acts as a relative perturbation of order 1e-6, far inside
// what leaves the V-cycle's contraction unchanged).
// Factor block per slot (sepf, sepf_stride floats): V^-1 transposed
// [vr][nt] (row j: V^-1[k][j] over k), V transposed [nt][vr] (row k: V[j][k]
// over j < vr), then 1/pivot, upper/pivot and lower/pivot [nt][nr + 1]
// (rows padded by one entry, so that the lanes of the radial sweeps, one
// eigenvalue k each, fall in different banks); vr = nt / 2 in the
// mirror-symmetric form (rows j < nt / 2 of V, columns j < nt / 2 of V^-1),
// else nt.  The scratch z has the same padded rows.

__device__ __forceinline__ void stage_f32c(const VSmemArgs& a, int slot, unsigned char* vraw) {
  const float4* fs = reinterpret_cast<const float4*>(a.sepf + size_t(slot) * a.sepf_stride);
  float4* fd = reinterpret_cast<float4*>(vraw + a.blk_off);
  for (int k = threadIdx.x; k < a.sepf_stride / 4; k += blockDim.x) cp_async_v(fd + k, fs + k, true);
}

// KB consecutive entries of a factor row starting at p (16-byte aligned for KB = 4).
template <int KB>
__device__ __forceinline__ void ld_kb(float (&w)[KB], const float* p) {
  if constexpr (KB == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else {
#pragma unroll
    for (int q = 0; q < KB; ++q) w[q] = p[q];
  }
}

// z = (1/pivot) .* ((V^-1 (x) I) f): each task takes KB eigenvalues k0 .. of
// one part (mirror-symmetric: sums f_j + f_{nt-1-j} for the even
// eigenvectors k < nt/2, differences for the odd ones) at one radial index,
// both components, so every f value it loads feeds 2 KB products.
template <int KB>
__device__ void f32c_forward(const LevelDev& Lc, const float2* fc, const float* ViT, const float* invd,
                             float* z, bool sym) {
  const int nr = Lc.nr, nt = Lc.nt, P = nr + 1, nc = P * nt, h = nt / 2, vr = sym ? h : nt;
  const int kper = sym ? h : nt, nkb = kper / KB, ntask = (sym ? 2 : 1) * nr * nkb;
  for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
    const int i = t % nr, rest = t / nr, kb = rest % nkb, part = rest / nkb;
    const int k0 = part * h + kb * KB;
    float ax[KB], ay[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) ax[q] = ay[q] = 0.f;
    for (int j = 0; j < vr; ++j) {
      float2 s = fc[vslot<float>(Lc, j, i)];
      if (sym) {
        const float2 v = fc[vslot<float>(Lc, nt - 1 - j, i)];
        s = part ? make_float2(s.x - v.x, s.y - v.y) : make_float2(s.x + v.x, s.y + v.y);
      }
      float w[KB];
      ld_kb<KB>(w, ViT + j * nt + k0);
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        ax[q] = fmaf(w[q], s.x, ax[q]);
        ay[q] = fmaf(w[q], s.y, ay[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int k = k0 + q;
      const float d = invd[k * P + i];
      z[k * P + i] = ax[q] * d;
      z[nc + k * P + i] = ay[q] * d;
    }
  }
}

// e = (V (x) I) x: each task takes JB rows j0 .. (mirror-symmetric: j < nt/2,
// writing e_j = E + O and e_{nt-1-j} = E - O from the even and odd
// eigenvector parts) at one radial index, both components.
template <int JB>
__device__ void f32c_back(const LevelDev& Lc, const float* z, const float* VT, float2* ec, bool sym) {
  const int nr = Lc.nr, nt = Lc.nt, P = nr + 1, nc = P * nt, h = nt / 2, vr = sym ? h : nt;
  const int njb = vr / JB, ntask = nr * njb;
  for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
    const int i = t % nr, j0 = (t / nr) * JB;
    float ex[JB], ey[JB], ox[JB], oy[JB];
#pragma unroll
    for (int q = 0; q < JB; ++q) ex[q] = ey[q] = ox[q] = oy[q] = 0.f;
    const int ke = sym ? h : nt;
    for (int k = 0; k < ke; ++k) {
      const float xr = z[k * P + i], xi = z[nc + k * P + i];
      float w[JB];
      ld_kb<JB>(w, VT + k * vr + j0);
#pragma unroll
      for (int q = 0; q < JB; ++q) {
        ex[q] = fmaf(w[q], xr, ex[q]);
        ey[q] = fmaf(w[q], xi, ey[q]);
      }
    }
    if (sym) {
      for (int k = h; k < nt; ++k) {
        const float xr = z[k * P + i], xi = z[nc + k * P + i];
        float w[JB];
        ld_kb<JB>(w, VT + k * vr + j0);
#pragma unroll
        for (int q = 0; q < JB; ++q) {
          ox[q] = fmaf(w[q], xr, ox[q]);
          oy[q] = fmaf(w[q], xi, oy[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < JB; ++q) {
      const int j = j0 + q;
      ec[vslot<float>(Lc, j, i)] = make_float2(ex[q] + ox[q], ey[q] + oy[q]);
      if (sym) ec[vslot<float>(Lc, nt - 1 - j, i)] = make_float2(ex[q] - ox[q], ey[q] - oy[q]);
    }
  }
}

// e = L_m^-1 f on the coarsest level Lc (cells in the FP32 swizzled layout);
// scratch z [2][nt][nr + 1] FP32 at dbl_off.
__device__ void coarsest_f32c(const VSmemArgs& a, int slot, unsigned char* vraw, const LevelDev& Lc,
                              const float2* fc, float2* ec) {
  const int nr = Lc.nr, nt = Lc.nt, P = nr + 1, nc = P * nt;
  const bool sym = a.sep_sym != 0;
  const int vr = sym ? nt / 2 : nt;
  float* z = reinterpret_cast<float*>(vraw + a.dbl_off);
  const float* ViT = a.blk_smem ? reinterpret_cast<const float*>(vraw + a.blk_off)
                                : a.sepf + size_t(slot) * a.sepf_stride;
  const float* VT = ViT + vr * nt;
  const float* invd = VT + nt * vr;
  const float* cp = invd + nc;
  const float* lid = cp + nc;
  if (vr % 4 == 0) f32c_forward<4>(Lc, fc, ViT, invd, z, sym);
  else f32c_forward<1>(Lc, fc, ViT, invd, z, sym);
  __syncthreads();
  // Thomas sweeps per (component, eigenvalue), one FMA per step each way:
  // dp_i = z_i - lid_i dp_{i-1}, then x_i = dp_i - cp_i x_{i+1}, in place;
  // the 2 nt systems on the first four warps
  {
    const int nsys = 2 * nt, per = (nsys + 3) / 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4 && lane < per && warp * per + lane < nsys) {
      const int q = warp * per + lane, c = q / nt, k = q - c * nt;
      float* __restrict__ zz = z + c * nc + k * P;
      const float* __restrict__ lk = lid + k * P;
      const float* __restrict__ ck = cp + k * P;
      // in batches of eight steps: the loads of a batch are issued together,
      // so one shared-memory latency is paid per batch, not per step
      float dp = zz[0];
      int i = 1;
      for (; i + 8 <= nr; i += 8) {
        float zv[8], lv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          zv[q] = zz[i + q];
          lv[q] = lk[i + q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          dp = fmaf(-lv[q], dp, zv[q]);
          zv[q] = dp;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) zz[i + q] = zv[q];
      }
      for (; i < nr; ++i) {
        dp = fmaf(-lk[i], dp, zz[i]);
        zz[i] = dp;
      }
      float xv = dp;
      i = nr - 2;
      for (; i >= 7; i -= 8) {
        float zv[8], cv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          zv[q] = zz[i - q];
          cv[q] = ck[i - q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          xv = fmaf(-cv[q], xv, zv[q]);
          zv[q] = xv;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) zz[i - q] = zv[q];
      }
      for (; i >= 0; --i) {
        xv = fmaf(-ck[i], xv, zz[i]);
        zz[i] = xv;
      }
    }
  }
  __syncthreads();
  if (vr % 4 == 0) f32c_back<4>(Lc, z, VT, ec, sym);
  else f32c_back<1>(Lc, z, VT, ec, sym);
  __syncthreads();
}

// The first fused level's right-hand side from global memory (this plane's
// n0 values at g) into its shared-memory slots by asynchronous copies: FP32
// as aligned cell pairs of 16 bytes (the even swizzle keeps pairs whole).
template <typename T>
__device__ __forceinline__ void stage_f0(const VSmemArgs& a, vec2_t<T>* sm, const vec2_t<T>* g) {
  const int nr0 = a.L[0].nr, n0 = nr0 * a.L[0].nt;
  if (sizeof(T) == 4 && nr0 % 2 == 0) {
    const float4* src = reinterpret_cast<const float4*>(g);
    float4* dst = reinterpret_cast<float4*>(sm + a.off_f[0]);
    RowWalk w(2 * threadIdx.x, 2 * blockDim.x, nr0);
    for (int k = threadIdx.x; 2 * k < n0; k += blockDim.x, w.next())
      cp_async_v(dst + vslot<T>(a.L[0], w.j, w.c) / 2, src + k, true);
  } else {
    RowWalk w(threadIdx.x, blockDim.x, nr0);
    for (int k = threadIdx.x; k < n0; k += blockDim.x, w.next())
      cp_async_v(sm + a.off_f[0] + vslot<T>(a.L[0], w.j, w.c), g + k, true);
  }
}

template <typename T, int NTH>
__global__ void __launch_bounds__(NTH, 1) k_vsmem(VSmemArgs a, Batch B, const vec2_t<T>* __restrict__ gf,
                                               vec2_t<T>* __restrict__ ge) {
  typedef vec2_t<T> V;
  extern __shared__ __align__(16) unsigned char vraw[];
  V* sm = reinterpret_cast<V*>(vraw);
  if (blockIdx.x >= *B.nact) return;
  const int p = B.act[blockIdx.x];
  const int slot = B.slot ? B.slot[p] : p;
  const int m = B.mode[slot];
  T s2;
  if constexpr (sizeof(T) == 8) s2 = B.s2d[slot]; else s2 = B.s2f[slot];
  const int K = a.nlev;
  const int nr0 = a.L[0].nr, n0 = nr0 * a.L[0].nt;
  // stage every level's coefficient tables and this mode's omega rows in
  // shared memory (after the error / right-hand-side arrays) and point a
  // block-local copy of the level descriptors at them
  __shared__ LevelDev sL[8];
  {
    // one flat copy of this slot's packed tables (each level's block starts
    // one element past an even element offset, so the two entries of a cell
    // pair are one aligned vector load), then block-local level descriptors
    T* tb = reinterpret_cast<T*>(sm + a.tab_off);
    {
      typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type W4;
      constexpr int per = int(sizeof(W4) / sizeof(T));
      const W4* src = reinterpret_cast<const W4*>(static_cast<const T*>(a.tabs) + size_t(slot) * a.tab_stride);
      W4* dst = reinterpret_cast<W4*>(tb);
      for (int k = threadIdx.x; k < a.tab_stride / per; k += blockDim.x) cp_async_v(dst + k, src + k, true);
    }
    if (threadIdx.x == 0) {
      int toff = 0;
      for (int l = 0; l < K; ++l) {
        const LevelDev& G = a.L[l];
        const int NR = G.nr + 2, NT = G.nt + 2;
        toff = (toff + 1) / 2 * 2 + 1;
        T* srt = tb + toff;
        T* stt = srt + RT_N * NR;
        T* sor = stt + TT_N * NT;
        T* sot = sor + G.nt;
        LevelDev d = G;
        if constexpr (sizeof(T) == 8) { d.rd = srt; d.td = stt; d.omr_d = sor; d.omt_d = sot; }
        else { d.rf = srt; d.tf = stt; d.omr_f = sor; d.omt_f = sot; }
        sL[l] = d;
        toff += RT_N * NR + TT_N * NT + G.nt + G.nr;
      }
    }
  }
  // this mode's coarsest-level factors (when they fit)
  const size_t blk_stride = size_t(a.blk_nt) * a.blk_n * (a.blk_n + 2);
  const size_t fac_stride = a.sep_stride > 0 ? size_t(a.sep_stride) : blk_stride;
  const LevelDev& Lcst = a.L[K - 1];
  if (a.f32c) {
    // FP32 V-cycle, separable coarsest level: its own factor block, staged
    // now unless it shares the first level's right-hand side space
    if constexpr (sizeof(T) == 4) {
      if (a.blk_smem && !a.restage)
        stage_f32c(a, slot, vraw);
    }
  } else if (a.blk_smem) {
    const double2* src = reinterpret_cast<const double2*>(
        (a.sep_stride > 0 ? a.sep : a.blk) + size_t(slot) * fac_stride);
    double2* dst = reinterpret_cast<double2*>(vraw + a.blk_off);
    for (int k = threadIdx.x; k < int(fac_stride / 2); k += blockDim.x) cp_async_v(dst + k, src + k, true);
  }
  // stage f of the first level, zero all errors
  stage_f0<T>(a, sm, gf + size_t(p) * n0);
  for (int l = 0; l < K; ++l) {
    const int n = a.L[l].nr * a.L[l].nt;
    if (sizeof(T) == 4 && n % 2 == 0 && a.off_e[l] % 2 == 0) {
      float4* d = reinterpret_cast<float4*>(sm + a.off_e[l]);
      for (int k = threadIdx.x; 2 * k < n; k += blockDim.x) d[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      for (int k = threadIdx.x; k < n; k += blockDim.x) sm[a.off_e[l] + k] = V{0, 0};
    }
  }
  // tables, factors and f arrive by asynchronous copies, all in flight at once
  cp_async_wait_all();
  __syncthreads();
  // Each phase works on register copies of the level descriptors: read
  // through sL, every shared-memory store of a phase could alias them and
  // force the descriptor fields to be loaded again.
  for (int l = 0; l < K - 1; ++l) {
    const LevelDev Lf = sL[l], Lq = sL[l + 1];
    s_smooth<T>(Lf, sm + a.off_e[l], sm + a.off_f[l], s2, a.nu1, a.n_sor);
    if constexpr (sizeof(T) == 4) {
      if (Lf.nr % 2 == 0 && Lf.nt % 2 == 0) s_restrict_f32(Lf, Lq, sm + a.off_e[l], sm + a.off_f[l], sm + a.off_f[l + 1], s2);
      else s_restrict<T>(Lf, Lq, sm + a.off_e[l], sm + a.off_f[l], sm + a.off_f[l + 1], s2);
    } else {
      s_restrict<T>(Lf, Lq, sm + a.off_e[l], sm + a.off_f[l], sm + a.off_f[l + 1], s2);
    }
  }
  if (a.f32c) {
    if constexpr (sizeof(T) == 4) {
      if (a.restage) {   // the factors take the first level's right-hand side space
        stage_f32c(a, slot, vraw);
        cp_async_wait_all();
        __syncthreads();
      }
      coarsest_f32c(a, slot, vraw, Lcst, sm + a.off_f[K - 1], sm + a.off_e[K - 1]);
      if (a.restage)   // the first level's right-hand side again, in flight during the prolongation
        stage_f0<T>(a, sm, gf + size_t(p) * n0);
    }
  } else if (a.sep_stride > 0) {
    // coarsest level, exact FP64 separable solve: L_m = L_r (x) I + D_r (x) L_t
    // with L_t = V diag(lambda) V^-1: z = (V^-1 (x) I) f, one tridiagonal
    // radial solve (L_r + lambda_k D_r) per eigenvalue k (Thomas), then
    // e = (V (x) I) z.
    const LevelDev& Lc = a.L[K - 1];
    const int nr = Lc.nr, nt = Lc.nt, nc = nr * nt;
    const V* fc = sm + a.off_f[K - 1];
    V* ec = sm + a.off_e[K - 1];
    double* z = reinterpret_cast<double*>(vraw + a.dbl_off);   // [2][nt][nr]
    const double* Fq = a.blk_smem ? reinterpret_cast<const double*>(vraw + a.blk_off)
                                  : a.sep + size_t(slot) * fac_stride;
    // mirror-symmetric layout (sep_sym): V rows j < h = nt/2, V^-1 columns
    // j < h; eigenvectors k < h even, k >= h odd
    const int h = nt / 2, vr = a.sep_sym ? h : nt;
    const double* Vm = Fq;                  // [vr][nt]
    const double* Vi = Vm + vr * nt;        // [nt][vr]
    const double* invd = Vi + nt * vr;
    const double* cp = invd + nt * nr;
    const double* lid = cp + nt * nr;
    // f in FP64, converted once (each value feeds several products; the
    // conversion itself runs on the FP64 pipe); mirror-symmetric: rows j < h
    // hold f_j + f_{nt-1-j} and rows h + j hold f_j - f_{nt-1-j}
    double* fd = z + 2 * nc;   // [2][nt][nr]
    if (a.sep_sym) {
      for (RowWalk w(threadIdx.x, blockDim.x, nr); w.j < h; w.next()) {
        const V u = fc[vslot<T>(Lc, w.j, w.c)], v = fc[vslot<T>(Lc, nt - 1 - w.j, w.c)];
        const double ux = u.x, uy = u.y, vx = v.x, vy = v.y;
        fd[w.j * nr + w.c] = ux + vx;
        fd[(h + w.j) * nr + w.c] = ux - vx;
        fd[nc + w.j * nr + w.c] = uy + vy;
        fd[nc + (h + w.j) * nr + w.c] = uy - vy;
      }
    } else {
      for (RowWalk w(threadIdx.x, blockDim.x, nr); w.j < nt; w.next()) {
        const V v = fc[vslot<T>(Lc, w.j, w.c)];
        fd[w.j * nr + w.c] = double(v.x);
        fd[nc + w.j * nr + w.c] = double(v.y);
      }
    }
    __syncthreads();
    // z = (1/pivot) .* ((V^-1 (x) I) f): the transform with the forward
    // sweep's first scaling folded in (mirror-symmetric: even eigenvectors
    // take the sums, odd ones the differences, over j < h)
    for (int q = threadIdx.x; q < 2 * nc; q += blockDim.x) {
      const int c = q / nc, r = q - c * nc, k = r / nr, i = r - k * nr;
      const double* fcol = fd + c * nc + (a.sep_sym && k >= h ? h * nr : 0) + i;
      double acc = 0.0;
      for (int j = 0; j < vr; ++j) acc += Vi[k * vr + j] * fcol[j * nr];
      z[q] = acc * invd[k * nr + i];
    }
    __syncthreads();
    // Thomas per (component, eigenvalue), one FMA per step each way:
    // dp_i = z_i - lid_i dp_{i-1}, then x_i = dp_i - cp_i x_{i+1}.  The 2 nt
    // independent systems run on the block's first four warps, eight lanes
    // each (one warp per scheduler: the FP64 pipe is narrow).
    for (int q = ((threadIdx.x >> 5) < 4 && (threadIdx.x & 31) < 8)
                     ? (threadIdx.x >> 5) * 8 + (threadIdx.x & 31)
                     : 2 * nt;
         q < 2 * nt; q += 32) {
      const int c = q / nt, k = q - c * nt;
      double* __restrict__ zz = z + c * nc + k * nr;
      const double* __restrict__ lk = lid + k * nr;
      const double* __restrict__ ck = cp + k * nr;
      double dp = zz[0];
#pragma unroll 4
      for (int i = 1; i < nr; ++i) {
        dp = fma(-lk[i], dp, zz[i]);
        zz[i] = dp;
      }
      double xv = dp;
#pragma unroll 4
      for (int i = nr - 2; i >= 0; --i) {
        xv = fma(-ck[i], xv, zz[i]);
        zz[i] = xv;
      }
    }
    __syncthreads();
    if (a.sep_sym) {   // e_j = E + O, e_{nt-1-j} = E - O (even, odd eigenvector parts)
      for (int q = threadIdx.x; q < h * nr; q += blockDim.x) {
        const int j = q / nr, i = q - j * nr;
        double ex = 0.0, ey = 0.0, ox = 0.0, oy = 0.0;
        for (int k = 0; k < h; ++k) {
          const double vk = Vm[j * nt + k];
          ex += vk * z[k * nr + i];
          ey += vk * z[nc + k * nr + i];
        }
        for (int k = h; k < nt; ++k) {
          const double vk = Vm[j * nt + k];
          ox += vk * z[k * nr + i];
          oy += vk * z[nc + k * nr + i];
        }
        ec[vslot<T>(Lc, j, i)] = V{T(ex + ox), T(ey + oy)};
        ec[vslot<T>(Lc, nt - 1 - j, i)] = V{T(ex - ox), T(ey - oy)};
      }
    } else {
      for (int q = threadIdx.x; q < nc; q += blockDim.x) {
        const int j = q / nr, i = q - j * nr;
        double ax = 0.0, ay = 0.0;
        for (int k = 0; k < nt; ++k) {
          const double vk = Vm[j * nt + k];
          ax += vk * z[k * nr + i];
          ay += vk * z[nc + k * nr + i];
        }
        ec[vslot<T>(Lc, j, i)] = V{T(ax), T(ay)};
      }
    }
    __syncthreads();
  } else if (a.blk_n > 0) {
    // coarsest level, exact FP64 block-tridiagonal solve (Schur complements
    // of the polar rows): forward z_J = f_J - b_J (S_{J-1}^{-1} z_{J-1}),
    // backward x_J = S_J^{-1} (z_J - c_J x_{J+1}).  Four warps (128 threads:
    // 2 components x n rows x g lanes per row) step through the 2 nt - 1
    // block products, joined by a named barrier.
    const int n = a.blk_n, nb = a.blk_nt, nc = a.nc;
    const LevelDev& Lc = a.L[K - 1];
    const V* fc = sm + a.off_f[K - 1];
    V* ec = sm + a.off_e[K - 1];
    double* z = reinterpret_cast<double*>(vraw + a.dbl_off);   // [2][nc]
    double* x = z + 2 * nc;                                     // [2][nc]
    const double* S = a.blk_smem ? reinterpret_cast<const double*>(vraw + a.blk_off)
                                 : a.blk + size_t(slot) * blk_stride;
    const double* bsub = S + size_t(nb) * n * n;
    const double* csup = bsub + size_t(nb) * n;
    const int t = threadIdx.x;
    if (t < 128) {
      const int g = 64 / n;
      const int sub = t & (g - 1), r = (t / g) % n, c = t / (n * g);
      auto fval = [&](int J) {
        const V v = fc[vslot<T>(Lc, J, r)];
        return double(c ? v.y : v.x);
      };
      if (sub == 0) z[c * nc + r] = fval(0);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      for (int J = 1; J < nb; ++J) {
        const double* Sr = S + size_t(J - 1) * n * n + size_t(r) * n;
        const double* zp = z + c * nc + (J - 1) * n;
        double acc = 0.0;
        for (int k = sub; k < n; k += g) acc += Sr[k] * zp[k];
        for (int o = g >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (sub == 0) z[c * nc + J * n + r] = fval(J) - bsub[J * n + r] * acc;
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
      for (int J = nb - 1; J >= 0; --J) {
        const double* Sr = S + size_t(J) * n * n + size_t(r) * n;
        const double* zJ = z + c * nc + J * n;
        double acc = 0.0;
        if (J == nb - 1) {
          for (int k = sub; k < n; k += g) acc += Sr[k] * zJ[k];
        } else {
          const double* xn = x + c * nc + (J + 1) * n;
          const double* cJ = csup + J * n;
          for (int k = sub; k < n; k += g) acc += Sr[k] * (zJ[k] - cJ[k] * xn[k]);
        }
        for (int o = g >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (sub == 0) x[c * nc + J * n + r] = acc;
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
      const int J = q / n, i = q - J * n;
      ec[vslot<T>(Lc, J, i)] = V{T(x[q]), T(x[nc + q])};
    }
    __syncthreads();
  } else {   // coarsest level: e = L^{-1} f, FP64 dot products, g threads per row
    const int nc = a.nc;
    const double* A = a.inv + size_t(slot) * nc * nc;
    const V* fc = sm + a.off_f[K - 1];
    V* ec = sm + a.off_e[K - 1];
    const LevelDev& Lc = a.L[K - 1];
    const int ncr = Lc.nr;
    // g lanes per row; nc is a power of two >= 16, so g * nc is a whole
    // number of warps and every warp below it takes part in the shuffles
    // (g > 1 only when g * nc fits in one pass of the block)
    int g = 1;
    while (g < 32 && g * 2 * nc <= int(blockDim.x)) g *= 2;   // uses all threads when nc >= 32
    for (int t = threadIdx.x; t < g * nc; t += blockDim.x) {
      const int row = t / g, sub = t & (g - 1);
      double sx = 0.0, sy = 0.0;
      for (int k = sub; k < nc; k += g) {
        const double c = A[size_t(row) * nc + k];
        const V fk = fc[vslot<T>(Lc, k / ncr, k % ncr)];
        sx += c * double(fk.x);
        sy += c * double(fk.y);
      }
      for (int o = g >> 1; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (sub == 0) ec[vslot<T>(Lc, row / ncr, row % ncr)] = V{T(sx), T(sy)};
    }
    __syncthreads();
  }
  for (int l = K - 2; l >= 0; --l) {
    const LevelDev Lf = sL[l], Lq = sL[l + 1];
    if constexpr (sizeof(T) == 4) {
      if (Lf.nr % 2 == 0 && Lf.nt % 2 == 0) s_prolong_f32(Lf, Lq, sm + a.off_e[l], sm + a.off_e[l + 1], m);
      else s_prolong<T>(Lf, Lq, sm + a.off_e[l], sm + a.off_e[l + 1], m);
    } else {
      s_prolong<T>(Lf, Lq, sm + a.off_e[l], sm + a.off_e[l + 1], m);
    }
    if (l == 0 && a.restage) {
      cp_async_wait_all();
      __syncthreads();
    }
    s_smooth<T>(Lf, sm + a.off_e[l], sm + a.off_f[l], s2, a.nu2, a.n_sor);
  }
  if (sizeof(T) == 4 && nr0 % 2 == 0) {   // FP32: aligned cell pairs, 16 bytes each
    const float4* src = reinterpret_cast<const float4*>(sm + a.off_e[0]);
    float4* dst = reinterpret_cast<float4*>(ge + size_t(p) * n0);
    RowWalk w(2 * threadIdx.x, 2 * blockDim.x, nr0);
    for (int k = threadIdx.x; 2 * k < n0; k += blockDim.x, w.next())
      dst[k] = src[vslot<T>(a.L[0], w.j, w.c) / 2];
  } else {
    RowWalk w(threadIdx.x, blockDim.x, nr0);
    for (int k = threadIdx.x; k < n0; k += blockDim.x, w.next())
      ge[size_t(p) * n0 + k] = sm[a.off_e[0] + vslot<T>(a.L[0], w.j, w.c)];
  }
}

// 512 threads (up to 128 registers each, no spills); each warp takes every
// 16th line of a colour.
template <typename T>
void launch_vsmem(const VSmemArgs& a, const Batch& B, const vec2_t<T>* gf, vec2_t<T>* ge,
                  cudaStream_t st) {
  constexpr int NTH = 512;
  static bool attr = false;
  if (!attr) {   // opt in to the largest dynamic size the kernel's static usage leaves
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_vsmem<T, NTH>) == cudaSuccess)
      cudaFuncSetAttribute(k_vsmem<T, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(227 * 1024 - fa.sharedSizeBytes));
    attr = true;
  }
  k_vsmem<T, NTH><<<B.max_planes, NTH, a.smem_bytes, st>>>(a, B, gf, ge);
}

template void launch_vsmem<float>(const VSmemArgs&, const Batch&, const float2*, float2*, cudaStream_t);
template void launch_vsmem<double>(const VSmemArgs&, const Batch&, const double2*, double2*, cudaStream_t);

}  // namespace ps
