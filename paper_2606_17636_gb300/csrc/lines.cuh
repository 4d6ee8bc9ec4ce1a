// Line relaxation building blocks shared by the smoothing kernels (Sec. 3.2):
// one warp relaxes one radial line or one polar / vertical line; each lane
// holds CPL consecutive cells in registers, neighbours across lanes come by
// shuffles, so the n_sor even-odd SOR sweeps touch no memory.
#pragma once
#include "kernels.h"

namespace ps {

template <typename T> __device__ __forceinline__ const T* rt_(const LevelDev& L);
template <> __device__ __forceinline__ const double* rt_<double>(const LevelDev& L) { return L.rd; }
template <> __device__ __forceinline__ const float* rt_<float>(const LevelDev& L) { return L.rf; }
template <typename T> __device__ __forceinline__ const T* tt_(const LevelDev& L);
template <> __device__ __forceinline__ const double* tt_<double>(const LevelDev& L) { return L.td; }
template <> __device__ __forceinline__ const float* tt_<float>(const LevelDev& L) { return L.tf; }
template <typename T> __device__ __forceinline__ const T* omr_(const LevelDev& L);
template <> __device__ __forceinline__ const double* omr_<double>(const LevelDev& L) { return L.omr_d; }
template <> __device__ __forceinline__ const float* omr_<float>(const LevelDev& L) { return L.omr_f; }
template <typename T> __device__ __forceinline__ const T* omt_(const LevelDev& L);
template <> __device__ __forceinline__ const double* omt_<double>(const LevelDev& L) { return L.omt_d; }
template <> __device__ __forceinline__ const float* omt_<float>(const LevelDev& L) { return L.omt_f; }
template <typename T> __device__ __forceinline__ T s2_(const Batch& B, int slot);
template <> __device__ __forceinline__ double s2_<double>(const Batch& B, int slot) { return B.s2d[slot]; }
template <> __device__ __forceinline__ float s2_<float>(const Batch& B, int slot) { return B.s2f[slot]; }

template <typename V> __device__ __forceinline__ V z2() { V v; v.x = 0; v.y = 0; return v; }

template <typename V> __device__ __forceinline__ V shup(V v) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
  return v;
}
template <typename V> __device__ __forceinline__ V shdn(V v) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
  v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
  return v;
}

// CPL consecutive complex values at p (16-byte vector accesses when possible).
template <typename V, int CPL>
__device__ __forceinline__ void ld_run(V (&d)[CPL], const V* p) {
  if constexpr (sizeof(V) == 8 && CPL % 2 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int c = 0; c < CPL / 2; ++c) {
      const float4 v = q[c];
      d[2 * c].x = v.x; d[2 * c].y = v.y; d[2 * c + 1].x = v.z; d[2 * c + 1].y = v.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < CPL; ++c) d[c] = p[c];
  }
}
template <typename V, int CPL>
__device__ __forceinline__ void st_run(V* p, const V (&d)[CPL]) {
  if constexpr (sizeof(V) == 8 && CPL % 2 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int c = 0; c < CPL / 2; ++c) q[c] = make_float4(d[2 * c].x, d[2 * c].y, d[2 * c + 1].x, d[2 * c + 1].y);
  } else {
#pragma unroll
    for (int c = 0; c < CPL; ++c) p[c] = d[c];
  }
}

// n_sor even-odd SOR sweeps of a line held in registers: x_k <- (1-w) x_k +
// w (g_k - up_k x_{k+1} - dn_k x_{k-1}) id_k, cells of even position first.
template <typename T, int CPL>
__device__ __forceinline__ void sor_line(vec2_t<T> (&ev)[CPL], const vec2_t<T> (&g)[CPL],
                                         const T (&up)[CPL], const T (&dn)[CPL], const T (&id)[CPL],
                                         T w, int k0, bool on, bool last, int n_sor) {
  typedef vec2_t<T> V;
  const int lane = threadIdx.x & 31;
  const T w1 = T(1) - w;
  for (int it = 0; it < n_sor; ++it) {
#pragma unroll
    for (int par = 0; par < 2; ++par) {
      V left = shup(ev[CPL - 1]);
      V right = shdn(ev[0]);
      if (lane == 0) left = z2<V>();
      if (last) right = z2<V>();
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        if (on && ((k0 + c) & 1) == par) {
          const V em = (c > 0) ? ev[c - 1] : left;
          const V ep = (c < CPL - 1) ? ev[c + 1] : right;
          const T tx = (g[c].x - up[c] * ep.x - dn[c] * em.x) * id[c];
          const T ty = (g[c].y - up[c] * ep.y - dn[c] * em.y) * id[c];
          ev[c].x = w1 * ev[c].x + w * tx;
          ev[c].y = w1 * ev[c].y + w * ty;
        }
      }
    }
  }
}

// Radial line j from registers: g = source line, un / us = neighbour lines
// j+1 / j-1, ev = own line on entry, relaxed line on exit (lane holds cells
// lane*CPL ..).
template <typename T, int CPL>
__device__ __forceinline__ void relax_rline_regs(const LevelDev& L, const T* rt, const T* tt, T s2,
                                                 T w, int j, vec2_t<T> (&g)[CPL],
                                                 const vec2_t<T> (&un)[CPL],
                                                 const vec2_t<T> (&us)[CPL], int n_sor,
                                                 vec2_t<T> (&ev)[CPL]) {
  const int lane = threadIdx.x & 31, nr = L.nr, NR = nr + 2, NT = L.nt + 2;
  const int i0 = lane * CPL;
  const bool on = i0 < nr;
  const T aN = tt[TT_AN * NT + j + 1], aS = tt[TT_AS * NT + j + 1];
  const T Tj = tt[TT_T * NT + j + 1], dtj = tt[TT_DT * NT + j + 1];
  T up[CPL], dn[CPL], id[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int i = i0 + c + 1;
    const T P = on ? rt[RT_P * NR + i] : T(0);
    g[c].x = g[c].x - P * (aN * un[c].x + aS * us[c].x);
    g[c].y = g[c].y - P * (aN * un[c].y + aS * us[c].y);
    up[c] = on ? rt[RT_AE * NR + i] : T(0);
    dn[c] = on ? rt[RT_AW * NR + i] : T(0);
    id[c] = on ? T(1) / (rt[RT_DR * NR + i] + P * dtj - s2 * rt[RT_Q * NR + i] * Tj) : T(0);
  }
  sor_line<T, CPL>(ev, g, up, dn, id, w, i0, on, i0 + CPL >= nr, n_sor);
}

// Radial line j: own line (nullptr = 0), neighbour lines j+1 / j-1 (nullptr =
// ghost 0), source line; contiguous storage.  Result in ev.
template <typename T, int CPL, bool VEC = true>
__device__ __forceinline__ void relax_rline(const LevelDev& L, const T* rt, const T* tt, T s2, T w,
                                            int j, const vec2_t<T>* own, const vec2_t<T>* nn,
                                            const vec2_t<T>* ss, const vec2_t<T>* fl_, int n_sor,
                                            vec2_t<T> (&ev)[CPL]) {
  typedef vec2_t<T> V;
  const int lane = threadIdx.x & 31, nr = L.nr;
  const int i0 = lane * CPL;
  const bool on = i0 < nr;
  V g[CPL], un[CPL], us[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) { ev[c] = z2<V>(); g[c] = z2<V>(); un[c] = z2<V>(); us[c] = z2<V>(); }
  if (on) {
    if constexpr (VEC) {
      ld_run<V, CPL>(g, fl_ + i0);
      if (own) ld_run<V, CPL>(ev, own + i0);
      if (nn) ld_run<V, CPL>(un, nn + i0);
      if (ss) ld_run<V, CPL>(us, ss + i0);
    } else {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        g[c] = fl_[i0 + c];
        if (own) ev[c] = own[i0 + c];
        if (nn) un[c] = nn[i0 + c];
        if (ss) us[c] = ss[i0 + c];
      }
    }
  }
  relax_rline_regs<T, CPL>(L, rt, tt, s2, w, j, g, un, us, n_sor, ev);
}

// Bilinear coarse correction (Sec. 3.1, Eq. prolongation_sph) at fine cell
// (i, j): coarse level C of plane p, parity sign of mode m at poles / axis.
template <typename T>
__device__ __forceinline__ vec2_t<T> coarse_at(const LevelDev& C, const vec2_t<T>* __restrict__ ec,
                                               int I, int J, int m) {
  typedef vec2_t<T> V;
  T fac = T(1);
  const T sgn = (m & 1) ? T(-1) : T(1);
  int Ic = I, Jc = J;
  if (I == 0) { if (C.gL == GH_ZERO) return z2<V>(); Ic = 1; if (C.gL == GH_PARITY) fac *= sgn; }
  if (I == C.nr + 1) { if (C.gR == GH_ZERO) return z2<V>(); Ic = C.nr; if (C.gR == GH_PARITY) fac *= sgn; }
  if (J == 0) { if (C.gB == GH_ZERO) return z2<V>(); Jc = 1; if (C.gB == GH_PARITY) fac *= sgn; }
  if (J == C.nt + 1) { if (C.gT == GH_ZERO) return z2<V>(); Jc = C.nt; if (C.gT == GH_PARITY) fac *= sgn; }
  V v = ec[size_t(Jc - 1) * C.nr + (Ic - 1)];
  v.x *= fac;
  v.y *= fac;
  return v;
}

template <typename T>
__device__ __forceinline__ vec2_t<T> prolong_at(const LevelDev& L, const T* rt, const T* tt,
                                                const LevelDev& C, const vec2_t<T>* __restrict__ ec,
                                                int i, int j, int m) {
  typedef vec2_t<T> V;
  const int i1 = i + 1, j1 = j + 1, NR = L.nr + 2, NT = L.nt + 2;
  const int I1 = (i1 & 1) ? (i1 + 1) / 2 - 1 : i1 / 2, J1 = (j1 & 1) ? (j1 + 1) / 2 - 1 : j1 / 2;
  const T p1 = rt[RT_P1 * NR + i1], p2 = rt[RT_P2 * NR + i1];
  const T q1 = tt[TT_P1 * NT + j1], q2 = tt[TT_P2 * NT + j1];
  const V a = coarse_at<T>(C, ec, I1, J1, m), b = coarse_at<T>(C, ec, I1 + 1, J1, m);
  const V c = coarse_at<T>(C, ec, I1, J1 + 1, m), d = coarse_at<T>(C, ec, I1 + 1, J1 + 1, m);
  V r;
  r.x = p1 * q1 * a.x + p2 * q1 * b.x + p1 * q2 * c.x + p2 * q2 * d.x;
  r.y = p1 * q1 * a.y + p2 * q1 * b.y + p1 * q2 * c.y + p2 * q2 * d.y;
  return r;
}

// Polar / vertical line i stored with row stride `ld` (an odd stride keeps
// the strided column loads to at most CPL-way shared-memory bank conflicts;
// they happen once per line, the SOR sweeps run in registers): own column,
// west and east neighbour columns (nullptr = ghost 0), source column.  Lane k
// holds cells j = k*CPL .. k*CPL+CPL-1; result in ev.
template <typename T, int CPL>
__device__ __forceinline__ void relax_tcol(const LevelDev& L, const T* rt, const T* tt, T s2, T w,
                                           int i, const vec2_t<T>* own, const vec2_t<T>* west,
                                           const vec2_t<T>* east, const vec2_t<T>* fcol, int ld,
                                           int n_sor, vec2_t<T> (&ev)[CPL]) {
  typedef vec2_t<T> V;
  const int lane = threadIdx.x & 31, nt = L.nt, NR = L.nr + 2, NT = nt + 2;
  const int j0 = lane * CPL;
  const bool on = j0 < nt;
  const T P = rt[RT_P * NR + i + 1], aE = rt[RT_AE * NR + i + 1], aW = rt[RT_AW * NR + i + 1];
  const T dr = rt[RT_DR * NR + i + 1], Qi = rt[RT_Q * NR + i + 1];
  V g[CPL];
  T up[CPL], dn[CPL], id[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int j = j0 + c;
    ev[c] = z2<V>();
    g[c] = z2<V>();
    up[c] = dn[c] = id[c] = T(0);
    if (on) {
      const V fv = fcol[size_t(j) * ld];
      const V ue = east ? east[size_t(j) * ld] : z2<V>();
      const V uw = west ? west[size_t(j) * ld] : z2<V>();
      g[c].x = fv.x - aE * ue.x - aW * uw.x;
      g[c].y = fv.y - aE * ue.y - aW * uw.y;
      if (own) ev[c] = own[size_t(j) * ld];
      up[c] = P * tt[TT_AN * NT + j + 1];
      dn[c] = P * tt[TT_AS * NT + j + 1];
      id[c] = T(1) / (dr + P * tt[TT_DT * NT + j + 1] - s2 * Qi * tt[TT_T * NT + j + 1]);
    }
  }
  sor_line<T, CPL>(ev, g, up, dn, id, w, j0, on, j0 + CPL >= nt, n_sor);
}

}  // namespace ps
