// Line relaxation building blocks shared by the smoothing kernels (Sec. 3.2):
// one warp relaxes one radial line or one polar / vertical line held in
// registers; neighbours across lanes come by shuffles, so the n_sor even-odd
// SOR sweeps touch no memory.
//
// Lane mapping of a line of n cells (n <= 32, or n = 32 CPL with CPL even):
//   CPL == 1   lane k holds cell k (lanes k >= n hold nothing);
//   CPL even   lane k holds the pairs (2k + 64q, 2k + 1 + 64q), q < CPL / 2,
//              in register slots 2q and 2q + 1.
// A warp's access to a contiguous line then covers whole 128-byte rows (no
// shared-memory bank conflicts, full global sectors), and each SOR half-sweep
// needs one shuffle per pair.
//
// Coefficient tables hold the entry of cell i at index i + 1 and start one
// element past an even element boundary, so the two entries of a pair are one
// aligned vector load.
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

// Inverse diagonal of a line relaxation.  FP32 (the smoother of the FP32
// V-cycle, a preconditioner inside FP64 refinement): the hardware
// approximation __fdividef (within 2 ulp for the diagonal's range); FP64:
// correctly rounded, the same value as 1 / x.
__device__ __forceinline__ float rcp_diag(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_diag(double x) { return __drcp_rn(x); }

// a * b + c with one rounding.  The relaxation formulas spell out which
// products fuse into which additions, so that every kernel that relaxes a
// line rounds exactly the same way whatever the code around it (left to the
// compiler, a sum of two products may fuse either one).
__device__ __forceinline__ float fmac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return __fma_rn(a, b, c); }

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
template <typename V> __device__ __forceinline__ V shidx(V v, int src) {
  v.x = __shfl_sync(0xffffffffu, v.x, src);
  v.y = __shfl_sync(0xffffffffu, v.y, src);
  return v;
}

// Asynchronous global -> shared copy of one complex value (zero-filled when
// !valid; src must still be a valid address), and the wait for all of them.
template <typename V>
__device__ __forceinline__ void cp_async_v(V* dst, const V* src, bool valid) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  const int n = valid ? int(sizeof(V)) : 0;
  if constexpr (sizeof(V) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Cell index held in register slot c of `lane`.
// Walks the (row, column) pairs of a row-major n-column array in steps of
// `step` flat elements from flat index `start`: one division at set-up, then
// an add and a conditional subtract per step (0 <= c < n throughout).
struct RowWalk {
  int j, c, dj, dc, n;
  __device__ __forceinline__ RowWalk(int start, int step, int n_) : n(n_) {
    j = start / n; c = start - j * n; dj = step / n; dc = step - dj * n;
  }
  __device__ __forceinline__ void next() {
    c += dc; j += dj;
    if (c >= n) { c -= n; ++j; }
  }
};

template <int CPL> __device__ __forceinline__ int lcell(int lane, int c) {
  if constexpr (CPL == 1) return lane;
  else return 2 * lane + 64 * (c >> 1) + (c & 1);
}

// Two consecutive complex values (one 16-byte access for float2).
template <typename V> __device__ __forceinline__ void ld_pair(V& a, V& b, const V* p) {
  if constexpr (sizeof(V) == 8) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a.x = v.x; a.y = v.y; b.x = v.z; b.y = v.w;
  } else {
    a = p[0];
    b = p[1];
  }
}
template <typename V> __device__ __forceinline__ void st_pair(V* p, const V& a, const V& b) {
  if constexpr (sizeof(V) == 8) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    p[0] = a;
    p[1] = b;
  }
}

// The lane's cells of a line of n cells stored contiguously at p.
template <typename V, int CPL>
__device__ __forceinline__ void ld_line(V (&d)[CPL], const V* p, int lane, int n) {
  if constexpr (CPL == 1) {
    d[0] = lane < n ? p[lane] : z2<V>();
  } else {
#pragma unroll
    for (int q = 0; q < CPL / 2; ++q) ld_pair(d[2 * q], d[2 * q + 1], p + 2 * lane + 64 * q);
  }
}
template <typename V, int CPL>
__device__ __forceinline__ void st_line(V* p, const V (&d)[CPL], int lane, int n) {
  if constexpr (CPL == 1) {
    if (lane < n) p[lane] = d[0];
  } else {
#pragma unroll
    for (int q = 0; q < CPL / 2; ++q) st_pair(p + 2 * lane + 64 * q, d[2 * q], d[2 * q + 1]);
  }
}

// Same for a row whose cell i is stored at row[i ^ s] (s < n, n a power of
// two): a pair stays one aligned vector, swapped when s is odd.
template <typename V, int CPL>
__device__ __forceinline__ void ld_line_swz(V (&d)[CPL], const V* row, int s, int lane, int n) {
  if constexpr (CPL == 1) {
    d[0] = lane < n ? row[lane ^ s] : z2<V>();
  } else {
#pragma unroll
    for (int q = 0; q < CPL / 2; ++q) {
      V a, b;
      ld_pair(a, b, row + ((2 * lane + 64 * q) ^ (s & ~1)));
      d[2 * q] = (s & 1) ? b : a;
      d[2 * q + 1] = (s & 1) ? a : b;
    }
  }
}
template <typename V, int CPL>
__device__ __forceinline__ void st_line_swz(V* row, int s, const V (&d)[CPL], int lane, int n) {
  if constexpr (CPL == 1) {
    if (lane < n) row[lane ^ s] = d[0];
  } else {
#pragma unroll
    for (int q = 0; q < CPL / 2; ++q) {
      const V a = (s & 1) ? d[2 * q + 1] : d[2 * q];
      const V b = (s & 1) ? d[2 * q] : d[2 * q + 1];
      st_pair(row + ((2 * lane + 64 * q) ^ (s & ~1)), a, b);
    }
  }
}

// Table entries of the lane's cells (entry of cell i at tab[i + 1]; 0 for
// cells beyond n).
template <typename T, int CPL>
__device__ __forceinline__ void ld_tab(T (&d)[CPL], const T* tab, int lane, int n) {
  if constexpr (CPL == 1) {
    d[0] = lane < n ? tab[lane + 1] : T(0);
  } else {
#pragma unroll
    for (int q = 0; q < CPL / 2; ++q) {
      const vec2_t<T> v = *reinterpret_cast<const vec2_t<T>*>(tab + 2 * lane + 64 * q + 1);
      d[2 * q] = v.x;
      d[2 * q + 1] = v.y;
    }
  }
}

// n_sor even-odd SOR sweeps of a line of n cells held in registers:
// x_k <- x_k + w ((g_k - up_k x_{k+1} - dn_k x_{k-1}) id_k - x_k) (the
// (1 - w) x_k + w (...) id_k of SOR in four fused operations per component),
// cells of even index first; the ghosts beyond both ends are zero.
template <typename T, int CPL>
__device__ __forceinline__ void sor_line(vec2_t<T> (&ev)[CPL], const vec2_t<T> (&g)[CPL],
                                         const T (&up)[CPL], const T (&dn)[CPL], const T (&id)[CPL],
                                         T w, int n, int n_sor) {
  typedef vec2_t<T> V;
  const int lane = threadIdx.x & 31;
  auto upd = [&](int c, const V& em, const V& ep) {
    const T rx = fmac(-dn[c], em.x, fmac(-up[c], ep.x, g[c].x));
    const T ry = fmac(-dn[c], em.y, fmac(-up[c], ep.y, g[c].y));
    ev[c].x = fmac(w, fmac(id[c], rx, -ev[c].x), ev[c].x);
    ev[c].y = fmac(w, fmac(id[c], ry, -ev[c].y), ev[c].y);
  };
  if constexpr (CPL == 1) {
    const bool on = lane < n, last = lane == n - 1;
#pragma unroll 1
    for (int it = 0; it < n_sor; ++it) {
#pragma unroll
      for (int par = 0; par < 2; ++par) {
        V left = shup(ev[0]);
        V right = shdn(ev[0]);
        if (lane == 0) left = z2<V>();
        if (last) right = z2<V>();
        if (on && (lane & 1) == par) upd(0, left, right);
      }
    }
  } else {
    constexpr int NP = CPL / 2;
    const int prv = (lane + 31) & 31, nxt = (lane + 1) & 31;
#pragma unroll 1
    for (int it = 0; it < n_sor; ++it) {
      V r[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) r[q] = shidx(ev[2 * q + 1], prv);   // odd cell 2k - 1 + 64q
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        V left = r[q];
        if (lane == 0) left = q == 0 ? z2<V>() : r[q > 0 ? q - 1 : 0];
        upd(2 * q, left, ev[2 * q + 1]);
      }
#pragma unroll
      for (int q = 0; q < NP; ++q) r[q] = shidx(ev[2 * q], nxt);       // even cell 2k + 2 + 64q
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        V right = r[q];
        if (lane == 31) right = q == NP - 1 ? z2<V>() : r[q + 1 < NP ? q + 1 : q];
        upd(2 * q + 1, ev[2 * q], right);
      }
    }
  }
}

// Coefficients of the lane's cells that every radial line of a level shares
// (they depend on the radial index only), and likewise for polar lines.
template <typename T, int CPL>
struct RLineTabs {
  T P[CPL], dr[CPL], q[CPL], up[CPL], dn[CPL];
};
template <typename T, int CPL>
struct TLineTabs {
  T dt[CPL], tj[CPL], an[CPL], as[CPL];
};

template <typename T, int CPL>
__device__ __forceinline__ void ld_rtabs(RLineTabs<T, CPL>& a, const LevelDev& L, const T* rt) {
  const int lane = threadIdx.x & 31, nr = L.nr, NR = nr + 2;
  ld_tab<T, CPL>(a.P, rt + RT_P * NR, lane, nr);
  ld_tab<T, CPL>(a.dr, rt + RT_DR * NR, lane, nr);
  ld_tab<T, CPL>(a.q, rt + RT_Q * NR, lane, nr);
  ld_tab<T, CPL>(a.up, rt + RT_AE * NR, lane, nr);
  ld_tab<T, CPL>(a.dn, rt + RT_AW * NR, lane, nr);
}
template <typename T, int CPL>
__device__ __forceinline__ void ld_ttabs(TLineTabs<T, CPL>& a, const LevelDev& L, const T* tt) {
  const int lane = threadIdx.x & 31, nt = L.nt, NT = nt + 2;
  ld_tab<T, CPL>(a.dt, tt + TT_DT * NT, lane, nt);
  ld_tab<T, CPL>(a.tj, tt + TT_T * NT, lane, nt);
  ld_tab<T, CPL>(a.an, tt + TT_AN * NT, lane, nt);
  ld_tab<T, CPL>(a.as, tt + TT_AS * NT, lane, nt);
}

// Radial line j: g = source values of the lane's cells (clobbered), un / us =
// lines j+1 / j-1 (zero beyond the plane), ev = own line on entry, relaxed
// line on exit; a = the level's radial-line coefficients of the lane's cells.
template <typename T, int CPL>
__device__ __forceinline__ void relax_r(const LevelDev& L, const RLineTabs<T, CPL>& a, const T* tt,
                                        T s2, T w, int j, vec2_t<T> (&g)[CPL],
                                        const vec2_t<T> (&un)[CPL], const vec2_t<T> (&us)[CPL],
                                        int n_sor, vec2_t<T> (&ev)[CPL]) {
  const int lane = threadIdx.x & 31, nr = L.nr, NT = L.nt + 2;
  const T aN = tt[TT_AN * NT + j + 1], aS = tt[TT_AS * NT + j + 1];
  const T Tj = tt[TT_T * NT + j + 1], dtj = tt[TT_DT * NT + j + 1];
  const bool on = CPL > 1 || lane < nr;
  T id[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    g[c].x = fmac(-a.P[c], fmac(aS, us[c].x, aN * un[c].x), g[c].x);
    g[c].y = fmac(-a.P[c], fmac(aS, us[c].y, aN * un[c].y), g[c].y);
    id[c] = on ? rcp_diag(fmac(-(s2 * a.q[c]), Tj, fmac(a.P[c], dtj, a.dr[c]))) : T(0);
  }
  sor_line<T, CPL>(ev, g, a.up, a.dn, id, w, nr, n_sor);
}

// Same, loading the coefficients from the level's table as it uses them (for
// kernels without registers to keep them): neighbour lines first (they die
// there), then the diagonal, then the along-line couplings.
template <typename T, int CPL>
__device__ __forceinline__ void relax_r(const LevelDev& L, const T* rt, const T* tt, T s2, T w,
                                        int j, vec2_t<T> (&g)[CPL], const vec2_t<T> (&un)[CPL],
                                        const vec2_t<T> (&us)[CPL], int n_sor,
                                        vec2_t<T> (&ev)[CPL]) {
  const int lane = threadIdx.x & 31, nr = L.nr, NR = nr + 2, NT = L.nt + 2;
  const T aN = tt[TT_AN * NT + j + 1], aS = tt[TT_AS * NT + j + 1];
  const T Tj = tt[TT_T * NT + j + 1], dtj = tt[TT_DT * NT + j + 1];
  const bool on = CPL > 1 || lane < nr;
  T P[CPL], up[CPL], dn[CPL], id[CPL];
  ld_tab<T, CPL>(P, rt + RT_P * NR, lane, nr);
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    g[c].x = fmac(-P[c], fmac(aS, us[c].x, aN * un[c].x), g[c].x);
    g[c].y = fmac(-P[c], fmac(aS, us[c].y, aN * un[c].y), g[c].y);
  }
  {
    T dr[CPL], q[CPL];
    ld_tab<T, CPL>(dr, rt + RT_DR * NR, lane, nr);
    ld_tab<T, CPL>(q, rt + RT_Q * NR, lane, nr);
#pragma unroll
    for (int c = 0; c < CPL; ++c) id[c] = on ? rcp_diag(fmac(-(s2 * q[c]), Tj, fmac(P[c], dtj, dr[c]))) : T(0);
  }
  ld_tab<T, CPL>(up, rt + RT_AE * NR, lane, nr);
  ld_tab<T, CPL>(dn, rt + RT_AW * NR, lane, nr);
  sor_line<T, CPL>(ev, g, up, dn, id, w, nr, n_sor);
}

// Polar / vertical line i: g = source values of the lane's cells (clobbered),
// ue / uw = columns i+1 / i-1 (zero beyond the plane), ev = own column on
// entry, relaxed column on exit; a = the level's polar-line coefficients of
// the lane's cells.
template <typename T, int CPL>
__device__ __forceinline__ void relax_t(const LevelDev& L, const T* rt, const TLineTabs<T, CPL>& a,
                                        T s2, T w, int i, vec2_t<T> (&g)[CPL],
                                        const vec2_t<T> (&ue)[CPL], const vec2_t<T> (&uw)[CPL],
                                        int n_sor, vec2_t<T> (&ev)[CPL]) {
  const int lane = threadIdx.x & 31, nt = L.nt, NR = L.nr + 2;
  const T P = rt[RT_P * NR + i + 1], aE = rt[RT_AE * NR + i + 1], aW = rt[RT_AW * NR + i + 1];
  const T dr = rt[RT_DR * NR + i + 1], Qi = rt[RT_Q * NR + i + 1];
  const bool on = CPL > 1 || lane < nt;
  T up[CPL], dn[CPL], id[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    g[c].x = fmac(-aW, uw[c].x, fmac(-aE, ue[c].x, g[c].x));
    g[c].y = fmac(-aW, uw[c].y, fmac(-aE, ue[c].y, g[c].y));
    id[c] = on ? rcp_diag(fmac(-(s2 * Qi), a.tj[c], fmac(P, a.dt[c], dr))) : T(0);
    up[c] = P * a.an[c];
    dn[c] = P * a.as[c];
  }
  sor_line<T, CPL>(ev, g, up, dn, id, w, nt, n_sor);
}

// Same, loading the coefficients as it uses them.
template <typename T, int CPL>
__device__ __forceinline__ void relax_t(const LevelDev& L, const T* rt, const T* tt, T s2, T w,
                                        int i, vec2_t<T> (&g)[CPL], const vec2_t<T> (&ue)[CPL],
                                        const vec2_t<T> (&uw)[CPL], int n_sor,
                                        vec2_t<T> (&ev)[CPL]) {
  const int lane = threadIdx.x & 31, nt = L.nt, NR = L.nr + 2, NT = nt + 2;
  const T P = rt[RT_P * NR + i + 1], aE = rt[RT_AE * NR + i + 1], aW = rt[RT_AW * NR + i + 1];
  const T dr = rt[RT_DR * NR + i + 1], Qi = rt[RT_Q * NR + i + 1];
  const bool on = CPL > 1 || lane < nt;
  T up[CPL], dn[CPL], id[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    g[c].x = fmac(-aW, uw[c].x, fmac(-aE, ue[c].x, g[c].x));
    g[c].y = fmac(-aW, uw[c].y, fmac(-aE, ue[c].y, g[c].y));
  }
  {
    T dt[CPL], tj[CPL];
    ld_tab<T, CPL>(dt, tt + TT_DT * NT, lane, nt);
    ld_tab<T, CPL>(tj, tt + TT_T * NT, lane, nt);
#pragma unroll
    for (int c = 0; c < CPL; ++c) id[c] = on ? rcp_diag(fmac(-(s2 * Qi), tj[c], fmac(P, dt[c], dr))) : T(0);
  }
  ld_tab<T, CPL>(up, tt + TT_AN * NT, lane, nt);
  ld_tab<T, CPL>(dn, tt + TT_AS * NT, lane, nt);
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    up[c] = P * up[c];
    dn[c] = P * dn[c];
  }
  sor_line<T, CPL>(ev, g, up, dn, id, w, nt, n_sor);
}

}  // namespace ps
