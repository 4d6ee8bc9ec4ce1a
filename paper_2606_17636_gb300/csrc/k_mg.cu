// Multigrid kernels for the per-mode Helmholtz problems (Sec. 3).
//
// Planes hold the real and imaginary part of one mode as the two components
// of a float2 / double2: the operator L_m is real, so both are relaxed by the
// same line operations.  Dirichlet ghosts of the error equation are zero; a
// face of zero area has a zero coefficient, so pole / axis ghosts never enter
// the stencil.
#include <cstdio>

#include "lines.cuh"

namespace ps {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ const T* rtab(const LevelDev& L);
template <> __device__ __forceinline__ const double* rtab<double>(const LevelDev& L) { return L.rd; }
template <> __device__ __forceinline__ const float* rtab<float>(const LevelDev& L) { return L.rf; }
template <typename T> __device__ __forceinline__ const T* ttab(const LevelDev& L);
template <> __device__ __forceinline__ const double* ttab<double>(const LevelDev& L) { return L.td; }
template <> __device__ __forceinline__ const float* ttab<float>(const LevelDev& L) { return L.tf; }
template <typename T> __device__ __forceinline__ const T* omr(const LevelDev& L);
template <> __device__ __forceinline__ const double* omr<double>(const LevelDev& L) { return L.omr_d; }
template <> __device__ __forceinline__ const float* omr<float>(const LevelDev& L) { return L.omr_f; }
template <typename T> __device__ __forceinline__ const T* omt(const LevelDev& L);
template <> __device__ __forceinline__ const double* omt<double>(const LevelDev& L) { return L.omt_d; }
template <> __device__ __forceinline__ const float* omt<float>(const LevelDev& L) { return L.omt_f; }
template <typename T> __device__ __forceinline__ T s2of(const Batch& B, int slot);
template <> __device__ __forceinline__ double s2of<double>(const Batch& B, int slot) { return B.s2d[slot]; }
template <> __device__ __forceinline__ float s2of<float>(const Batch& B, int slot) { return B.s2f[slot]; }

#define RTAB(tab, id, i) (tab)[(id) * (L.nr + 2) + (i)]
#define TTAB(tab, id, j) (tab)[(id) * (L.nt + 2) + (j)]

template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

template <typename V, typename T> __device__ __forceinline__ V vmk(T a, T b);
template <> __device__ __forceinline__ float2 vmk<float2, float>(float a, float b) { return make_float2(a, b); }
template <> __device__ __forceinline__ double2 vmk<double2, double>(double a, double b) { return make_double2(a, b); }

enum { ST_ACTIVE = 1, ST_OK = 0, ST_STAGNATED = 2, ST_NOTCONV = -4, ST_NONFINITE = -5 };

// Grids of the per-plane kernels are bounded (a few blocks per SM) and loop
// over work items w = k * bpp + b (active plane k, block b of bpp), so the
// cost of a launch follows the active planes, not the planes allocated.
static int work_grid(long items) {
  static int sms = 0;   // cached on first use (the solver's set-up, before any capture)
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 132;
  }
  const long cap = long(sms) * 8;
  return int(items < cap ? (items > 0 ? items : 1) : cap);
}

__device__ __forceinline__ bool plane_of(const Batch& B, int k, int& p, int& slot) {
  if (k >= *B.nact) return false;
  p = B.act[k];
  slot = B.slot ? B.slot[p] : p;
  return true;
}

// ---------------------------------------------------------------------------
// Defect and area-weighted restriction (Sec. 3.1): one thread per coarse cell
// computes the defect f - L e of its four children and their weighted sum.
// The children 2I, 2I + 1 of a row are an aligned pair, and so are their
// neighbours in the rows above and below (one vector access each); the
// defect's fused operations are spelled out as in the fused V-cycle's
// restriction.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(LevelDev L, LevelDev C, Batch B,
                                                  const vec2_t<T>* __restrict__ e,
                                                  const vec2_t<T>* __restrict__ f,
                                                  vec2_t<T>* __restrict__ fc) {
  typedef vec2_t<T> V;
  const int nact = *B.nact, nc = C.nr * C.nt, bpp = (nc + blockDim.x - 1) / blockDim.x;
  const int nr = L.nr, nt = L.nt;
  const T* rt = rtab<T>(L);
  const T* tt = ttab<T>(L);
  const V z = vzero<V>();
  for (int w = blockIdx.x; w < nact * bpp; w += gridDim.x) {
    const int k = w / bpp;
    const int cidx = (w - k * bpp) * blockDim.x + threadIdx.x;
    if (cidx >= nc) continue;
    const int p = B.act[k];
    const int slot = B.slot ? B.slot[p] : p;
    const int J = cidx / C.nr, I = cidx - J * C.nr, i0 = 2 * I, j0 = 2 * J;
    const T s2 = s2of<T>(B, slot);
    const size_t base = size_t(p) * nr * nt;
    const V* ep = e + base;
    const V* fp = f + base;
    // e on rows j0 - 1 .. j0 + 2 at columns i0, i0 + 1; W and E neighbours on rows j0, j0 + 1
    V r[4][2], W[2], E[2], fv[2][2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 - 1 + q;
      if (j >= 0 && j < nt) ld_pair(r[q][0], r[q][1], ep + size_t(j) * nr + i0);
      else r[q][0] = r[q][1] = z;
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const size_t row = size_t(j0 + b) * nr;
      W[b] = i0 > 0 ? ep[row + i0 - 1] : z;
      E[b] = i0 + 2 < nr ? ep[row + i0 + 2] : z;
      ld_pair(fv[b][0], fv[b][1], fp + row + i0);
    }
    T ax = 0, ay = 0;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int i = i0 + a, j = j0 + b;
        const V c = r[b + 1][a];
        const V Ev = a ? E[b] : r[b + 1][1];
        const V Wv = a ? r[b + 1][0] : W[b];
        const V N = r[b + 2][a], S = r[b][a];
        const T aE = RTAB(rt, RT_AE, i + 1), aW = RTAB(rt, RT_AW, i + 1), P = RTAB(rt, RT_P, i + 1);
        const T aN = P * TTAB(tt, TT_AN, j + 1), aS = P * TTAB(tt, TT_AS, j + 1);
        const T d = fmac(-(s2 * RTAB(rt, RT_Q, i + 1)), TTAB(tt, TT_T, j + 1),
                         fmac(P, TTAB(tt, TT_DT, j + 1), RTAB(rt, RT_DR, i + 1)));
        const T rx = fv[b][a].x - fmac(d, c.x, fmac(aS, S.x, fmac(aN, N.x, fmac(aW, Wv.x, aE * Ev.x))));
        const T ry = fv[b][a].y - fmac(d, c.y, fmac(aS, S.y, fmac(aN, N.y, fmac(aW, Wv.y, aE * Ev.y))));
        const T wgt = RTAB(rt, RT_RW, i + 1) * TTAB(tt, TT_RW, j + 1);
        ax = fmac(wgt, rx, ax);
        ay = fmac(wgt, ry, ay);
      }
    fc[size_t(p) * nc + cidx] = vmk<V, T>(ax, ay);
  }
}

template <typename T>
void launch_restrict(const LevelDev& F, const LevelDev& C, const Batch& B, const vec2_t<T>* e,
                     const vec2_t<T>* f, vec2_t<T>* fc, cudaStream_t st) {
  const int n = C.nr * C.nt;
  k_restrict<T><<<work_grid(long((n + 255) / 256) * B.max_planes), 256, 0, st>>>(F, C, B, e, f, fc);
}

// ---------------------------------------------------------------------------
// Bilinear prolongation in (r^2, theta) / (R, z) and correction (Sec. 3.1).
// ---------------------------------------------------------------------------
// e += P ec over the active planes: one thread per coarse cell (I, J) updates
// its four children (2I + a, 2J + b) from the 3 x 3 coarse neighbourhood,
// loaded once (ghosts by the coarse level's rules, chosen per column and row);
// the children of one row are an aligned pair.  The values and the order of
// operations are those of s_prolong in the fused kernel.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(LevelDev L, LevelDev C, Batch B,
                                                 vec2_t<T>* __restrict__ e,
                                                 const vec2_t<T>* __restrict__ ec) {
  typedef vec2_t<T> V;
  const int nact = *B.nact, nc = C.nr * C.nt, n = L.nr * L.nt;
  const int bpp = (nc + blockDim.x - 1) / blockDim.x;
  const T* rt = rtab<T>(L);
  const T* tt = ttab<T>(L);
  for (int w = blockIdx.x; w < nact * bpp; w += gridDim.x) {
    const int k = w / bpp;
    const int q = (w - k * bpp) * blockDim.x + threadIdx.x;
    if (q >= nc) continue;
    const int p = B.act[k];
    const int slot = B.slot ? B.slot[p] : p;
    const bool odd = (B.mode[slot] & 1) != 0;
    const int J = q / C.nr, I = q - J * C.nr;
    const V* ecp = ec + size_t(p) * nc;
    int ic[3], jc[3];
    bool zc[3], zr[3], nc_[3], nr_[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {   // 1-based coarse column I + u and row J + u
      const int x = I + u, rx = x == 0 ? C.gL : (x == C.nr + 1 ? C.gR : -1);
      ic[u] = min(max(x, 1), C.nr) - 1;
      zc[u] = rx == GH_ZERO;
      nc_[u] = rx == GH_PARITY && odd;
      const int y = J + u, ry = y == 0 ? C.gB : (y == C.nt + 1 ? C.gT : -1);
      jc[u] = min(max(y, 1), C.nt) - 1;
      zr[u] = ry == GH_ZERO;
      nr_[u] = ry == GH_PARITY && odd;
    }
    V cv[3][3];
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const V x = ecp[size_t(jc[v]) * C.nr + ic[u]];
        V r;
        r.x = (zc[u] || zr[v]) ? T(0) : ((nc_[u] != nr_[v]) ? -x.x : x.x);
        r.y = (zc[u] || zr[v]) ? T(0) : ((nc_[u] != nr_[v]) ? -x.y : x.y);
        cv[v][u] = r;
      }
    const int i0 = 2 * I;
    const T p1a = RTAB(rt, RT_P1, i0 + 1), p2a = RTAB(rt, RT_P2, i0 + 1);
    const T p1b = RTAB(rt, RT_P1, i0 + 2), p2b = RTAB(rt, RT_P2, i0 + 2);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int j = 2 * J + b;
      const T q1 = TTAB(tt, TT_P1, j + 1), q2 = TTAB(tt, TT_P2, j + 1);
      V* row = e + size_t(p) * n + size_t(j) * L.nr + i0;
      V uu[2];
      ld_pair(uu[0], uu[1], row);
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const T p1 = a ? p1b : p1a, p2 = a ? p2b : p2a;
        const V A = cv[b][a], Bv = cv[b][a + 1], Cv = cv[b + 1][a], D = cv[b + 1][a + 1];
        const T w11 = p1 * q1, w21 = p2 * q1, w12 = p1 * q2, w22 = p2 * q2;
        uu[a].x += fmac(w22, D.x, fmac(w12, Cv.x, fmac(w21, Bv.x, w11 * A.x)));
        uu[a].y += fmac(w22, D.y, fmac(w12, Cv.y, fmac(w21, Bv.y, w11 * A.y)));
      }
      st_pair(row, uu[0], uu[1]);
    }
  }
}

template <typename T>
void launch_prolong(const LevelDev& F, const LevelDev& C, const Batch& B, vec2_t<T>* e,
                    const vec2_t<T>* ec, cudaStream_t st) {
  const int n = C.nr * C.nt;
  k_prolong<T><<<work_grid(long((n + 255) / 256) * B.max_planes), 256, 0, st>>>(F, C, B, e, ec);
}

// ---------------------------------------------------------------------------
// FP64 solution update and residual with per-plane norms (the outer loop of
// the mixed-precision iterative refinement, and of the FP64 path).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_update(int n, Batch B, double2* __restrict__ u, const vec2_t<T>* __restrict__ e) {
  const int nact = *B.nact, bpp = (n + blockDim.x - 1) / blockDim.x;
  for (int w = blockIdx.x; w < nact * bpp; w += gridDim.x) {
    const int k = w / bpp;
    const int idx = (w - k * bpp) * blockDim.x + threadIdx.x;
    if (idx >= n) continue;
    const size_t o = size_t(B.act[k]) * n + idx;
    const vec2_t<T> v = e[o];
    double2 x = u[o];
    x.x += from_buf<T>(v.x);
    x.y += from_buf<T>(v.y);
    u[o] = x;
  }
}

template <typename T>
void launch_update(const LevelDev& L, const Batch& B, double2* u, const vec2_t<T>* e,
                   cudaStream_t st) {
  const int n = L.nr * L.nt;
  k_update<T><<<work_grid(long((n + 255) / 256) * B.max_planes), 256, 0, st>>>(n, B, u, e);
}

int residual_blocks(int nr, int nt) {
  work_grid(1);   // queries the SM count once, outside any stream capture
  return (nr * nt + 255) / 256;
}

__device__ void retire_block(int* act, int* nact, const Sum4* __restrict__ psum, RetireState S,
                             double tol, int max_cycles, int stagnation, int use_cond,
                             unsigned long long handle, int* scan, int tail_planes);

// FP64 defect at (i, j) from the per-cell products (one FP64 operation for
// the mode's diagonal read from its own table dm, five fused multiply-adds per
// component starting from the right-hand side).
__device__ __forceinline__ double2 defect_tab(const LevelDev& L, const double* __restrict__ ct,
                                              const double* __restrict__ dm, int n,
                                              const double2* __restrict__ e,
                                              const double2* __restrict__ f, int i, int j) {
  const int nr = L.nr, nt = L.nt, idx = j * nr + i;
  const double2 c = e[idx];
  const double2 E = (i + 1 < nr) ? e[idx + 1] : make_double2(0.0, 0.0);
  const double2 W = (i > 0) ? e[idx - 1] : make_double2(0.0, 0.0);
  const double2 N = (j + 1 < nt) ? e[idx + nr] : make_double2(0.0, 0.0);
  const double2 S = (j > 0) ? e[idx - nr] : make_double2(0.0, 0.0);
  const double aE = RTAB(L.rd, RT_AE, i + 1), aW = RTAB(L.rd, RT_AW, i + 1);
  const double aN = ct[idx], aS = ct[n + idx];
  const double d = dm[idx];
  const double2 fv = f[idx];
  double rx = fma(-aE, E.x, fv.x), ry = fma(-aE, E.y, fv.y);
  rx = fma(-aW, W.x, rx);
  ry = fma(-aW, W.y, ry);
  rx = fma(-aN, N.x, rx);
  ry = fma(-aN, N.y, ry);
  rx = fma(-aS, S.x, rx);
  ry = fma(-aS, S.y, ry);
  return make_double2(fma(-d, c.x, rx), fma(-d, c.y, ry));
}


// The four sums of one work item or block, combined across a warp (lane 0).
__device__ __forceinline__ SqPart sq_warp_sum4(const SqPart& q) {
  SqPart t;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const SqAcc a = sq_warp_sum(SqAcc{q.s[c], q.e[c]});
    t.s[c] = a.s;
    t.e[c] = a.e;
  }
  return t;
}
__device__ __forceinline__ SqPart sq_part(SqAcc x, SqAcc y, SqAcc z, SqAcc w) {
  SqPart q;
  q.s[0] = x.s; q.s[1] = y.s; q.s[2] = z.s; q.s[3] = w.s;
  q.e[0] = x.e; q.e[1] = y.e; q.e[2] = z.e; q.e[3] = w.e;
  return q;
}
__device__ __forceinline__ SqPart sq_part_zero() {
  const SqAcc z = sq_zero();
  return sq_part(z, z, z, z);
}
// Warp 0 combines the per-warp sums the block left in sh[0 .. nw).
__device__ __forceinline__ SqPart sq_block_tail(const SqPart* sh, int lane, int nw) {
  return sq_warp_sum4(lane < nw ? sh[lane] : sq_part_zero());
}

// The residual work items of one launch.  ZERO: u = 0 on the first
// iteration, so r = f and |r|^2 = |f|^2 (no stencil); CPT: cells per thread
// and work item.  Both are fixed per launch, so each combination is its own
// loop and no branch of the other remains in the cell loop.
template <typename T, bool ZERO, int CPT>
__device__ __forceinline__ void residual_items(const LevelDev& L, const Batch& B,
                                               const double2* __restrict__ f,
                                               const double2* __restrict__ u,
                                               vec2_t<T>* __restrict__ r, SqPart* part, Sum4* psum,
                                               int* cnt, int bpp, const RetireArgs& ra,
                                               const double* __restrict__ ctab,
                                               const double* __restrict__ dtab, int nact,
                                               bool want_f, SqPart* sh, int* flag, int* scan) {
  const int nr = L.nr, nt = L.nt, n = nr * nt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = int(blockDim.x >> 5);
  const int ipp = (bpp + CPT - 1) / CPT;   // items per plane
  for (int w = blockIdx.x; w < nact * ipp; w += gridDim.x) {
    const int k = w / ipp, bx = w - k * ipp;
    const int p = B.act[k];
    const int slot = B.slot ? B.slot[p] : p;
    const size_t base = size_t(p) * n;
    // the residual is FP64; its norm only drives the convergence test, so
    // the volume-weighted squares of its FP32 rounding are summed in FP32
    // (SqAcc: exact power-of-two scaling, no under- or overflow)
    SqAcc ax = sq_zero(), ay = sq_zero(), az = sq_zero(), aw = sq_zero();
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int idx = (bx * CPT + c) * blockDim.x + threadIdx.x;
      if (idx < n) {
        const int j = idx / nr, i = idx - j * nr;
        double2 rv;
        if constexpr (ZERO) rv = f[base + idx];
        else rv = defect_tab(L, ctab, dtab + size_t(slot) * n, n, u + base, f + base, i, j);
        const vec2_t<T> ro = vmk<vec2_t<T>, T>(to_buf<T>(rv.x), to_buf<T>(rv.y));
        r[base + idx] = ro;
        const float dv = L.rf[RT_V * (nr + 2) + i + 1] * L.tf[TT_V * (nt + 2) + j + 1];
        sq_add(ax, ro.x, dv);   // the residual as stored: FP32 values, or FP64 ones
        sq_add(ay, ro.y, dv);
        if (!ZERO && want_f) {
          const double2 fv = f[base + idx];
          sq_add(az, fv.x, dv);
          sq_add(aw, fv.y, dv);
        }
      }
    }
    ax = sq_warp_sum(ax);
    ay = sq_warp_sum(ay);
    if (ZERO) {   // r = f: the same sums
      az = ax;
      aw = ay;
    } else if (want_f) {
      az = sq_warp_sum(az);
      aw = sq_warp_sum(aw);
    }
    if (lane == 0) sh[warp] = sq_part(ax, ay, az, aw);
    __syncthreads();
    if (warp == 0) {
      const SqPart t = sq_block_tail(sh, lane, nw);
      if (lane == 0) {
        part[size_t(p) * bpp + bx] = t;
        __threadfence();
        flag[0] = (atomicAdd(&cnt[p], 1) == ipp - 1);
      }
    }
    __syncthreads();
    if (flag[0]) {   // the plane's last item: its sums over the items in item order
      __threadfence();
      SqPart t = sq_part_zero();
      for (int b = threadIdx.x; b < ipp; b += blockDim.x) {
        const SqPart* q = &part[size_t(p) * bpp + b];
        const float4 qs = __ldcg(reinterpret_cast<const float4*>(q->s));
        const int4 qb = __ldcg(reinterpret_cast<const int4*>(q->e));
        const float vs[4] = {qs.x, qs.y, qs.z, qs.w};
        const int vb[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const SqAcc m = sq_merge(SqAcc{t.s[c], t.e[c]}, SqAcc{vs[c], vb[c]});
          t.s[c] = m.s;
          t.e[c] = m.e;
        }
      }
      t = sq_warp_sum4(t);
      if (lane == 0) sh[warp] = t;   // warp 0 read sh before the barrier above
      __syncthreads();
      if (warp == 0) {
        const SqPart q = sq_block_tail(sh, lane, nw);
        if (lane == 0) {
          psum[p] = sum4(sq_value(SqAcc{q.s[0], q.e[0]}), sq_value(SqAcc{q.s[1], q.e[1]}),
                         sq_value(SqAcc{q.s[2], q.e[2]}), sq_value(SqAcc{q.s[3], q.e[3]}));
          cnt[p] = 0;
          __threadfence();
          flag[1] = (atomicAdd(ra.gcnt, 1) == nact - 1);
        }
      }
      __syncthreads();
      if (flag[1]) {   // every plane's sum is in: retire converged planes (App. B)
        __threadfence();
        retire_block(const_cast<int*>(B.act), const_cast<int*>(B.nact), psum, ra.S, ra.tol,
                     ra.max_cycles, ra.stagnation, ra.use_cond, ra.handle, scan, ra.tail_planes);
        if (threadIdx.x == 0) *ra.gcnt = 0;
      }
    }
    __syncthreads();   // sh and flag are reused by the next work item
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_residual(LevelDev L, Batch B, const double2* __restrict__ f,
                                                  const double2* __restrict__ u,
                                                  vec2_t<T>* __restrict__ r, SqPart* part,
                                                  Sum4* psum, int* cnt, int bpp, RetireArgs ra,
                                                  const double* __restrict__ ctab,
                                                  const double* __restrict__ dtab) {
  __shared__ SqPart sh[8];
  __shared__ int flag[2];
  __shared__ int scan[256];
  // nact is read once: the retiring block rewrites it only after every work
  // item of this launch has been summed
  const int nact = *B.nact;
  const bool want_f = *ra.S.iter == 0;     // |f| is needed on the first iteration only
  // from a zero initial guess the first defect is f itself (no stencil)
  const bool r_is_f = want_f && ra.zero_guess;
  // Work items of CPT x 256 cells: with many planes active the per-item
  // reduction, fence and arrival count are paid once per 1024 cells; with few
  // planes every item is 256 cells, spreading a plane's FP64 work over more
  // SMs.  bpp (the caller's) is the item count for CPT = 1.
  if (r_is_f) {
    if (nact >= 16)
      residual_items<T, true, 4>(L, B, f, u, r, part, psum, cnt, bpp, ra, ctab, dtab, nact, want_f, sh, flag, scan);
    else
      residual_items<T, true, 1>(L, B, f, u, r, part, psum, cnt, bpp, ra, ctab, dtab, nact, want_f, sh, flag, scan);
  } else {
    if (nact >= 16)
      residual_items<T, false, 4>(L, B, f, u, r, part, psum, cnt, bpp, ra, ctab, dtab, nact, want_f, sh, flag, scan);
    else
      residual_items<T, false, 1>(L, B, f, u, r, part, psum, cnt, bpp, ra, ctab, dtab, nact, want_f, sh, flag, scan);
  }
}

template <typename T>
void launch_residual(const LevelDev& L, const Batch& B, const double2* f, const double2* u,
                     vec2_t<T>* r, SqPart* part, Sum4* psum, int* cnt, const RetireArgs& ra,
                     cudaStream_t st, const double* ctab, const double* dtab) {
  const int bpp = residual_blocks(L.nr, L.nt);
  k_residual<T><<<work_grid(long(bpp) * B.max_planes), 256, 0, st>>>(L, B, f, u, r, part, psum,
                                                                       cnt, bpp, ra, ctab, dtab);
}

// ---------------------------------------------------------------------------
// Retirement (App. B criterion, per mode and component) and compaction.
// ---------------------------------------------------------------------------

__device__ void retire_block(int* act, int* nact, const Sum4* __restrict__ psum, RetireState S,
                             double tol, int max_cycles, int stagnation, int use_cond,
                             unsigned long long handle, int* scan, int tail_planes) {
  __shared__ double smax[32];
  __shared__ int base_out;
  const int n = *nact;
  const int iter = *S.iter;
  const int tid = threadIdx.x;
  if (iter == 0) {
    double mx = 0.0;
    for (int k = tid; k < n; k += blockDim.x) {
      const int p = act[k];
      const Sum4 s = psum[p];
      S.nf2[p] = make_double2(s.z, s.w);
      mx = fmax(mx, fmax(s.z, s.w));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) smax[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0.0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) m2 = fmax(m2, smax[w]);
      *S.fmax2 = m2;
    }
    __syncthreads();
  }
  const double floor2 = 1e-28 * (*S.fmax2);
  const double tol2 = tol * tol;
  if (tid == 0) base_out = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += blockDim.x) {
    const int k = c0 + tid;
    int keep = 0, p = -1;
    if (k < n) {
      p = act[k];
      const Sum4 s = psum[p];
      const double2 nf = S.nf2[p];
      const double2 prev = S.nr2[p];
      const double tre = tol2 * fmax(nf.x, floor2), tim = tol2 * fmax(nf.y, floor2);
      int st = ST_ACTIVE;
      if (!isfinite(s.x) || !isfinite(s.y)) st = ST_NONFINITE;
      else if (s.x <= tre && s.y <= tim) st = ST_OK;
      else if (iter >= max_cycles) st = ST_NOTCONV;
      else if (stagnation && iter >= 3 && s.x + s.y > 0.81 * (prev.x + prev.y)) st = ST_STAGNATED;
      S.nr2[p] = make_double2(s.x, s.y);
      S.cycles[p] = iter;
      S.status[p] = st;
      keep = (st == ST_ACTIVE);
    }
    // compaction: rank within the warp from a ballot, warp offsets from an
    // exclusive prefix over the block's warps
    const int lane = tid & 31, wid = tid >> 5, nw = int(blockDim.x >> 5);
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) scan[wid] = __popc(bal);
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int w = 0; w < nw; ++w) {
        const int c = scan[w];
        scan[w] = acc;
        acc += c;
      }
      scan[nw] = acc;
    }
    __syncthreads();
    if (keep) act[base_out + scan[wid] + __popc(bal & ((1u << lane) - 1u))] = p;
    __syncthreads();
    if (tid == 0) base_out += scan[nw];
    __syncthreads();
  }
  if (tid == 0) {
    // continue flag: 0 done, 1 another batched iteration, 2 this iteration's
    // V-cycle and update, then the tail kernel finishes the remaining planes
    const int cont = base_out == 0 ? 0 : (base_out > tail_planes ? 1 : 2);
    *nact = base_out;
    *S.iter = iter + 1;
    *S.cont = cont;
    if (use_cond) cudaGraphSetConditional(handle, cont == 1 ? 1u : 0u);
  }
}

__global__ void k_init_active(int* act, int* nact, int n, RetireState S) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    act[k] = k;
    S.cycles[k] = 0;
    S.status[k] = ST_ACTIVE;
    S.nr2[k] = make_double2(0.0, 0.0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *nact = n;
    *S.iter = 0;
    *S.cont = 1;
  }
}

void launch_init_active(int* act, int* nact, int n, RetireState S, cudaStream_t st) {
  k_init_active<<<(n + 255) / 256, 256, 0, st>>>(act, nact, n, S);
}

#define INST(T)                                                                                  \
  template void launch_restrict<T>(const LevelDev&, const LevelDev&, const Batch&,               \
                                   const vec2_t<T>*, const vec2_t<T>*, vec2_t<T>*, cudaStream_t); \
  template void launch_prolong<T>(const LevelDev&, const LevelDev&, const Batch&, vec2_t<T>*,   \
                                  const vec2_t<T>*, cudaStream_t);                               \
  template void launch_update<T>(const LevelDev&, const Batch&, double2*, const vec2_t<T>*,     \
                                 cudaStream_t);                                                  \
  template void launch_residual<T>(const LevelDev&, const Batch&, const double2*,               \
                                   const double2*, vec2_t<T>*, SqPart*, Sum4*, int*,      \
                                   const RetireArgs&, cudaStream_t, const double*, const double*);
INST(float)
INST(double)

}  // namespace ps
