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
// (halo rows).  n_sor even-odd SOR sweeps move information at most 2 n_sor
// cells along the line, so the values the CTA keeps -- its own rows -- are
// exactly those of a relaxation of the whole line.  A level's error lives in
// the CTA's own rows and two buffers of halo rows used in turn: a step reads
// halo buffer b and updates the own rows, then writes its boundary rows into
// the neighbours' halo buffer b^1 (distributed shared memory stores), and the
// cluster synchronises once; a CTA still reading buffer b never sees a
// neighbour's newer rows.  The two
// radial colours share one step: a CTA recomputes the neighbour's first
// colour-0 row that its own last colour-1 row needs.  Prolongation is
// computed by each CTA for its halo rows too (it holds the coarse rows they
// need), so the halo stays current without an exchange.
//
// Row storage: cell (j, i) of a level sits at column i ^ sw(j) of its row,
// with sw(j) = (j / 2) mod min(8, n_r / 2).  The 8 lanes that relax a polar
// segment (two rows each) then read 8 distinct 8-byte slots, and the four
// columns of a warp pass are chosen so that two of them fall in each half
// of a 16-column block: a column load takes the minimum two wavefronts.  A
// radial line still reads whole 16-byte pairs (the line helpers swap a pair
// for odd sw).
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
static_assert(sizeof(D4) == sizeof(SqPart) && alignof(D4) == alignof(SqPart),
              "the warp sums reuse the D4 reduction slots");

__device__ __forceinline__ V vz() { return make_float2(0.f, 0.f); }

// Row r (relative to the CTA's first row, -h <= r < s + h) of a row block
// (the right-hand side, rows -h .. s + h - 1 contiguous).
__device__ __forceinline__ V* rowp(unsigned char* sm, int off, int nr, int h, int r) {
  return reinterpret_cast<V*>(sm) + off + (r + h) * nr;
}
// Row r of a level's error seen with halo buffer b.
__device__ __forceinline__ V* erow(unsigned char* sm, const TailLevel& t, int h, int b, int r) {
  V* base = reinterpret_cast<V*>(sm);
  const int nr = t.L.nr;
  if (r < 0) return base + t.eh[b] + (r + h) * nr;
  if (r >= t.s) return base + t.eh[b] + (h + r - t.s) * nr;
  return base + t.eo + r * nr;
}
// Column swizzle of global row j.
__device__ __forceinline__ int tsw(int nr, int j) { return (j >> 1) & ((nr < 16 ? nr : 16) / 2 - 1); }

// Copies the own rows [r0, r1) (row r at src + r nr) to CTA tgt, whose own
// rows start delta rows after ours (our row r is its row r - delta): into its
// right-hand-side block at dst (eblock = 0) or its error halo buffer at dst
// (eblock = 1: rows above its own at slots 0..h-1, below at h..2h-1).
__device__ void push_rows(cg::cluster_group& cl, unsigned char* sm, const V* src, int dst, int eblock,
                          int s, int nr, int h, int r0, int r1, int tgt, int delta) {
  if (r1 <= r0) return;
  const int chunks = nr >> 1;   // two cells per 16-byte store
  V* tb = cl.map_shared_rank(reinterpret_cast<V*>(sm), tgt);
  const int n = (r1 - r0) * chunks;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int q = idx / chunks, c = idx - q * chunks, r = r0 + q, rt = r - delta;
    const int slot = !eblock ? rt + h : (rt < 0 ? rt + h : h + rt - s);
    *reinterpret_cast<float4*>(tb + dst + slot * nr + 2 * c) =
        *reinterpret_cast<const float4*>(src + r * nr + 2 * c);
  }
}

// The CTA's own rows into the halo rows of every CTA whose halo (h rows on
// each side) covers them.
__device__ void push_halo(cg::cluster_group& cl, unsigned char* sm, const V* src, int dst, int eblock,
                          int s, int nr, int h, int rank, int C) {
  for (int d = 1; (d - 1) * s < h; ++d) {
    if (rank + d < C) push_rows(cl, sm, src, dst, eblock, s, nr, h, max(0, d * s - h), s, rank + d, d * s);
    if (rank - d >= 0) push_rows(cl, sm, src, dst, eblock, s, nr, h, 0, min(s, h - (d - 1) * s), rank - d, -d * s);
  }
}

// ---- neighbour signalling for the smoothing steps ---------------------------
// A smoothing step ends with the CTA's boundary rows stored into the
// neighbours' halo buffer b^1 by asynchronous distributed-shared-memory
// stores that also count their bytes on the receiver's mbarrier of that
// buffer (st.async ... complete_tx); the receiver announces the bytes it
// expects and waits for that mbarrier phase.  So a CTA waits only for the
// CTAs whose rows it reads, not for the whole cluster, and no memory fence
// is needed.  Every CTA that sends to a CTA also receives from it (the halos
// are symmetric), so neighbours are never more than one step apart: a
// buffer is not rewritten before its reader has finished the step that
// reads it, and one phase's bytes never mix with the next phase's.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return unsigned(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned peer_u32(unsigned local, int rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait (about one second of polling at the maximum SM clock); false
// when it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}
__device__ __forceinline__ void st_async16(unsigned addr, float4 v, unsigned bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
      "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
      "r"(__float_as_uint(v.w)), "r"(bar)
      : "memory");
}

// Own rows [r0, r1) into CTA tgt's error halo buffer at dst (slots as
// push_rows with eblock = 1), counted on tgt's mbarrier `bar` (local address).
__device__ void push_rows_async(unsigned char* sm, const V* src, int dst, int s, int nr, int h, int r0,
                                int r1, int tgt, int delta, unsigned bar) {
  if (r1 <= r0) return;
  const unsigned rb = peer_u32(smem_u32(sm), tgt), rbar = peer_u32(bar, tgt);
  const int chunks = nr >> 1;
  const int n = (r1 - r0) * chunks;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int q = idx / chunks, c = idx - q * chunks, r = r0 + q, rt = r - delta;
    const int slot = rt < 0 ? rt + h : h + rt - s;
    st_async16(rb + unsigned((dst + slot * nr + 2 * c) * sizeof(V)),
               *reinterpret_cast<const float4*>(src + r * nr + 2 * c), rbar);
  }
}

// Halo rows a CTA receives per step: from rank - d its rows
// [max(0, d s - h), s), from rank + d its rows [0, min(s, h - (d - 1) s)).
__device__ __forceinline__ int halo_rows_in(int s, int h, int rank, int C) {
  int n = 0;
  for (int d = 1; (d - 1) * s < h; ++d) {
    if (rank - d >= 0) n += s - max(0, d * s - h);
    if (rank + d < C) n += min(s, h - (d - 1) * s);
  }
  return n;
}

// End of a smoothing step: the own rows into the neighbours' halo buffer
// b^1, then wait until the neighbours' rows have arrived in ours.  `bars`:
// local addresses of this level's two mbarriers; bit pb + b of `phase` is
// the parity of the next completion of mbarrier b.  A wait that gives up
// sets `dead`.
__device__ void publish_wait(unsigned char* sm, const TailLevel& t, int h, int b, int rank, int C,
                             const unsigned* bars, unsigned& phase, int pb, bool& dead) {
  const V* src = reinterpret_cast<const V*>(sm) + t.eo;
  const int s = t.s, nr = t.L.nr, bn = b ^ 1;
  for (int d = 1; (d - 1) * s < h; ++d) {
    if (rank + d < C) push_rows_async(sm, src, t.eh[bn], s, nr, h, max(0, d * s - h), s, rank + d, d * s, bars[bn]);
    if (rank - d >= 0)
      push_rows_async(sm, src, t.eh[bn], s, nr, h, 0, min(s, h - (d - 1) * s), rank - d, -d * s, bars[bn]);
  }
  if (threadIdx.x == 0)
    mbar_expect(bars[bn], unsigned(halo_rows_in(s, h, rank, C) * nr * int(sizeof(V))));
  if (!dead && !mbar_wait(bars[bn], (phase >> (pb + bn)) & 1u)) dead = true;
  phase ^= 1u << (pb + bn);
  __syncthreads();   // the next step rewrites the own rows this step sent
}

// One radial line (own row r, or the first row of the next CTA) relaxed in
// place (Sec. 3.2; the helpers of the level-wide pass), halo buffer b.
template <int CPL>
__device__ __forceinline__ void t_rline(const LevelDev& L, const RLineTabs<float, CPL>& tabs,
                                        unsigned char* sm, const TailLevel& t, int h, int b, int j0,
                                        int r, float s2, int n_sor) {
  const int lane = threadIdx.x & 31, nr = L.nr, nt = L.nt, j = j0 + r;
  V ev[CPL], g[CPL], un[CPL], us[CPL];
  V* row = erow(sm, t, h, b, r);
  ld_line_swz<V, CPL>(ev, row, tsw(nr, j), lane, nr);
  ld_line_swz<V, CPL>(g, rowp(sm, t.fo, nr, h, r), tsw(nr, j), lane, nr);
  if (j + 1 < nt) {
    ld_line_swz<V, CPL>(un, erow(sm, t, h, b, r + 1), tsw(nr, j + 1), lane, nr);
  } else {
#pragma unroll
    for (int c = 0; c < CPL; ++c) un[c] = vz();
  }
  if (j > 0) {
    ld_line_swz<V, CPL>(us, erow(sm, t, h, b, r - 1), tsw(nr, j - 1), lane, nr);
  } else {
#pragma unroll
    for (int c = 0; c < CPL; ++c) us[c] = vz();
  }
  relax_r<float, CPL>(L, tabs, L.tf, s2, L.omr_f[j], j, g, un, us, n_sor, ev);
  st_line_swz<V, CPL>(row, tsw(nr, j), ev, lane, nr);
}

// Both radial colours of the own rows, one warp per line: colour 0 (even
// rows, and the next CTA's first row -- in the halo buffer -- which the own
// last colour-1 row needs: its inputs are the own last row, the halo rows
// and the halo right-hand side, so the value equals the neighbour's), then
// colour 1.
template <int CPL>
__device__ void t_rpass(const LevelDev& L, unsigned char* sm, const TailLevel& t, int h, int b,
                        int j0, float s2, int n_sor) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  RLineTabs<float, CPL> tabs;
  ld_rtabs<float, CPL>(tabs, L, L.rf);
  const int n0 = t.s / 2 + (j0 + t.s < L.nt ? 1 : 0);
  for (int w = warp; w < n0; w += nw) t_rline<CPL>(L, tabs, sm, t, h, b, j0, 2 * w, s2, n_sor);
  __syncthreads();
  for (int w = warp; w < t.s / 2; w += nw) t_rline<CPL>(L, tabs, sm, t, h, b, j0, 2 * w + 1, s2, n_sor);
}

__device__ void t_rstep(const LevelDev& L, unsigned char* sm, const TailLevel& t, int h, int b,
                        int j0, float s2, int n_sor) {
  switch (L.nr <= 32 ? 1 : L.nr >> 5) {
    case 1: t_rpass<1>(L, sm, t, h, b, j0, s2, n_sor); break;
    case 2: t_rpass<2>(L, sm, t, h, b, j0, s2, n_sor); break;
    case 4: t_rpass<4>(L, sm, t, h, b, j0, s2, n_sor); break;
    default: t_rpass<8>(L, sm, t, h, b, j0, s2, n_sor); break;
  }
}

// Polar lines of colour `color`: LPC lanes relax one column's segment of
// rows [rlo, rhi) (own rows and up to h halo rows each side, clipped to the
// plane), each lane two consecutive rows (an even and an odd global row), with
// the even-odd SOR sweeps of the line smoother: an even row's neighbours are
// the lane's odd row and the previous lane's odd row (a shuffle), an odd
// row's the lane's even row and the next lane's even row.  32 / LPC columns
// per warp pass; the own rows are kept.  The segment starts at an even row
// (h and the CTA's first row are even).
template <int LPC>
__device__ void t_tcols(const LevelDev& L, unsigned char* sm, const TailLevel& t, int h, int b,
                        int j0, float s2, int n_sor, int color) {
  const int nr = L.nr, nt = L.nt, NR = nr + 2, NT = nt + 2;
  const float* rt = L.rf;
  const float* tt = L.tf;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int per = 32 / LPC;
  const int sub = lane / LPC, k = lane - sub * LPC;
  const int rlo = max(-h, -j0), rhi = min(t.s + h, nt - j0);
  // the lane's rows r0 (even global row) and r0 + 1, and their coefficients
  const int r0 = rlo + 2 * k;
  bool on[2];
  int rr[2], sw[2];
  float dtj[2], tj[2], anj[2], asj[2];
  V* er[2];
  const V* fr[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    on[c] = r0 + c < rhi;
    rr[c] = on[c] ? r0 + c : rlo;
    const int j = j0 + rr[c];
    sw[c] = tsw(nr, j);
    er[c] = erow(sm, t, h, b, rr[c]);
    fr[c] = rowp(sm, t.fo, nr, h, rr[c]);
    dtj[c] = tt[TT_DT * NT + j + 1];
    tj[c] = tt[TT_T * NT + j + 1];
    anj[c] = tt[TT_AN * NT + j + 1];
    asj[c] = tt[TT_AS * NT + j + 1];
  }
  const bool first = k == 0;
  const int ncol = nr >> 1;   // columns of this colour: a multiple of 8
  // pass p takes, from the block of 8 columns u = p / (8 / per), offsets
  // {0, 1, 4, 5} (+2 on odd passes) for four groups, {0, 4} (+0..3) for two
  const int passes = ncol / per;
  for (int p = warp; p < passes; p += nw) {   // the same trip count on every lane
    const int u = p / (8 / per), v = p - u * (8 / per);
    const int q = 8 * u + (per == 4 ? 2 * v + (sub & 1) + 4 * (sub >> 1) : v + 4 * sub);
    const int i = 2 * q + color;
    const float P = rt[RT_P * NR + i + 1], aE = rt[RT_AE * NR + i + 1], aW = rt[RT_AW * NR + i + 1];
    const float dr = rt[RT_DR * NR + i + 1], Qi = rt[RT_Q * NR + i + 1];
    const float w = L.omt_f[i], w1 = 1.0f - w;
    V x[2], g[2];
    float up[2], dn[2], id[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      x[c] = g[c] = vz();
      up[c] = dn[c] = id[c] = 0.f;
      if (on[c]) {
        const V* e = er[c];
        x[c] = e[i ^ sw[c]];
        const V ue = (i + 1 < nr) ? e[(i + 1) ^ sw[c]] : vz();
        const V uw = (i > 0) ? e[(i - 1) ^ sw[c]] : vz();
        const V fv = fr[c][i ^ sw[c]];
        g[c].x = fv.x - aE * ue.x - aW * uw.x;
        g[c].y = fv.y - aE * ue.y - aW * uw.y;
        id[c] = rcp_diag(dr + P * dtj[c] - s2 * Qi * tj[c]);
        up[c] = P * anj[c];
        dn[c] = P * asj[c];
      }
    }
    for (int it = 0; it < n_sor; ++it) {
      {   // even rows: below, the previous lane's odd row; above, the own odd row
        V em = shup(x[1]);
        if (first) em = vz();
        const float tx = (g[0].x - up[0] * x[1].x - dn[0] * em.x) * id[0];
        const float ty = (g[0].y - up[0] * x[1].y - dn[0] * em.y) * id[0];
        x[0].x = w1 * x[0].x + w * tx;
        x[0].y = w1 * x[0].y + w * ty;
      }
      {   // odd rows: below, the own even row; above, the next lane's even row
        V ep = shdn(x[0]);
        if (k == LPC - 1) ep = vz();
        const float tx = (g[1].x - up[1] * ep.x - dn[1] * x[0].x) * id[1];
        const float ty = (g[1].y - up[1] * ep.y - dn[1] * x[0].y) * id[1];
        x[1].x = w1 * x[1].x + w * tx;
        x[1].y = w1 * x[1].y + w * ty;
      }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (on[c] && rr[c] >= 0 && rr[c] < t.s) er[c][i ^ sw[c]] = x[c];
  }
}

__device__ void t_tstep(const LevelDev& L, unsigned char* sm, const TailLevel& t, int h, int b,
                        int j0, float s2, int n_sor, int color) {
  if (t.s + 2 * h <= 16) t_tcols<8>(L, sm, t, h, b, j0, s2, n_sor, color);
  else t_tcols<16>(L, sm, t, h, b, j0, s2, n_sor, color);
}

// `cycles` smoothing cycles of one level (Algorithm 1: radial lines, then
// polar lines, each in zebra order); after each step the own rows are
// published to the neighbours, whose rows are awaited.
__device__ void t_smooth(const LevelDev& L, unsigned char* sm, const TailLevel& t, int h, int& b,
                         int rank, int C, float s2, int n_sor, int cycles, const unsigned* bars,
                         unsigned& phase, int pb, bool& dead) {
  const int j0 = rank * t.s;
  for (int cyc = 0; cyc < cycles; ++cyc)
    for (int step = 0; step < 3; ++step) {
      if (step == 0) t_rstep(L, sm, t, h, b, j0, s2, n_sor);
      else t_tstep(L, sm, t, h, b, j0, s2, n_sor, step - 1);
      __syncthreads();
      publish_wait(sm, t, h, b, rank, C, bars, phase, pb, dead);
      b ^= 1;
    }
}

// Coarse right-hand side of the CTA's own coarse rows: the area-weighted
// restriction of the defect f - L e (Sec. 3.1), with the expression of the
// other restriction kernels.  out: the coarse row block (swizzled) or, with
// swz = 0, a plain [s_c][n_r] array.
__device__ void t_restrict(const LevelDev& L, const LevelDev& Cl, unsigned char* sm,
                           const TailLevel& tf, const TailLevel& tc, int h, int b, int rank,
                           float s2, V* out, bool swz) {
  const int nr = L.nr, nt = L.nt, NR = nr + 2, NT = nt + 2, ncr = Cl.nr;
  const float* rt = L.rf;
  const float* tt = L.tf;
  const int j0 = rank * tf.s, j0c = rank * tc.s;
  const int n = tc.s * ncr;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int R = idx / ncr, I = idx - R * ncr;
    float ax = 0.f, ay = 0.f;
    for (int bb = 0; bb < 2; ++bb)
      for (int a = 0; a < 2; ++a) {
        const int i = 2 * I + a, rr = 2 * R + bb, j = j0 + rr;
        const V* er = erow(sm, tf, h, b, rr);
        const int sw = tsw(nr, j);
        const V c = er[i ^ sw];
        const V E = (i + 1 < nr) ? er[(i + 1) ^ sw] : vz();
        const V W = (i > 0) ? er[(i - 1) ^ sw] : vz();
        const V N = (j + 1 < nt) ? erow(sm, tf, h, b, rr + 1)[i ^ tsw(nr, j + 1)] : vz();
        const V S = (j > 0) ? erow(sm, tf, h, b, rr - 1)[i ^ tsw(nr, j - 1)] : vz();
        const float aE = rt[RT_AE * NR + i + 1], aW = rt[RT_AW * NR + i + 1], P = rt[RT_P * NR + i + 1];
        const float aN = P * tt[TT_AN * NT + j + 1], aS = P * tt[TT_AS * NT + j + 1];
        const float d = rt[RT_DR * NR + i + 1] + P * tt[TT_DT * NT + j + 1] -
                        s2 * rt[RT_Q * NR + i + 1] * tt[TT_T * NT + j + 1];
        const V fv = rowp(sm, tf.fo, nr, h, rr)[i ^ sw];
        const float rx = fv.x - (aE * E.x + aW * W.x + aN * N.x + aS * S.x + d * c.x);
        const float ry = fv.y - (aE * E.y + aW * W.y + aN * N.y + aS * S.y + d * c.y);
        const float wgt = rt[RT_RW * NR + i + 1] * tt[TT_RW * NT + j + 1];
        ax += wgt * rx;
        ay += wgt * ry;
      }
    out[R * ncr + (swz ? (I ^ tsw(ncr, j0c + R)) : I)] = make_float2(ax, ay);
  }
}

// Coarse-grid value at 1-based coarse indices (I, J) with the ghost rules of
// the coarse level (zero next to a Dirichlet side, (-1)^m times the
// neighbour across a pole or the axis, the neighbour itself across a
// Neumann face or the origin).
__device__ __forceinline__ V t_cval(const LevelDev& Cl, unsigned char* sm, const TailLevel& tc,
                                    int h, int bc, int j0c, int I, int J, int m) {
  float fac = 1.f;
  const float sgn = (m & 1) ? -1.f : 1.f;
  int Ic = I, Jc = J;
  if (I == 0) { if (Cl.gL == GH_ZERO) return vz(); Ic = 1; if (Cl.gL == GH_PARITY) fac *= sgn; }
  if (I == Cl.nr + 1) { if (Cl.gR == GH_ZERO) return vz(); Ic = Cl.nr; if (Cl.gR == GH_PARITY) fac *= sgn; }
  if (J == 0) { if (Cl.gB == GH_ZERO) return vz(); Jc = 1; if (Cl.gB == GH_PARITY) fac *= sgn; }
  if (J == Cl.nt + 1) { if (Cl.gT == GH_ZERO) return vz(); Jc = Cl.nt; if (Cl.gT == GH_PARITY) fac *= sgn; }
  const V v = erow(sm, tc, h, bc, Jc - 1 - j0c)[(Ic - 1) ^ tsw(Cl.nr, Jc - 1)];
  return make_float2(fac * v.x, fac * v.y);
}

// e += P e_coarse on the fine rows [rlo, rhi) of block b (own rows and halo
// rows, clipped to the plane), bilinear in (r^2, theta) / (R, z) (Sec. 3.1).
__device__ void t_prolong(const LevelDev& L, const LevelDev& Cl, unsigned char* sm,
                          const TailLevel& tf, const TailLevel& tc, int h, int bf, int bc,
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
    const V a = t_cval(Cl, sm, tc, h, bc, j0c, I1, J1, m);
    const V bv = t_cval(Cl, sm, tc, h, bc, j0c, I1 + 1, J1, m);
    const V c = t_cval(Cl, sm, tc, h, bc, j0c, I1, J1 + 1, m);
    const V d = t_cval(Cl, sm, tc, h, bc, j0c, I1 + 1, J1 + 1, m);
    V* e = erow(sm, tf, h, bf, r) + (i ^ tsw(nr, j));
    V u = *e;
    u.x += p1 * q1 * a.x + p2 * q1 * bv.x + p1 * q2 * c.x + p2 * q2 * d.x;
    u.y += p1 * q1 * a.y + p2 * q1 * bv.y + p1 * q2 * c.y + p2 * q2 * d.y;
    *e = u;
  }
}

// Exact FP64 solve of the coarsest level (separable form L_m = L_r (x) I +
// D_r (x) L_t, L_t = V diag(lambda) V^-1): the CTA of rank c transforms and
// Thomas-solves its own eigenvalues k, every CTA receives all of z, and each
// back-transforms its own rows and the coarse halo rows its prolongation
// reads.  G: the gathered coarse right-hand side [nt][nr] (all rows).
__device__ void t_coarsest(cg::cluster_group& cl, const TailArgs& a, const LevelDev& Lc,
                           unsigned char* sm, const TailLevel& tc, int h, int rank, int slot) {
  const int nr = Lc.nr, nt = Lc.nt, nc = nr * nt, C = a.C, sc = tc.s, k0 = rank * sc;
  const V* G = reinterpret_cast<const V*>(sm + a.g_off);
  double2* Z = reinterpret_cast<double2*>(sm + a.z_off);    // [nt][nr], both components
  double2* zl = reinterpret_cast<double2*>(sm + a.zl_off);  // [sc][nr], own eigenvalues
  const double* Fq = a.sep + size_t(slot) * a.sep_stride;
  const int hh = nt / 2, vr = a.sep_sym ? hh : nt;
  const double* Vm = Fq;
  const double* Vi = Vm + vr * nt;
  const double* invd = Vi + nt * vr;
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
  // the Thomas sweeps of the own eigenvalues as the precomputed matrix
  // product x = A_k z (written into the own rows of Z): `parts` threads per
  // output share its dot product
  {
    const int nout = 2 * sc * nr;
    int parts = 1;
    while (parts < 32 && parts * 2 * nout <= int(blockDim.x)) parts *= 2;
    const int seg = (nr + parts - 1) / parts;
    for (int t = threadIdx.x; t < ((nout * parts + 31) / 32) * 32; t += blockDim.x) {
      const int o = t / parts, part = t - o * parts;
      double acc = 0.0;
      int kk = 0, c = 0, i = 0;
      if (o < nout) {
        c = o / (sc * nr);
        const int rq = o - c * sc * nr;
        kk = rq / nr;
        i = rq - kk * nr;
        const double* Ak = a.cinv + ((size_t(slot) * nt + k0 + kk) * nr + i) * nr;
        const double* zk = reinterpret_cast<const double*>(zl + kk * nr) + c;
        for (int mm = part * seg; mm < min(nr, (part + 1) * seg); ++mm) acc = fma(Ak[mm], zk[2 * mm], acc);
      }
      for (int off = parts >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (o < nout && part == 0) {
        double2* zo = Z + (k0 + kk) * nr + i;
        if (c) zo->y = acc;
        else zo->x = acc;
      }
    }
  }
  __syncthreads();
  // every other CTA receives the own rows of x
  {
    const int n = sc * nr;
    for (int tgt = 0; tgt < C; ++tgt) {
      if (tgt == rank) continue;
      double2* zt = cl.map_shared_rank(Z, tgt);
      for (int q = threadIdx.x; q < n; q += blockDim.x) zt[k0 * nr + q] = Z[k0 * nr + q];
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
    erow(sm, tc, h, 0, j - j0c)[i ^ tsw(nr, j)] = make_float2(ex, ey);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kTailThreads, 1)
    k_tail(TailArgs a, Batch B, RetireState S, const double2* __restrict__ fg, double2* __restrict__ ug) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ LevelDev sL[8];
  __shared__ D4 red[kTailThreads / 32];
  __shared__ __align__(8) unsigned long long hbar[8][2];   // per level and halo buffer
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
  // FP64 solution: the own rows stay in global memory (L2-resident, written
  // only by this CTA); the halo rows j0 - 1 and j0 + s0 are kept here and
  // updated with the same values their owners add, so no CTA reads a row
  // another CTA writes during the kernel
  const TailLevel& t0 = a.lv[0];
  const int nr0 = t0.L.nr, nt0 = t0.L.nt, s0 = t0.s, j00 = rank * s0, n0 = nr0 * nt0;
  const size_t base = size_t(p) * n0;
  double2* Uh = reinterpret_cast<double2*>(sm + a.u_off);   // [2][nr0]: rows -1 and s0
  double2* Uo = ug + base + size_t(j00) * nr0;               // own rows (global)
  for (int idx = threadIdx.x; idx < 2 * nr0; idx += blockDim.x) {
    const int side = idx / nr0, i = idx - side * nr0, j = side ? j00 + s0 : j00 - 1;
    Uh[idx] = (j >= 0 && j < nt0) ? ug[base + size_t(j) * nr0 + i] : make_double2(0.0, 0.0);
  }
  cp_async_wait_all();
  if (threadIdx.x < 2 * K) {
    mbar_init(smem_u32(&hbar[threadIdx.x >> 1][threadIdx.x & 1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // every CTA of the cluster has started, and its mbarriers are initialised,
  // before any writes into a peer's shared memory
  cl.sync();
  unsigned phase = 0;   // bit 2 l + b: parity of the next completion of hbar[l][b]
  bool dead = false;    // a neighbour wait gave up (reported as non-finite)
  int bl[8];   // per level: the row block the next step reads
#pragma unroll
  for (int l = 0; l < 8; ++l) bl[l] = 0;
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
    // (SqAcc, as in the level-wide residual kernel)
    SqAcc ax = sq_zero(), ay = sq_zero();
    {
      const LevelDev& L0 = sL[0];
      for (int idx = threadIdx.x; idx < s0 * nr0; idx += blockDim.x) {
        const int r = idx / nr0, i = idx - r * nr0, j = j00 + r;
        const double2* ur = Uo + r * nr0;
        const double2* un = r + 1 < s0 ? ur + nr0 : Uh + nr0;
        const double2* us = r > 0 ? ur - nr0 : Uh;
        const double2 c = ur[i];
        const double2 E = (i + 1 < nr0) ? ur[i + 1] : make_double2(0.0, 0.0);
        const double2 W = (i > 0) ? ur[i - 1] : make_double2(0.0, 0.0);
        const double2 N = (j + 1 < nt0) ? un[i] : make_double2(0.0, 0.0);
        const double2 Sv = (j > 0) ? us[i] : make_double2(0.0, 0.0);
        const size_t cq = size_t(j) * nr0 + i;
        const double aE = rd0[RT_AE * NR0 + i + 1], aW = rd0[RT_AW * NR0 + i + 1];
        const double aN = a.ctab[cq], aS = a.ctab[n0 + cq];
        const double d = fma(-s2d, a.ctab[3 * size_t(n0) + cq], a.ctab[2 * size_t(n0) + cq]);
        const double2 fv = fg[base + cq];
        double rx = fma(-aE, E.x, fv.x), ry = fma(-aE, E.y, fv.y);
        rx = fma(-aW, W.x, rx);
        ry = fma(-aW, W.y, ry);
        rx = fma(-aN, N.x, rx);
        ry = fma(-aN, N.y, ry);
        rx = fma(-aS, Sv.x, rx);
        ry = fma(-aS, Sv.y, ry);
        rx = fma(-d, c.x, rx);
        ry = fma(-d, c.y, ry);
        const V ro = make_float2(f64_to_f32(rx), f64_to_f32(ry));
        rowp(sm, t0.fo, nr0, h, r)[i ^ tsw(nr0, j)] = ro;
        const float dv = L0.rf[RT_V * NR0 + i + 1] * L0.tf[TT_V * NT0 + j + 1];
        sq_add(ax, ro.x, dv);
        sq_add(ay, ro.y, dv);
      }
    }
    ax = sq_warp_sum(ax);
    ay = sq_warp_sum(ay);
    SqPart* rq = reinterpret_cast<SqPart*>(red);   // the same 32 bytes per warp
    if ((threadIdx.x & 31) == 0) {
      SqPart q;
      q.s[0] = ax.s; q.s[1] = ay.s; q.s[2] = 0.f; q.s[3] = 0.f;
      q.e[0] = ax.e; q.e[1] = ay.e; q.e[2] = sq_zero().e; q.e[3] = sq_zero().e;
      rq[threadIdx.x >> 5] = q;
    }
    __syncthreads();
    if (threadIdx.x < C) {   // the CTA's partial (FP64) to every CTA of the cluster
      SqAcc sx = sq_zero(), sy = sq_zero();
      for (int w = 0; w < int(blockDim.x >> 5); ++w) {
        sx = sq_merge(sx, SqAcc{rq[w].s[0], rq[w].e[0]});
        sy = sq_merge(sy, SqAcc{rq[w].s[1], rq[w].e[1]});
      }
      const D4 tsum{sq_value(sx), sq_value(sy), dead ? 1.0 : 0.0, 0.0};
      *cl.map_shared_rank(part + rank, int(threadIdx.x)) = tsum;
    }
    __syncthreads();
    push_halo(cl, sm, rowp(sm, t0.fo, nr0, h, 0), t0.fo, 0, s0, nr0, h, rank, C);
    cl.sync();
    // App. B criterion, evaluated identically by every thread of the cluster
    double sx = 0.0, sy = 0.0, sdead = 0.0;
    for (int c = 0; c < C; ++c) { sx += part[c].x; sy += part[c].y; sdead += part[c].z; }
    int st = TS_ACTIVE;
    if (!isfinite(sx) || !isfinite(sy) || sdead != 0.0) st = TS_NONFINITE;
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
      {   // e = 0 on the own rows and the halo buffer the first step reads
        V* eo = reinterpret_cast<V*>(sm) + t.eo;
        V* eh = reinterpret_cast<V*>(sm) + t.eh[bl[l]];
        for (int k = threadIdx.x; k < t.s * L.nr; k += blockDim.x) eo[k] = vz();
        for (int k = threadIdx.x; k < 2 * h * L.nr; k += blockDim.x) eh[k] = vz();
      }
      __syncthreads();
      const unsigned bars[2] = {smem_u32(&hbar[l][0]), smem_u32(&hbar[l][1])};
      t_smooth(L, sm, t, h, bl[l], rank, C, s2, a.n_sor, t.nu1, bars, phase, 2 * l, dead);
      const TailLevel& tc = a.lv[l + 1];
      const LevelDev Lq = sL[l + 1];
      if (l + 1 < K - 1) {
        t_restrict(L, Lq, sm, t, tc, h, bl[l], rank, s2, rowp(sm, tc.fo, Lq.nr, h, 0), true);
        __syncthreads();
        push_halo(cl, sm, rowp(sm, tc.fo, Lq.nr, h, 0), tc.fo, 0, tc.s, Lq.nr, h, rank, C);
        cl.sync();   // the coarse level's first step reads the halo row s of f
      } else {
        V* G = reinterpret_cast<V*>(sm + a.g_off);
        V* own = G + rank * tc.s * Lq.nr;
        t_restrict(L, Lq, sm, t, tc, h, bl[l], rank, s2, own, false);
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
    t_coarsest(cl, a, sL[K - 1], sm, a.lv[K - 1], h, rank, slot);
    for (int l = K - 2; l >= 0; --l) {
      const TailLevel& t = a.lv[l];
      const LevelDev L = sL[l];
      t_prolong(L, sL[l + 1], sm, t, a.lv[l + 1], h, bl[l], bl[l + 1], rank, m);
      __syncthreads();
      const unsigned bars[2] = {smem_u32(&hbar[l][0]), smem_u32(&hbar[l][1])};
      t_smooth(L, sm, t, h, bl[l], rank, C, s2, a.n_sor, t.nu2, bars, phase, 2 * l, dead);
    }
    // u += e on the own rows and the two halo rows (the halo rows of e are
    // current, so every copy of a row gets the owner's values)
    for (int idx = threadIdx.x; idx < (s0 + 2) * nr0; idx += blockDim.x) {
      const int r = idx / nr0 - 1, i = idx - (idx / nr0) * nr0, j = j00 + r;
      if (j < 0 || j >= nt0) continue;
      const V v = erow(sm, t0, h, bl[0], r)[i ^ tsw(nr0, j)];
      double2* x = r < 0 ? Uh + i : (r >= s0 ? Uh + nr0 + i : Uo + r * nr0 + i);
      double2 y = *x;
      y.x += f32_to_f64(v.x);
      y.y += f32_to_f64(v.y);
      *x = y;
    }
    __syncthreads();
    ++it;
  }
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
