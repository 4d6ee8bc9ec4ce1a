// Fused-colour line smoothing for levels held in global memory (Sec. 3.2).
//
// One launch relaxes both zebra colours of one direction: it reads e_in and
// writes e_out (ping-pong), so the colour-0 lines a block needs are never
// overwritten by another block.  The first colour-1 neighbour that belongs to
// the next block is recomputed from e_in (one extra line or column per block),
// giving exactly the values the two-launch ordering produces.  A smoothing
// cycle is a radial pass e -> tmp followed by a polar pass tmp -> e.
//
// Tile shapes: a radial block owns Wmax = 8 or 4 lines (one warp per line),
// a polar block TWmax columns (8, 16 or 32; at most 160 KB of staged tile);
// both are options the autotuner may change.  Re-tiling: grids are sized for
// all planes with the widest tiles; when only a few planes are active the
// blocks are spread over them with narrower tiles (up to 4x more blocks per
// plane, at least two lines or columns per block so that a block's first
// line or column keeps colour 0), so a lone slow mode still uses many SMs.
#include <cstdio>

#include "lines.cuh"

namespace ps {

// Blocks per plane for the active count: base * mult, mult in {1, 2, 4},
// mult <= cap.
__device__ __forceinline__ int spread(int base, int nact, int cap) {
  const int G = int(gridDim.x * gridDim.y);
  int mult = 1;
  while (mult < 4 && mult < cap && nact * base * mult * 2 <= G) mult *= 2;
  return mult;
}


// Radial pass, both colours: a block of 32 Wmax threads owns W lines
// [j0, j0+W), W = Wmax / mult.
// Every line it reads is first staged in shared memory with asynchronous
// copies (all loads in flight at once): e lines j0-1 .. j0+W+1 (zero beyond
// the plane, or all zero for a zero initial guess) and f lines j0 .. j0+W.
template <typename T>
__device__ __forceinline__ void stage_lines(vec2_t<T>* dst, const vec2_t<T>* plane, int j_first,
                                            int nlines, int nr, int nt, bool zero) {
  typedef vec2_t<T> V;
  constexpr int per = 16 / int(sizeof(V));   // complex values per 16-byte chunk
  const int chunks = nr / per;                // nr is a multiple of 2
  for (RowWalk w(threadIdx.x, blockDim.x, chunks); w.j < nlines; w.next()) {
    const int q = w.j, c = w.c, j = j_first + q;
    const bool valid = !zero && j >= 0 && j < nt;
    const V* src = plane + (valid ? size_t(j) * nr + c * per : 0);
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst + size_t(q) * nr + c * per));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 16 : 0) : "memory");
  }
}

template <typename T, int CPL>
__global__ void __launch_bounds__(256) k_rpass2(LevelDev L, Batch B, const vec2_t<T>* __restrict__ ein,
                                                vec2_t<T>* __restrict__ eout,
                                                const vec2_t<T>* __restrict__ f, int zero_init,
                                                int n_sor, int Wmax) {
  typedef vec2_t<T> V;
  extern __shared__ __align__(16) unsigned char sraw[];
  const int nact = *B.nact;
  const int mult = spread(int(gridDim.x), nact, Wmax / 2);
  const int per = int(gridDim.x) * mult;
  const int b = int(blockIdx.y * gridDim.x + blockIdx.x);
  const int k = b / per;
  if (k >= nact) return;
  const int W = Wmax / mult;
  const int j0 = (b - k * per) * W;
  const int p = B.act[k];
  const int slot = B.slot ? B.slot[p] : p;
  const int nr = L.nr, nt = L.nt;
  V* se = reinterpret_cast<V*>(sraw);   // e lines j0-1 .. j0+W+1 (line j at se + (j - j0 + 1) nr)
  V* sf = se + size_t(W + 3) * nr;       // f lines j0 .. j0+W
  V* s0 = sf + size_t(W + 1) * nr;       // relaxed colour-0 lines j0, j0+2, .., j0+W
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t base = size_t(p) * nr * nt;
  stage_lines<T>(se, ein + base, j0 - 1, W + 3, nr, nt, zero_init != 0);
  stage_lines<T>(sf, f + base, j0, W + 1, nr, nt, false);
  cp_async_wait_all();
  __syncthreads();
  const T* rt = rt_<T>(L);
  const T* tt = tt_<T>(L);
  const T s2 = s2_<T>(B, slot);
  const T* om = omr_<T>(L) + size_t(slot) * nt;
  auto eline = [&](int j) { return se + size_t(j - j0 + 1) * nr; };
  if (warp <= W / 2) {            // colour 0: lines j0, j0+2, .., j0+W
    const int j = j0 + 2 * warp;
    if (j < nt) {
      V ev[CPL], g[CPL], un[CPL], us[CPL];
      ld_line<V, CPL>(ev, eline(j), lane, nr);
      ld_line<V, CPL>(un, eline(j + 1), lane, nr);
      ld_line<V, CPL>(us, eline(j - 1), lane, nr);
      ld_line<V, CPL>(g, sf + size_t(j - j0) * nr, lane, nr);
      relax_r<T, CPL>(L, rt, tt, s2, om[j], j, g, un, us, n_sor, ev);
      st_line<V, CPL>(s0 + warp * nr, ev, lane, nr);
    }
  }
  __syncthreads();
  if (warp < W / 2) {             // colour 1: lines j0+1, .., j0+W-1
    const int j = j0 + 1 + 2 * warp;
    if (j < nt) {
      V ev[CPL], g[CPL], un[CPL], us[CPL];
      ld_line<V, CPL>(ev, eline(j), lane, nr);
      ld_line<V, CPL>(g, sf + size_t(j - j0) * nr, lane, nr);
      ld_line<V, CPL>(us, s0 + warp * nr, lane, nr);
      if (j + 1 < nt) {
        ld_line<V, CPL>(un, s0 + (warp + 1) * nr, lane, nr);
      } else {
#pragma unroll
        for (int c = 0; c < CPL; ++c) un[c] = z2<V>();
      }
      relax_r<T, CPL>(L, rt, tt, s2, om[j], j, g, un, us, n_sor, ev);
      st_line<V, CPL>(eout + base + size_t(j) * nr, ev, lane, nr);
    }
  } else if (warp < W) {          // store the block's colour-0 lines
    const int q = warp - W / 2, j = j0 + 2 * q;
    if (j < nt) {
      V ev[CPL];
      ld_line<V, CPL>(ev, s0 + q * nr, lane, nr);
      st_line<V, CPL>(eout + base + size_t(j) * nr, ev, lane, nr);
    }
  }
}

// Polar pass, both colours: a block owns TW columns [i0, i0+TW), TW =
// TWmax / mult; shared memory holds columns i0-1 .. i0+TW+1 of e_in and f.
// Tile layout: cell (j, cc) at j * SW + (cc ^ x(j)) with the odd stride
// SW = TW + 5 and x(j) = bit 4 of j under the pair lane mapping (else 0), so
// the 16 rows a half-warp reads fall on 16 distinct 8-byte bank slots.
__device__ __forceinline__ int tile_sw(int tw) { return tw + 5; }
template <int CPL>
__device__ __forceinline__ int tslot(int j, int cc, int SW) {
  return j * SW + (CPL == 1 ? cc : (cc ^ ((j >> 4) & 1)));
}

// u != nullptr: the last pass of a V-cycle adds its result to the FP64
// solution (u += e, the refinement's update) instead of storing e.
template <typename T, int CPL>
__global__ void __launch_bounds__(256) k_tpass2(LevelDev L, Batch B, const vec2_t<T>* __restrict__ ein,
                                                vec2_t<T>* __restrict__ eout,
                                                const vec2_t<T>* __restrict__ f, int n_sor, int TWmax,
                                                double2* __restrict__ u) {
  typedef vec2_t<T> V;
  extern __shared__ __align__(16) unsigned char sraw[];
  const int nact = *B.nact;
  const int mult = spread(int(gridDim.x), nact, TWmax / 2);
  const int per = int(gridDim.x) * mult;
  const int b = int(blockIdx.y * gridDim.x + blockIdx.x);
  const int kp = b / per;
  if (kp >= nact) return;
  const int TW = TWmax / mult;
  const int i0 = (b - kp * per) * TW;
  const int p = B.act[kp];
  const int slot = B.slot ? B.slot[p] : p;
  const int nr = L.nr, nt = L.nt;
  const int SW = tile_sw(TW), TC = TW + 3;
  V* se = reinterpret_cast<V*>(sraw);   // [nt][SW], column cc <-> i0 - 1 + cc
  V* sf = se + size_t(nt) * SW;          // same layout for f
  const size_t base = size_t(p) * nr * nt;
  for (RowWalk w(threadIdx.x, blockDim.x, TC); w.j < nt; w.next()) {
    const int j = w.j, cc = w.c, i = i0 - 1 + cc;
    const bool in = i >= 0 && i < nr;
    const int o = tslot<CPL>(j, cc, SW);
    const size_t g = base + size_t(j) * nr + (in ? i : 0);
    cp_async_v(se + o, ein + g, in);
    cp_async_v(sf + o, f + g, in);
  }
  cp_async_wait_all();
  __syncthreads();
  const T* rt = rt_<T>(L);
  const T* tt = tt_<T>(L);
  const T s2 = s2_<T>(B, slot);
  const T* om = omt_<T>(L) + size_t(slot) * nr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const bool on = CPL > 1 || lane < nt;
  for (int color = 0; color < 2; ++color) {
    const int ncol = color == 0 ? TW / 2 + 1 : TW / 2;   // colour 0 includes column i0+TW
    for (int k = warp; k < ncol; k += nw) {
      const int i = i0 + color + 2 * k;
      if (i >= nr) continue;
      const int cc = i - i0 + 1;
      V ev[CPL], g[CPL], ue[CPL], uw[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = lcell<CPL>(lane, c);
        ev[c] = g[c] = ue[c] = uw[c] = z2<V>();
        if (on) {
          ev[c] = se[tslot<CPL>(j, cc, SW)];
          uw[c] = se[tslot<CPL>(j, cc - 1, SW)];
          ue[c] = se[tslot<CPL>(j, cc + 1, SW)];
          g[c] = sf[tslot<CPL>(j, cc, SW)];
        }
      }
      relax_t<T, CPL>(L, rt, tt, s2, om[i], i, g, ue, uw, n_sor, ev);
      if (on) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) se[tslot<CPL>(lcell<CPL>(lane, c), cc, SW)] = ev[c];
      }
    }
    __syncthreads();
  }
  for (RowWalk w(threadIdx.x, blockDim.x, TW); w.j < nt; w.next()) {
    const V v = se[tslot<CPL>(w.j, w.c + 1, SW)];
    const size_t o = base + size_t(w.j) * nr + i0 + w.c;
    if (u) {
      double2 x = u[o];
      x.x += from_buf<T>(v.x);
      x.y += from_buf<T>(v.y);
      u[o] = x;
    } else {
      eout[o] = v;
    }
  }
}

// Polar tile width: the requested width (0: 32), at most n_r, halved until
// the staged tile (e and f, n_t x (TW + 5) each) fits in 160 KB.
static int tile_w(int nr, int nt, size_t vb, int want) {
  int tw = want > 0 ? want : 32;
  if (tw > nr) tw = nr;
  while (tw > 2 && size_t(nt) * 2 * (tw + 5) * vb > 160 * 1024) tw /= 2;
  return tw;
}

int smooth_tile_cols(int nr, int nt, size_t vb, int want) { return tile_w(nr, nt, vb, want); }

// Shared memory of a radial block of Wmax lines: e lines (W + 3), f lines
// (W + 1) and the relaxed colour-0 lines (W / 2 + 1).
static size_t rpass_smem(int nr, int Wmax, size_t vb) {
  return size_t(Wmax + 3 + Wmax + 1 + Wmax / 2 + 1) * nr * vb;
}
// The widest radial block (8, 4 or 2 lines, at most `want`) within 200 KB.
static int rpass_lines(int nr, size_t vb, int want) {
  int w = want >= 8 ? 8 : (want >= 4 ? 4 : 2);
  while (w > 2 && rpass_smem(nr, w, vb) > 200 * 1024) w /= 2;
  return w;
}

bool smooth_fits(int nr, int nt, size_t vb) {
  const int tw = tile_w(nr, nt, vb, 2);
  return rpass_smem(nr, 2, vb) <= 200 * 1024 && size_t(nt) * 2 * (tw + 5) * vb <= 200 * 1024;
}

template <typename T, int CPL>
static void rpass2(const LevelDev& L, const Batch& B, const vec2_t<T>* ein, vec2_t<T>* eout,
                   const vec2_t<T>* f, bool zi, int n_sor, int Wmax, cudaStream_t st) {
  const size_t sm = rpass_smem(L.nr, Wmax, sizeof(vec2_t<T>));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rpass2<T, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  dim3 grid((L.nt + Wmax - 1) / Wmax, B.max_planes);
  k_rpass2<T, CPL><<<grid, 32 * Wmax, sm, st>>>(L, B, ein, eout, f, zi ? 1 : 0, n_sor, Wmax);
}

template <typename T, int CPL>
static void tpass2(const LevelDev& L, const Batch& B, const vec2_t<T>* ein, vec2_t<T>* eout,
                   const vec2_t<T>* f, int n_sor, int cols, double2* u, cudaStream_t st) {
  const int TW = tile_w(L.nr, L.nt, sizeof(vec2_t<T>), cols);
  const size_t sm = size_t(L.nt) * 2 * (TW + 5) * sizeof(vec2_t<T>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tpass2<T, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  dim3 grid(L.nr / TW, B.max_planes);
  k_tpass2<T, CPL><<<grid, 256, sm, st>>>(L, B, ein, eout, f, n_sor, TW, u);
}

template <typename T>
static void rpass2_any(const LevelDev& L, const Batch& B, const vec2_t<T>* ein, vec2_t<T>* eout,
                       const vec2_t<T>* f, bool zi, int n_sor, int Wmax, cudaStream_t st) {
  switch (L.nr <= 32 ? 1 : L.nr / 32) {
    case 1: rpass2<T, 1>(L, B, ein, eout, f, zi, n_sor, Wmax, st); break;
    case 2: rpass2<T, 2>(L, B, ein, eout, f, zi, n_sor, Wmax, st); break;
    case 4: rpass2<T, 4>(L, B, ein, eout, f, zi, n_sor, Wmax, st); break;
    case 8: rpass2<T, 8>(L, B, ein, eout, f, zi, n_sor, Wmax, st); break;
    case 16: rpass2<T, 16>(L, B, ein, eout, f, zi, n_sor, Wmax, st); break;
    case 32: rpass2<T, 32>(L, B, ein, eout, f, zi, n_sor, Wmax, st); break;
    default: std::fprintf(stderr, "psolve: radial size %d unsupported\n", L.nr);
  }
}

template <typename T>
static void tpass2_any(const LevelDev& L, const Batch& B, const vec2_t<T>* ein, vec2_t<T>* eout,
                       const vec2_t<T>* f, int n_sor, int cols, double2* u, cudaStream_t st) {
  switch (L.nt <= 32 ? 1 : L.nt / 32) {
    case 1: tpass2<T, 1>(L, B, ein, eout, f, n_sor, cols, u, st); break;
    case 2: tpass2<T, 2>(L, B, ein, eout, f, n_sor, cols, u, st); break;
    case 4: tpass2<T, 4>(L, B, ein, eout, f, n_sor, cols, u, st); break;
    case 8: tpass2<T, 8>(L, B, ein, eout, f, n_sor, cols, u, st); break;
    case 16: tpass2<T, 16>(L, B, ein, eout, f, n_sor, cols, u, st); break;
    case 32: tpass2<T, 32>(L, B, ein, eout, f, n_sor, cols, u, st); break;
    default: std::fprintf(stderr, "psolve: polar size %d unsupported\n", L.nt);
  }
}

template <typename T>
void launch_smooth(const LevelDev& L, const Batch& B, vec2_t<T>* e, const vec2_t<T>* f,
                   vec2_t<T>* tmp, int cycles, int n_sor, bool zero_init, Tiles tiles,
                   cudaStream_t st, double2* u) {
  const int Wmax = rpass_lines(L.nr, sizeof(vec2_t<T>), tiles.lines_r == 4 ? 4 : 8);
  for (int c = 0; c < cycles; ++c) {
    rpass2_any<T>(L, B, e, tmp, f, zero_init && c == 0, n_sor, Wmax, st);
    tpass2_any<T>(L, B, tmp, e, f, n_sor, tiles.cols_t, c == cycles - 1 ? u : nullptr, st);
  }
}

template void launch_smooth<float>(const LevelDev&, const Batch&, float2*, const float2*, float2*,
                                   int, int, bool, Tiles, cudaStream_t, double2*);
template void launch_smooth<double>(const LevelDev&, const Batch&, double2*, const double2*,
                                    double2*, int, int, bool, Tiles, cudaStream_t, double2*);

}  // namespace ps
