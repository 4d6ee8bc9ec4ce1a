// Launch interface of the device kernels (all asynchronous on `st`).
#pragma once
#include <cuda_runtime.h>

#include "plan.h"

namespace ps {

template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };
template <typename T> using vec2_t = typename Vec2<T>::type;

// Device view of one multigrid level.
// Four FP64 partial sums (|r|^2 and |f|^2 of both components of a plane),
// 16-byte aligned like CUDA's vector types.
struct __align__(16) Sum4 {
  double x, y, z, w;
};
#ifdef __CUDACC__
// IEEE 754 conversions between binary64 and binary32 on the integer pipes:
// GB300 runs FP64 arithmetic at about 1/64 of its FP32 rate, the hardware
// conversions occupy that pipe, and the FP64 kernels of the refinement loop
// are bound by it.  Every case is formed from the bit fields (a hardware
// fallback for the rare cases would still be issued for every value when the
// compiler turns the branch into a select).
// binary64 -> binary32, round to nearest, ties to even.  Normal results: the
// sign, the rebiased exponent, the top 23 fraction bits, and one unit added
// when the 29 dropped bits exceed half a unit or equal it with an odd kept
// part (a carry into the exponent is the correct rounding, up to infinity).
// Subnormal results: the 53-bit significand shifted right by 30 - e bits
// (e the rebiased exponent), rounded the same way (a carry gives the smallest
// normal number).  Overflow gives infinity; NaN stays a quiet NaN.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hi = unsigned(b >> 32), lo = unsigned(b);
  const unsigned sign = hi & 0x80000000u;
  const int E = int((hi >> 20) & 0x7ffu), e = E - 1023 + 127;
  if (e > 0 && e < 255) {
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu, half = 0x10000000u;
    unsigned f = sign | (unsigned(e) << 23) | m;
    f += (rest > half || (rest == half && (m & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
  }
  const unsigned long long frac = b & 0xfffffffffffffull;
  if (E == 0x7ff) return __uint_as_float(frac ? (sign | 0x7fc00000u | unsigned(frac >> 29)) : (sign | 0x7f800000u));
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const int sh = 30 - e;
  if (sh > 53) return __uint_as_float(sign);   // below half the smallest subnormal (FP64 subnormals, zeros)
  const unsigned long long sig = frac | (1ull << 52);
  const unsigned long long m = sig >> sh, rest = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  const unsigned long long r = m + ((rest > half || (rest == half && (m & 1ull))) ? 1ull : 0ull);
  return __uint_as_float(sign | unsigned(r));
}
// binary32 -> binary64, exact: normal values rebias the exponent by
// 1023 - 127 and move the 23 fraction bits to the top of the 52; subnormals
// are normalised at their leading bit; zeros keep their sign; infinities and
// NaN (made quiet, payload kept) keep the all-ones exponent.
__device__ __forceinline__ double f32_to_f64(float x) {
  typedef unsigned long long u64;
  const unsigned b = __float_as_uint(x);
  const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  u64 d;
  if (e != 0u && e != 0xffu) {
    d = (u64(sign) << 32) | (u64(e + 896u) << 52) | (u64(m) << 29);
  } else if (e == 0xffu) {
    d = (u64(sign) << 32) | (0x7ffull << 52) | (m ? (1ull << 51) : 0ull) | (u64(m) << 29);
  } else if (m == 0u) {
    d = u64(sign) << 32;
  } else {
    const int p = 31 - __clz(int(m));   // m 2^-149 = 1.f 2^(p - 149)
    d = (u64(sign) << 32) | (u64(p - 149 + 1023) << 52) | ((u64(m) << (52 - p)) & 0xfffffffffffffull);
  }
  return __longlong_as_double(static_cast<long long>(d));
}

// Volume-weighted sums of squares in FP32 over the whole binary64 range.  A
// sum is an FP32 value s with an exponent e and stands for s 2^(2e): every
// value v is entered as v 2^-e, e being the largest exponent met so far
// (clamped to binary32's normal range for FP32 values, binary64's for FP64
// values), so the largest scaled value lies in [1, 2) and no square under-
// or overflows FP32 whatever the scale of the data (the weights are at most
// 1).  When a larger exponent arrives the sum so far is scaled down to it
// (a part below 2^-126 of the new scale is dropped, far below FP32's
// rounding).  Non-finite values give non-finite sums.  Only integer and
// FP32 instructions: the reduction of the FP64 residual kernel stays off
// the FP64 pipe.
struct SqAcc {
  float s;
  int e;
};
__device__ __forceinline__ float pow2f(int k) {   // 2^k for k in [-126, 127], 0 below
  return k < -126 ? 0.f : __uint_as_float(unsigned(k + 127) << 23);
}
__device__ __forceinline__ SqAcc sq_zero() { return SqAcc{0.f, -1022}; }
__device__ __forceinline__ void sq_add(SqAcc& a, float v, float w) {
  const int eb = int((__float_as_uint(v) >> 23) & 0xffu);
  const int ne = max(a.e, min(max(eb, 1), 253) - 127);
  a.s *= pow2f(2 * (a.e - ne));
  a.e = ne;
  const float x = v * pow2f(-ne);   // exact while the scaled value is normal
  a.s = __fmaf_rn(w * x, x, a.s);
}
__device__ __forceinline__ void sq_add(SqAcc& a, double v, float w) {
  const long long bits = __double_as_longlong(v);
  const int eb = int((bits >> 52) & 0x7ff);
  const int ne = max(a.e, min(max(eb, 1), 2046) - 1023);
  a.s *= pow2f(2 * (a.e - ne));
  a.e = ne;
  // v 2^-ne through the exponent field: inf and NaN kept, zero where the
  // scaled value (or v itself) is below binary64's normal range
  const int sb = eb - ne;
  const double y = eb == 2047 ? v
                 : (eb == 0 || sb < 1 ? 0.0 : __longlong_as_double(bits - static_cast<long long>(ne) * (1ll << 52)));
  const float x = f64_to_f32(y);
  a.s = __fmaf_rn(w * x, x, a.s);
}
__device__ __forceinline__ SqAcc sq_merge(SqAcc a, SqAcc c) {
  const int e = max(a.e, c.e);
  return SqAcc{__fmaf_rn(a.s, pow2f(2 * (a.e - e)), c.s * pow2f(2 * (c.e - e))), e};
}
// The sum over the warp's 32 lanes, complete in lane 0.
__device__ __forceinline__ SqAcc sq_warp_sum(SqAcc a) {
  const int e = __reduce_max_sync(0xffffffffu, a.e);
  float s = a.s * pow2f(2 * (a.e - e));
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return SqAcc{s, e};
}
// s 2^(2e) in FP64 through the exponent field: exact inside binary64's
// normal range, infinity above it, zero below it.
__device__ __forceinline__ double sq_value(SqAcc a) {
  const double d = f32_to_f64(a.s);
  if (a.s == 0.f || !isfinite(a.s)) return d;
  const long long bits = __double_as_longlong(d);
  const int eb = int((bits >> 52) & 0x7ff) + 2 * a.e;
  if (eb >= 2047) return __longlong_as_double(0x7ff0000000000000ll);
  if (eb < 1) return 0.0;
  return __longlong_as_double(bits + static_cast<long long>(2 * a.e) * (1ll << 52));
}
#endif

// One work item's four sums of squares as SqAcc pairs (s[c], e[c]).
struct __align__(16) SqPart {
  float s[4];
  int e[4];
};

#ifdef __CUDACC__
// An FP64 value in the buffer precision T, and back.
template <typename T>
__device__ __forceinline__ T to_buf(double x) {
  if constexpr (sizeof(T) == sizeof(float)) return f64_to_f32(x);
  else return x;
}
template <typename T>
__device__ __forceinline__ double from_buf(T x) {
  if constexpr (sizeof(T) == sizeof(float)) return f32_to_f64(x);
  else return x;
}
#endif

__host__ __device__ __forceinline__ Sum4 sum4(double x, double y, double z, double w) {
  return Sum4{x, y, z, w};
}

struct LevelDev {
  int nr, nt;
  const double* rd;   // RT_N x (nr+2) radial tables
  const double* td;   // TT_N x (nt+2) polar tables
  const float* rf;    // float copies
  const float* tf;
  const double* omr_d;  // [slots][nt]  r-line relaxation parameters
  const double* omt_d;  // [slots][nr]  polar-line relaxation parameters
  const float* omr_f;
  const float* omt_f;
  int gL, gR, gB, gT;   // coarse-ghost rules when this level is prolongated from
};

// A batch of planes: plane p of a level buffer starts at p * nr * nt; its
// mode slot is slot[p] (identity when slot == nullptr); the mode's
// [sin(m pi/N)/(pi/N)]^2 is s2[slot].  Only the planes act[0..*nact) are
// touched; grids are sized for max_planes and surplus blocks return.
struct Batch {
  const int* act;
  const int* nact;
  const int* slot;     // plane -> mode slot (nullptr: identity)
  const int* mode;     // slot -> azimuthal mode number m (pole / axis parity)
  const double* s2d;   // slot -> s_m^2
  const float* s2f;
  int max_planes;
};

// ---- FFT (k_fft.cu) --------------------------------------------------------
// f[m][j][i] (double2) = scale * sum_k rho[i][j][k] e^{-2 pi i m k / N}
void launch_fft_forward(const double* rho, double2* f, int nr, int nt, int N, double scale,
                        const double2* tw, cudaStream_t st);
void launch_fft_inverse(const double2* fh, double* phi, int nr, int nt, int N,
                        const double2* tw, cudaStream_t st);

// ---- multigrid (k_mg.cu), T = float or double ---------------------------------
// Tile shapes of the level-wide smoothing passes: radial lines per block
// (8 or 4) and polar columns per block (8, 16 or 32; 0 = the widest that
// fits).  They change only how lines are grouped into blocks: every tile
// shape gives bitwise the same result.
struct Tiles {
  int lines_r = 8;
  int cols_t = 0;
};
// Polar columns per block that the polar pass uses for a level of nr x nt
// cells of vb bytes each when `want` are requested (0: the widest).
int smooth_tile_cols(int nr, int nt, size_t vb, int want);
// Whether lines of nr (radial) and nt (polar) cells of vb-byte values fit the
// level-wide passes' shared-memory staging.
bool smooth_fits(int nr, int nt, size_t vb);
// `cycles` alternating-line smoothing cycles (k_smooth.cu); tmp is a
// scratch buffer of the level's size (ping-pong between the two passes).
// u: the last pass adds e to this FP64 solution (the refinement's update)
// and leaves e unwritten.
template <typename T>
void launch_smooth(const LevelDev& L, const Batch& B, vec2_t<T>* e, const vec2_t<T>* f,
                   vec2_t<T>* tmp, int cycles, int n_sor, bool zero_init, Tiles tiles,
                   cudaStream_t st, double2* u = nullptr);

// Lower part of a V-cycle in shared memory, one block per plane (k_vsmem.cu).
struct VSmemArgs {
  int nlev;              // levels first .. coarsest
  LevelDev L[8];
  int off_e[8], off_f[8];   // shared-memory offsets (complex elements)
  const double* inv;     // dense coarsest-level inverse [slots][nc][nc] (blk_n == 0)
  const double* blk;     // coarsest-level block factors [slots][blk_stride] (blk_n > 0)
  int nc;
  int blk_n, blk_nt;     // block size (= coarsest nr) and block count (= coarsest nt)
  int blk_smem;          // 1: this slot's factors are staged in shared memory at blk_off
  int dbl_off, blk_off;  // byte offsets in shared memory: FP64 solve scratch, staged factors
  const double* sep;     // separable coarsest-level factors [slots][sep_stride] (sep_stride > 0)
  int sep_stride;
  int sep_sym;           // mirror-symmetric separable layout (see Hierarchy::sep_sym)
  // FP32 V-cycle with a separable coarsest level, solved in FP32: sepf per
  // slot (sepf_stride floats) holds V^-1 transposed [vr][nt], V transposed
  // [nt][vr], then 1/pivot, upper/pivot and lower/pivot [nt][nr + 1] each
  // (padded rows), all rounded once from the FP64 factors.  blk_smem: staged at blk_off;
  // restage = 1: over the first level's right-hand side, which is copied in
  // again from the input after the coarsest solve.
  int f32c, restage;
  const float* sepf;
  int sepf_stride;
  int nu1, nu2, n_sor;
  int tab_off;           // shared-memory offset (complex elements) of the staged tables
  const void* tabs;      // per-slot packed tables (T), tab_stride elements per slot
  int tab_stride;
  size_t smem_bytes;
};
template <typename T>
void launch_vsmem(const VSmemArgs& a, const Batch& B, const vec2_t<T>* gf, vec2_t<T>* ge,
                  cudaStream_t st);
template <typename T>
void launch_restrict(const LevelDev& F, const LevelDev& C, const Batch& B,
                     const vec2_t<T>* e,
                     const vec2_t<T>* f,
                     vec2_t<T>* fc,
                     cudaStream_t st);
template <typename T>
void launch_prolong(const LevelDev& F, const LevelDev& C, const Batch& B,
                    vec2_t<T>* e,
                    const vec2_t<T>* ec,
                    cudaStream_t st);
// u += e over the planes of the batch (level-0 sizes)
template <typename T>
void launch_update(const LevelDev& L, const Batch& B, double2* u,
                   const vec2_t<T>* e,
                   cudaStream_t st);
// Convergence bookkeeping state (per plane) and the retirement parameters.
struct RetireState {
  double2* nf2;      // [planes] |f|^2 per component (set on iteration 0)
  double2* nr2;      // [planes] latest |r|^2
  int* cycles;       // [planes]
  int* status;       // [planes]
  int* iter;         // scalar
  int* cont;         // scalar: 1 while planes remain
  double* fmax2;     // scalar: max over planes of |f|^2 (iteration 0)
};
struct RetireArgs {
  RetireState S;
  double tol;
  int max_cycles, stagnation, use_cond;
  unsigned long long handle;   // graph conditional (use_cond)
  int* gcnt;                   // completion counter, zero between launches
  int zero_guess;              // u is zero on the first iteration: r = f there
  int tail_planes;             // hand over to the tail kernel once at most this many remain (0: never)
};

// r = f - L u (FP64), stored as T2, and the volume-weighted norms per plane
// (deterministic: each work item writes its FP32 partial sums (SqAcc) to
// part[p * nblk + b]; the last item of a plane to finish combines them in a
// fixed order and stores them as FP64 in psum[p]).  The last
// plane to finish then applies the App. B criterion to every active plane,
// counts cycles, sets the status, compacts the active list and sets the
// continue flag (and the graph conditional).
// ctab: the level's per-cell FP64 products [4][nt][nr] (P aN, P aS,
// DR + P DT, Q T), the same for every mode; dtab: the diagonal
// DR + P DT - s_m^2 Q T per mode slot [slots][nt][nr].
template <typename T>
void launch_residual(const LevelDev& L, const Batch& B, const double2* f, const double2* u,
                     vec2_t<T>* r, SqPart* part, Sum4* psum, int* cnt, const RetireArgs& ra,
                     cudaStream_t st, const double* ctab, const double* dtab);
int residual_blocks(int nr, int nt);

void launch_init_active(int* act, int* nact, int n, RetireState S, cudaStream_t st);

// ---- cluster-resident tail iterations (k_tail.cu) ------------------------------
// One level of the tail kernel's per-CTA layout: each CTA of a cluster owns
// `s` consecutive rows of the level (rows rank * s ..).  Its error lives in
// the own rows eo and two halo buffers eh[0], eh[1] (h rows above, then h
// rows below), used in turn by the smoothing steps; the right-hand side in
// one block fo of rows -h .. s + h - 1.  Offsets in complex FP32 elements.
struct TailLevel {
  LevelDev L;        // global tables, ghost rules
  int s;             // rows per CTA
  int eo, eh[2], fo;
  int tab;           // offset (floats) of this level's tables in a slot's packed block
  int nu1, nu2;      // smoothing cycles before / after the coarse correction
};
struct TailArgs {
  int nlev, C, h, n_sor;    // levels, CTAs per cluster, halo rows, SOR sweeps per line
  TailLevel lv[8];
  const float* tabs;        // per-slot packed FP32 tables of every level
  int tab_stride;           // floats per slot
  int tab_off, g_off, z_off, zl_off, u_off, part_off;   // shared-memory byte offsets
  size_t smem_bytes;
  const double* ctab;       // level-0 per-cell FP64 products [4][nt][nr]
  const double* sep;        // separable coarsest-level factors per slot
  int sep_stride, sep_sym;
  const double* cinv;       // per slot and eigenvalue k: the radial Thomas sweeps as a
                            // matrix [nt][nr][nr] (x = A_k z, z the scaled transform)
  double tol;
  int max_cycles, stagnation;
  int* titer;               // scratch: max iteration count over the clusters
  int* tdone;               // scratch: clusters finished
};
// Finishes the active planes B.act[0..*B.nact) (at most `clusters`) with one
// cluster of a.C CTAs per plane, iterating residual -> V-cycle -> update on
// chip until each plane meets the App. B criterion (FP32 V-cycles, FP64
// residual and update: the mixed path).
void launch_tail(const TailArgs& a, const Batch& B, const RetireState& S, const double2* f,
                 double2* u, int clusters, cudaStream_t st);
// Clusters of a.C CTAs with a.smem_bytes each that can be resident at once
// (0 when the configuration cannot launch).
int tail_max_clusters(const TailArgs& a);

// ---- boundary treatment (k_bc.cu) ---------------------------------------------
struct BDev {
  int nb;
  int ncell;            // domain cells next to at least one boundary ghost
  const int* adj;       // [nb] adjacent cell index (j-1)*nr + (i-1)
  const double* sig;    // [nb] screening coefficient (incl. 1/(4 pi G))
  const double* cpl;    // [nb] coefficient of the ghost value in L at adj
  const int* cell;      // [ncell] cell index
  const int* cbp;       // [2*ncell] boundary points touching the cell (-1 = none)
  int plane_cells;      // nr * nt
};
void launch_screening(const BDev& b, const double2* psi, double2* sigma, int M, cudaStream_t st);
void launch_boundary_potential(const double* gt, const double2* sigma, double2* theta, int M,
                               int nb, cudaStream_t st);
// nd densities of one geometry, planes p = b M + m: every mode's table is read
// once for up to eight densities
void launch_boundary_potential_multi(const double* gt, const double2* sigma, double2* theta, int M,
                                     int nb, int nd, cudaStream_t st);
// f2 = f - sum over the adjacent ghosts of cpl * (-theta), in place on f
void launch_rhs_ghosts(const BDev& b, double2* f, const double2* theta, int M, cudaStream_t st);

}  // namespace ps
