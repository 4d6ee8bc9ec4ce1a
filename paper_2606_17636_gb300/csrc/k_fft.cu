// Azimuthal transforms (Sec. 2.2): real rows of n_phi values along phi,
// two rows packed as one complex sequence per warp, a radix-2 Stockham FFT
// in shared memory, split into the two half spectra (m = 0..N/2), written
// transposed to the mode-major plane layout [m][j][i].  The inverse rebuilds
// the full Hermitian spectrum of two rows, transforms, and writes the real
// and imaginary outputs as the two rows.
#include <cstdio>

#include "kernels.h"

namespace ps {

// One complex FFT of length N (power of two) by one warp; data in x, scratch
// in y; returns the buffer that holds the result.  sign < 0: e^{-2 pi i},
// sign > 0: e^{+2 pi i} (conjugate twiddles).  tw[k] = e^{-2 pi i k / N}.
__device__ double2* warp_fft(double2* x, double2* y, int N, int logN, const double2* __restrict__ tw,
                             int sign) {
  const int lane = threadIdx.x & 31;
  const int half = N >> 1;
  for (int t = 0; t < logN; ++t) {
    const int s = 1 << t;            // stride of the current sub-sequences
    const int m = half >> t;         // half length of the current sub-sequences
    for (int b = lane; b < half; b += 32) {
      const int p = b >> t, q = b & (s - 1);
      const double2 a = x[q + s * p];
      const double2 c = x[q + s * (p + m)];
      const double2 d = make_double2(a.x - c.x, a.y - c.y);
      y[q + s * (2 * p)] = make_double2(a.x + c.x, a.y + c.y);
      // twiddle e^{-+2 pi i p s / N}: the factors 1 (p s = 0) and -+i
      // (p s = N/4) take no FP64 multiplies; the branch is uniform over a
      // warp's 32 consecutive butterflies once s >= 32 (the last stages)
      const int k = p * s;
      double2 t;
      if (k == 0) {
        t = d;
      } else if (k == (N >> 2)) {
        t = sign < 0 ? make_double2(d.y, -d.x) : make_double2(-d.y, d.x);
      } else {
        double2 w = tw[k];
        if (sign > 0) w.y = -w.y;
        t = make_double2(d.x * w.x - d.y * w.y, d.x * w.y + d.y * w.x);
      }
      y[q + s * (2 * p + 1)] = t;
    }
    __syncwarp();
    double2* z = x;
    x = y;
    y = z;
  }
  return x;
}

__global__ void k_fft_fwd(const double* __restrict__ rho, double2* __restrict__ out, int nr, int nt,
                          int N, int logN, double scale, const double2* __restrict__ tw, int rows) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.y;
  const int i0 = blockIdx.x * rows;
  const int M = N / 2 + 1;
  const int S = 2 * N + 4;          // per-warp region: x[N+2], y[N+2]
  double2* x = sm + size_t(warp) * S;
  double2* y = x + N + 2;
  const int ia = i0 + 2 * warp, ib = ia + 1;
  if (2 * warp < rows) {
    const double* ra = rho + (size_t(ia) * nt + j) * N;
    const double* rb = rho + (size_t(ib) * nt + j) * N;
    const bool okb = ib < nr;
    if (ia < nr)
      for (int k = lane; k < N; k += 32) x[k] = make_double2(ra[k], okb ? rb[k] : 0.0);
    __syncwarp();
    double2* z = warp_fft(x, y, N, logN, tw, -1);
    double2* o = (z == x) ? y : x;   // the free buffer (N+2 entries) takes both half spectra
    for (int mm = lane; mm < M; mm += 32) {
      const double2 zp = z[mm], zm = z[(N - mm) & (N - 1)];
      // X_a = (Z[m] + conj Z[N-m]) / 2,  X_b = (Z[m] - conj Z[N-m]) / (2i)
      o[mm] = make_double2(0.5 * scale * (zp.x + zm.x), 0.5 * scale * (zp.y - zm.y));
      o[M + mm] = make_double2(0.5 * scale * (zp.y + zm.y), -0.5 * scale * (zp.x - zm.x));
    }
  }
  __syncthreads();
  // transposed store: out[m][j][i0 + r]; every warp ran logN stages, so the
  // spectra sit in y when logN is even and in x otherwise
  const int R = rows < nr - i0 ? rows : nr - i0;
  const int off = (logN % 2 == 0) ? N + 2 : 0;
  for (int idx = threadIdx.x; idx < M * rows; idx += blockDim.x) {
    const int mm = idx / rows, r = idx - mm * rows;
    if (r >= R) continue;
    const double2* src = sm + size_t(r >> 1) * S + off + (r & 1) * M;
    out[(size_t(mm) * nt + j) * nr + i0 + r] = src[mm];
  }
}

__global__ void k_fft_inv(const double2* __restrict__ fh, double* __restrict__ phi, int nr, int nt,
                          int N, int logN, const double2* __restrict__ tw, int rows) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.y;
  const int i0 = blockIdx.x * rows;
  const int M = N / 2 + 1;
  const int R = rows < nr - i0 ? rows : nr - i0;
  const int S = 2 * N + 4;
  // stage the spectra of the block's rows: row r -> sm[(r>>1)*S + (r&1)*M + m]
  for (int idx = threadIdx.x; idx < M * rows; idx += blockDim.x) {
    const int mm = idx / rows, r = idx - mm * rows;
    double2 v = make_double2(0.0, 0.0);
    if (r < R) v = fh[(size_t(mm) * nt + j) * nr + i0 + r];
    if (mm == 0 || mm == N / 2) v.y = 0.0;   // only real parts of m = 0, N/2
    sm[size_t(r >> 1) * S + (r & 1) * M + mm] = v;
  }
  __syncthreads();
  if (2 * warp < rows) {
    double2* x = sm + size_t(warp) * S;
    double2* y = x + N + 2;
    // Z[m] = X_a[m] + i X_b[m] over m = 0..N-1, upper half by conjugation;
    // build it in registers first (x holds X_a, X_b), then write y.
    for (int mm = lane; mm < N; mm += 32) {
      double2 a, b;
      if (mm < M) { a = x[mm]; b = x[M + mm]; }
      else { a = x[N - mm]; b = x[M + N - mm]; a.y = -a.y; b.y = -b.y; }
      y[mm] = make_double2(a.x - b.y, a.y + b.x);
    }
    __syncwarp();
    double2* z = warp_fft(y, x, N, logN, tw, +1);
    const int ia = i0 + 2 * warp, ib = ia + 1;
    if (ia < nr) {
      double* pa = phi + (size_t(ia) * nt + j) * N;
      for (int k = lane; k < N; k += 32) pa[k] = z[k].x;
    }
    if (ib < nr) {
      double* pb = phi + (size_t(ib) * nt + j) * N;
      for (int k = lane; k < N; k += 32) pb[k] = z[k].y;
    }
  }
}

static int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

static int rows_for(int N) { return N <= 512 ? 16 : 8; }

void launch_fft_forward(const double* rho, double2* f, int nr, int nt, int N, double scale,
                        const double2* tw, cudaStream_t st) {
  const int rows = rows_for(N);
  const size_t sm = size_t(rows / 2) * (2 * N + 4) * sizeof(double2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fft_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  dim3 grid((nr + rows - 1) / rows, nt);
  k_fft_fwd<<<grid, 32 * (rows / 2), sm, st>>>(rho, f, nr, nt, N, ilog2(N), scale, tw, rows);
}

void launch_fft_inverse(const double2* fh, double* phi, int nr, int nt, int N, const double2* tw,
                        cudaStream_t st) {
  const int rows = rows_for(N);
  const size_t sm = size_t(rows / 2) * (2 * N + 4) * sizeof(double2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fft_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  dim3 grid((nr + rows - 1) / rows, nt);
  k_fft_inv<<<grid, 32 * (rows / 2), sm, st>>>(fh, phi, nr, nt, N, ilog2(N), tw, rows);
}

}  // namespace ps
