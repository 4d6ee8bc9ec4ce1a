// Batched multigrid solver: level upload, V-cycle schedule and the outer
// refinement loop with per-mode retirement (Sec. 3, App. B; Sec. 5.2's
// mode-by-mode iteration replaced by a batch that drops converged modes).
#include "solver.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

namespace ps {

void* Arena::get(size_t n) {
  if (n == 0) n = 16;
  n = (n + 255) & ~size_t(255);
  void* p = nullptr;
  if (alloc_fn) {
    p = alloc_fn(n, user);
    if (p && (reinterpret_cast<uintptr_t>(p) & 255)) {   // kernels rely on 256-byte alignment
      if (free_fn) free_fn(p, user);
      p = nullptr;
    }
  } else if (cudaMalloc(&p, n) != cudaSuccess) {
    p = nullptr;
  }
  if (p) {
    blocks.push_back(p);
    bytes += n;
  }
  return p;
}

void Arena::release_all() {
  for (void* p : blocks) {
    if (free_fn) free_fn(p, user);
    else cudaFree(p);
  }
  blocks.clear();
  bytes = 0;
}

template <typename X>
static X* upload(Arena& A, const std::vector<X>& v) {
  X* d = static_cast<X*>(A.get(v.size() * sizeof(X)));
  if (d && !v.empty()) cudaMemcpy(d, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice);
  return d;
}

// A coefficient table with one leading pad element: the returned pointer is
// one element past the (256-byte aligned) block start, so entry i + 1 of cell
// i puts every even cell at an even element offset (aligned pair loads).
template <typename X>
static X* upload_tab(Arena& A, const std::vector<X>& v) {
  std::vector<X> pad(v.size() + 1, X(0));
  std::copy(v.begin(), v.end(), pad.begin() + 1);
  X* d = upload(A, pad);
  return d ? d + 1 : nullptr;
}

static std::vector<float> to_f(const std::vector<double>& v) {
  return std::vector<float>(v.begin(), v.end());
}

// The FP32 copy of a level table with its volume row (len entries from
// row * len) scaled by a power of two that brings the largest entry into
// [1/2, 1).  The row only weights the squares of the convergence norms
// (App. B), whose test compares ratios of two such sums, so the scaling
// leaves every decision unchanged, and it keeps the weights (and the product
// of the radial and polar ones) inside FP32's range for grids in any length
// unit.
static std::vector<float> to_f_volume(const std::vector<double>& v, int row, int len) {
  std::vector<float> out = to_f(v);
  double mx = 0.0;
  for (int i = 0; i < len; ++i) mx = std::max(mx, std::fabs(v[size_t(row) * len + i]));
  if (mx > 0.0 && std::isfinite(mx)) {
    int e = 0;
    std::frexp(mx, &e);
    for (int i = 0; i < len; ++i)
      out[size_t(row) * len + i] = float(std::ldexp(v[size_t(row) * len + i], -e));
  }
  return out;
}

bool MGSolver::init(Arena& A, const PlaneGeo& fine, bool neumann, const std::vector<int>& modes,
                    const std::vector<int>& plane_slot, int mp, const MGOptions& o,
                    std::string& err) {
  opt = o;
  max_planes = mp;
  if (!plan_hierarchy(fine, neumann, modes, opt.coarsest_size, opt.precision, H, err)) return false;
  const int nl = int(H.lv.size());
  // line lengths the level-wide passes hold in registers and shared memory:
  // at most 1024 cells (FP32) or 512 (FP64), and a staged polar tile that
  // fits (smooth_fits)
  {
    const int lim = opt.precision ? 1024 : 512;
    const int nr0 = H.lv[0].g.r.n, nt0 = H.lv[0].g.t.n;
    if (nr0 > lim || nt0 > lim || !smooth_fits(nr0, nt0, opt.precision ? sizeof(float2) : sizeof(double2))) {
      err = "lines of " + std::to_string(nr0 > nt0 ? nr0 : nt0) + " cells exceed the " +
            (opt.precision ? "FP32" : "FP64") + " smoothing kernels (at most " + std::to_string(lim) + ")";
      return false;
    }
  }
  lv.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const LevelHost& h = H.lv[l];
    LevelDev& d = lv[l];
    d.nr = h.g.r.n;
    d.nt = h.g.t.n;
    d.rd = upload_tab(A, h.rtab);
    d.td = upload_tab(A, h.ttab);
    d.rf = upload_tab(A, to_f_volume(h.rtab, RT_V, d.nr + 2));
    d.tf = upload_tab(A, to_f_volume(h.ttab, TT_V, d.nt + 2));
    d.omr_d = upload(A, h.om_r);
    d.omt_d = upload(A, h.om_t);
    d.omr_f = upload(A, to_f(h.om_r));
    d.omt_f = upload(A, to_f(h.om_t));
    d.gL = h.gL; d.gR = h.gR; d.gB = h.gB; d.gT = h.gT;
    if (!d.rd || !d.omt_f) { err = "out of device memory"; return false; }
  }
  std::vector<double> s2(modes.size());
  for (size_t k = 0; k < modes.size(); ++k) s2[k] = fine.s2(modes[k]);
  d_s2 = upload(A, s2);
  d_s2f = upload(A, to_f(s2));
  d_mode = upload(A, modes);
  d_slot = plane_slot.empty() ? nullptr : upload(A, plane_slot);
  {   // level-0 per-cell products for the FP64 residual (mode independent)
    const LevelHost& h0 = H.lv[0];
    const int nr = lv[0].nr, nt = lv[0].nt, NR = nr + 2, NT = nt + 2;
    const size_t n = size_t(nr) * nt;
    std::vector<double> ct(4 * n);
    for (int j = 0; j < nt; ++j)
      for (int i = 0; i < nr; ++i) {
        const size_t q = size_t(j) * nr + i;
        const double P = h0.rtab[RT_P * NR + i + 1];
        ct[q] = P * h0.ttab[TT_AN * NT + j + 1];
        ct[n + q] = P * h0.ttab[TT_AS * NT + j + 1];
        ct[2 * n + q] = std::fma(P, h0.ttab[TT_DT * NT + j + 1], h0.rtab[RT_DR * NR + i + 1]);
        ct[3 * n + q] = h0.rtab[RT_Q * NR + i + 1] * h0.ttab[TT_T * NT + j + 1];
      }
    d_ctab = upload(A, ct);
    if (!d_ctab) { err = "out of device memory"; return false; }
    // the mode's diagonal per slot and cell, D_r + P D_theta - s_m^2 Q T:
    // the same correctly rounded fused multiply-add the residual would
    // otherwise repeat on every iteration
    std::vector<double> dm(s2.size() * n);
    for (size_t k = 0; k < s2.size(); ++k)
      for (size_t q = 0; q < n; ++q) dm[k * n + q] = std::fma(-s2[k], ct[3 * n + q], ct[2 * n + q]);
    d_dtab = upload(A, dm);
    if (!d_dtab) { err = "out of device memory"; return false; }
  }
  if (!H.coarse_inv.empty()) d_inv = upload(A, H.coarse_inv);
  if (!H.coarse_blk.empty()) d_blk = upload(A, H.coarse_blk);
  if (!H.coarse_sep.empty()) d_sep = upload(A, H.coarse_sep);
  const size_t vb = vbytes();
  e.assign(nl, nullptr);
  f.assign(nl, nullptr);
  for (int l = 0; l < nl; ++l) {
    const size_t n = size_t(mp) * lv[l].nr * lv[l].nt * vb;
    e[l] = A.get(n);
    f[l] = A.get(n);
    if (!e[l] || !f[l]) { err = "out of device memory"; return false; }
  }
  tmp = A.get(size_t(mp) * lv[0].nr * lv[0].nt * vb);
  if (!tmp) { err = "out of device memory"; return false; }
  // shared-memory V-cycle: the deepest levels whose error and right-hand
  // side fit next to the coarse-solve scratch (lines of at most 128 cells).
  // The mixed path solves a separable coarsest level in FP32 (scratch z,
  // 8 bytes per cell, rows padded by one cell); the FP64 path keeps f and z
  // in FP64, 32 bytes per cell.
  const bool f32c = opt.precision && H.sep_stride > 0;
  const size_t zf32 = 8 * size_t(lv[nl - 1].nt) * (lv[nl - 1].nr + 1);
  first = nl - 1;
  {
    const size_t zx_bytes = (f32c ? zf32 : 32 * size_t(H.nc)) + 16;
    const size_t budget = (f32c ? 224 : 210) * 1024;
    size_t bytes = zx_bytes;
    const size_t tb = vb / 2;   // bytes of one real table entry
    for (int l = nl - 1; l >= 0; --l) {
      bytes += 2 * size_t(lv[l].nr) * lv[l].nt * vb;
      bytes += (size_t(RT_N) * (lv[l].nr + 2) + size_t(TT_N) * (lv[l].nt + 2) + lv[l].nr + lv[l].nt + 2) * tb;
      if (bytes > budget || lv[l].nr > 128 || lv[l].nt > 128 || nl - l > 8) break;
      first = l;
    }
    vs.nlev = nl - first;
    size_t off = 0;
    for (int k = 0; k < vs.nlev; ++k) {
      const LevelDev& d = lv[first + k];
      vs.L[k] = d;
      vs.off_e[k] = int(off);
      off += size_t(d.nr) * d.nt;
      vs.off_f[k] = int(off);
      off += size_t(d.nr) * d.nt;
    }
    vs.tab_off = int(off);
    // per-slot packed copy of the fused levels' tables and this slot's omega
    // rows, laid out exactly as the kernel's shared-memory copy: per level,
    // at the next odd element offset, RT_N x (nr+2) radial and TT_N x (nt+2)
    // polar entries, then nt r-line and nr polar-line omegas
    size_t tab = 0;
    std::vector<size_t> lvl_off(vs.nlev);
    for (int k = 0; k < vs.nlev; ++k) {
      const LevelDev& d = lv[first + k];
      tab = (tab + 1) / 2 * 2 + 1;
      lvl_off[k] = tab;
      tab += size_t(RT_N) * (d.nr + 2) + size_t(TT_N) * (d.nt + 2) + d.nr + d.nt;
    }
    tab = (tab + 3) / 4 * 4;
    vs.tab_stride = int(tab);
    {
      const size_t S = modes.size();
      std::vector<double> pk(S * tab, 0.0);
      for (size_t q = 0; q < S; ++q)
        for (int k = 0; k < vs.nlev; ++k) {
          const LevelHost& h = H.lv[first + k];
          const int nr = lv[first + k].nr, nt = lv[first + k].nt;
          double* o = pk.data() + q * tab + lvl_off[k];
          std::copy(h.rtab.begin(), h.rtab.end(), o);
          o += size_t(RT_N) * (nr + 2);
          std::copy(h.ttab.begin(), h.ttab.end(), o);
          o += size_t(TT_N) * (nt + 2);
          std::copy(h.om_r.begin() + q * nt, h.om_r.begin() + (q + 1) * nt, o);
          o += nt;
          std::copy(h.om_t.begin() + q * nr, h.om_t.begin() + (q + 1) * nr, o);
        }
      if (opt.precision) vs.tabs = upload(A, to_f(pk));
      else vs.tabs = upload(A, pk);
      if (!vs.tabs) { err = "out of device memory"; return false; }
    }
    size_t sbytes = (off * vb + tab * (vb / 2) + 15) / 16 * 16;
    vs.dbl_off = int(sbytes);
    sbytes += f32c ? zf32 : 32 * size_t(H.nc);
    vs.inv = d_inv;
    vs.blk = d_blk;
    vs.nc = H.nc;
    vs.blk_n = H.blk_n;
    vs.blk_nt = H.blk_nt;
    vs.sep = d_sep;
    vs.sep_stride = H.sep_stride;
    vs.sep_sym = H.sep_sym;
    const size_t blk_bytes = H.sep_stride > 0
                                 ? size_t(H.sep_stride) * sizeof(double)
                                 : size_t(H.blk_nt) * H.blk_n * (H.blk_n + 2) * sizeof(double);
    vs.blk_smem = ((H.blk_n > 0 || H.sep_stride > 0) && sbytes + blk_bytes <= 220 * 1024) ? 1 : 0;
    vs.blk_off = int(sbytes);
    vs.f32c = f32c ? 1 : 0;
    vs.restage = 0;
    vs.sepf = nullptr;
    vs.sepf_stride = 0;
    if (f32c) {
      // the FP32 factor block per slot (see VSmemArgs::sepf), rounded once
      // from the FP64 factors; staged in its own space when it fits, else
      // over the first fused level's right-hand side (K >= 2: it is the
      // kernel's input, staged again from global memory after the coarsest
      // solve), else read from global memory
      const int nrc = lv[nl - 1].nr, ntc = lv[nl - 1].nt, vr = H.sep_sym ? ntc / 2 : ntc;
      const size_t ncc = size_t(nrc) * ntc;
      const size_t pc = size_t(ntc) * (nrc + 1);   // padded rows
      vs.sepf_stride = int((2 * size_t(vr) * ntc + 3 * pc + 3) / 4 * 4);
      const size_t S_ = modes.size();
      std::vector<float> pf(S_ * size_t(vs.sepf_stride), 0.f);
      for (size_t q = 0; q < S_; ++q) {
        const double* Vm = H.coarse_sep.data() + q * H.sep_stride;   // [vr][nt]
        const double* Vi = Vm + size_t(vr) * ntc;                     // [nt][vr]
        const double* rest = Vi + size_t(ntc) * vr;                   // 1/pivot, upper, lower
        float* o = pf.data() + q * vs.sepf_stride;
        for (int j = 0; j < vr; ++j)
          for (int k = 0; k < ntc; ++k) o[size_t(j) * ntc + k] = float(Vi[size_t(k) * vr + j]);
        o += size_t(vr) * ntc;
        for (int k = 0; k < ntc; ++k)
          for (int j = 0; j < vr; ++j) o[size_t(k) * vr + j] = float(Vm[size_t(j) * ntc + k]);
        o += size_t(ntc) * vr;
        for (int t = 0; t < 3; ++t)
          for (int k = 0; k < ntc; ++k)
            for (int i = 0; i < nrc; ++i) o[t * pc + size_t(k) * (nrc + 1) + i] = float(rest[t * ncc + size_t(k) * nrc + i]);
      }
      vs.sepf = upload(A, pf);
      if (!vs.sepf) { err = "out of device memory"; return false; }
      const size_t fac = 4 * size_t(vs.sepf_stride);
      const size_t f0 = size_t(vs.L[0].nr) * vs.L[0].nt * vb;
      if (sbytes + fac <= 224 * 1024) {
        vs.blk_smem = 1;
      } else if (vs.nlev >= 2 && fac <= f0) {
        vs.blk_smem = 1;
        vs.restage = 1;
        vs.blk_off = int(size_t(vs.off_f[0]) * vb);
      } else {
        vs.blk_smem = 0;
      }
      if (vs.blk_smem && !vs.restage) sbytes += fac;
    } else if (vs.blk_smem) {
      sbytes += blk_bytes;
    }
    vs.smem_bytes = sbytes + 16;
    if (H.nc < 16 || (H.nc & (H.nc - 1))) { err = "coarsest level must have a power-of-two size >= 16"; return false; }
    vs.nu1 = opt.nu1;
    vs.nu2 = opt.nu2;
    vs.n_sor = opt.n_sor;
  }
  const int nblk = residual_blocks(lv[0].nr, lv[0].nt);
  d_act = static_cast<int*>(A.get(sizeof(int) * mp));
  d_nact = static_cast<int*>(A.get(sizeof(int)));
  d_part = static_cast<SqPart*>(A.get(sizeof(SqPart) * size_t(mp) * nblk));
  d_psum = static_cast<Sum4*>(A.get(sizeof(Sum4) * mp));
  d_cnt = static_cast<int*>(A.get(sizeof(int) * mp));
  d_cycles = static_cast<int*>(A.get(sizeof(int) * mp));
  d_status = static_cast<int*>(A.get(sizeof(int) * mp));
  d_nf2 = static_cast<double2*>(A.get(sizeof(double2) * mp));
  d_nr2 = static_cast<double2*>(A.get(sizeof(double2) * mp));
  d_iter = static_cast<int*>(A.get(sizeof(int)));
  d_cont = static_cast<int*>(A.get(sizeof(int)));
  d_fmax2 = static_cast<double*>(A.get(sizeof(double)));
  d_gcnt = static_cast<int*>(A.get(sizeof(int)));
  if (!d_fmax2 || !d_cnt || !d_gcnt) { err = "out of device memory"; return false; }
  cudaMemset(d_cnt, 0, sizeof(int) * mp);
  cudaMemset(d_gcnt, 0, sizeof(int));
  if (cudaMallocHost(&h_cont, sizeof(int)) != cudaSuccess) { err = "pinned allocation failed"; return false; }
  batch.act = d_act;
  batch.nact = d_nact;
  batch.slot = d_slot;
  batch.mode = d_mode;
  batch.s2d = d_s2;
  batch.s2f = d_s2f;
  batch.max_planes = mp;
  S.nf2 = d_nf2;
  S.nr2 = d_nr2;
  S.cycles = d_cycles;
  S.status = d_status;
  S.iter = d_iter;
  S.cont = d_cont;
  S.fmax2 = d_fmax2;
  if (opt.precision) {
    // per-slot packed FP32 tables of every level for the cluster-resident
    // tail: per level, at the next odd element offset, RT_N x (nr+2) radial
    // and TT_N x (nt+2) polar entries, then nt r-line and nr polar-line
    // omegas of the slot
    std::vector<int> nrs(nl), nts(nl);
    for (int l = 0; l < nl; ++l) { nrs[l] = lv[l].nr; nts[l] = lv[l].nt; }
    const size_t tab = tail_tables(nrs, nts, tl);
    std::vector<size_t> off(nl);
    for (int l = 0; l < nl && l < 8; ++l) off[l] = size_t(tl.lv[l].tab);
    const size_t S_ = modes.size();
    std::vector<float> pk(S_ * tab, 0.f);
    for (size_t q = 0; q < S_; ++q)
      for (int l = 0; l < nl && l < 8; ++l) {
        const LevelHost& hl = H.lv[l];
        const int nr = lv[l].nr, nt = lv[l].nt;
        float* o = pk.data() + q * tab + off[l];
        // the FP32 level tables as uploaded (volume rows scaled alike), so
        // the tail's norms match the level-wide residual kernel's
        const std::vector<float> rt = to_f_volume(hl.rtab, RT_V, nr + 2);
        const std::vector<float> tt = to_f_volume(hl.ttab, TT_V, nt + 2);
        o = std::copy(rt.begin(), rt.end(), o);
        o = std::copy(tt.begin(), tt.end(), o);
        o = std::copy(hl.om_r.begin() + q * nt, hl.om_r.begin() + (q + 1) * nt, o);
        std::copy(hl.om_t.begin() + q * nr, hl.om_t.begin() + (q + 1) * nr, o);
      }
    d_tail_tabs = upload(A, pk);
    if (H.sep_stride > 0 && !H.large) {   // the tail kernel takes the small coarsest level only
      // per slot and eigenvalue k the two Thomas sweeps of the coarsest
      // radial systems applied to unit vectors: column m of A_k is the
      // sweeps' result for z = e_m (the tail applies them as one FP64
      // matrix product instead of a chain of dependent steps)
      const int nrc = lv[nl - 1].nr, ntc = lv[nl - 1].nt, vr = H.sep_sym ? ntc / 2 : ntc;
      std::vector<double> ci(S_ * size_t(ntc) * nrc * nrc);
      std::vector<double> zz(nrc);
      for (size_t q = 0; q < S_; ++q) {
        const double* Fq = H.coarse_sep.data() + q * H.sep_stride;
        const double* invd = Fq + size_t(vr) * ntc + size_t(ntc) * vr;
        const double* cp = invd + size_t(ntc) * nrc;
        const double* lid = cp + size_t(ntc) * nrc;
        for (int k = 0; k < ntc; ++k)
          for (int m = 0; m < nrc; ++m) {
            std::fill(zz.begin(), zz.end(), 0.0);
            zz[m] = 1.0;
            double dp = zz[0];
            for (int i = 1; i < nrc; ++i) { dp = std::fma(-lid[k * nrc + i], dp, zz[i]); zz[i] = dp; }
            double xv = dp;
            for (int i = nrc - 2; i >= 0; --i) { xv = std::fma(-cp[k * nrc + i], xv, zz[i]); zz[i] = xv; }
            double* Ak = ci.data() + ((q * ntc + k) * size_t(nrc)) * nrc;
            for (int i = 0; i < nrc; ++i) Ak[size_t(i) * nrc + m] = zz[i];
          }
      }
      tl.cinv = upload(A, ci);
      if (!tl.cinv) { err = "out of device memory"; return false; }
    }
    tl.titer = static_cast<int*>(A.get(2 * sizeof(int)));
    tl.tdone = tl.titer ? tl.titer + 1 : nullptr;
    if (!d_tail_tabs || !tl.titer) { err = "out of device memory"; return false; }
    cudaMemset(tl.titer, 0, 2 * sizeof(int));
    prepare_tail();
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { err = std::string("multigrid setup: ") + cudaGetErrorString(e); return false; }
  return true;
}

// ---- typed dispatch -----------------------------------------------------------
void MGSolver::smooth(int l, void* ee, const void* ff, int cycles, bool zi, cudaStream_t st,
                      double2* u) {
  if (opt.precision)
    launch_smooth<float>(lv[l], batch, (float2*)ee, (const float2*)ff, (float2*)tmp, cycles,
                         opt.n_sor, zi, opt.tiles, st, u);
  else
    launch_smooth<double>(lv[l], batch, (double2*)ee, (const double2*)ff, (double2*)tmp, cycles,
                          opt.n_sor, zi, opt.tiles, st, u);
}
void MGSolver::restrict_(int l, const void* ee, const void* ff, void* fc, cudaStream_t st) {
  if (opt.precision)
    launch_restrict<float>(lv[l], lv[l + 1], batch, (const float2*)ee, (const float2*)ff, (float2*)fc, st);
  else
    launch_restrict<double>(lv[l], lv[l + 1], batch, (const double2*)ee, (const double2*)ff, (double2*)fc, st);
}
void MGSolver::prolong(int l, void* ee, const void* ec, cudaStream_t st) {
  if (opt.precision)
    launch_prolong<float>(lv[l], lv[l + 1], batch, (float2*)ee, (const float2*)ec, st);
  else
    launch_prolong<double>(lv[l], lv[l + 1], batch, (double2*)ee, (const double2*)ec, st);
}
void MGSolver::fused(cudaStream_t st) {
  if (opt.precision)
    launch_vsmem<float>(vs, batch, (const float2*)f[first], (float2*)e[first], st);
  else
    launch_vsmem<double>(vs, batch, (const double2*)f[first], (double2*)e[first], st);
}
void MGSolver::residual(const double2* ff, const double2* u, double tol, cudaStream_t st,
                        int use_cond, unsigned long long cond) {
  RetireArgs ra;
  ra.S = S;
  ra.tol = tol;
  ra.max_cycles = opt.max_cycles;
  ra.stagnation = opt.stagnation;
  ra.use_cond = use_cond;
  ra.handle = cond;
  ra.gcnt = d_gcnt;
  ra.zero_guess = zero_guess;
  ra.tail_planes = tail_planes;
  if (opt.precision)
    launch_residual<float>(lv[0], batch, ff, u, (float2*)f[0], d_part, d_psum, d_cnt, ra, st, d_ctab, d_dtab);
  else
    launch_residual<double>(lv[0], batch, ff, u, (double2*)f[0], d_part, d_psum, d_cnt, ra, st, d_ctab, d_dtab);
}

void MGSolver::residual_to(const double2* ff, const double2* u, void* r, cudaStream_t st) {
  RetireArgs ra;
  ra.S = S;
  ra.tol = 0.0;
  ra.max_cycles = opt.max_cycles;
  ra.stagnation = opt.stagnation;
  ra.use_cond = 0;
  ra.handle = 0;
  ra.gcnt = d_gcnt;
  ra.zero_guess = 0;
  ra.tail_planes = 0;
  if (opt.precision)
    launch_residual<float>(lv[0], batch, ff, u, (float2*)r, d_part, d_psum, d_cnt, ra, st, d_ctab, d_dtab);
  else
    launch_residual<double>(lv[0], batch, ff, u, (double2*)r, d_part, d_psum, d_cnt, ra, st, d_ctab, d_dtab);
}

// One V-cycle on the error equation L e_0 = f_0 (f_0 = FP64 residual in the
// buffer precision), e_0 starting from zero (Sec. 3: pre-smoothing, defect
// restriction, coarse correction, prolongation, post-smoothing).  Levels
// below `first` run as level-wide kernels over all active planes; the rest
// runs in the shared-memory kernel, one block per plane.
// With post-smoothing on level 0, the update (with u) rides on its last pass.
bool MGSolver::vcycle(cudaStream_t st, double2* u) {
  for (int l = 0; l < first; ++l) {
    if (opt.nu1 > 0) smooth(l, e[l], f[l], opt.nu1, true, st);
    else cudaMemsetAsync(e[l], 0, size_t(max_planes) * lv[l].nr * lv[l].nt * vbytes(), st);
    restrict_(l, e[l], f[l], f[l + 1], st);
  }
  fused(st);
  bool updated = false;
  for (int l = first - 1; l >= 0; --l) {
    prolong(l, e[l], e[l + 1], st);
    if (opt.nu2 > 0) {
      double2* uu = l == 0 ? u : nullptr;
      smooth(l, e[l], f[l], opt.nu2, false, st, uu);
      updated = uu != nullptr;
    }
  }
  return updated;
}

void MGSolver::set_schedule(int nu1, int nu2, int n_sor, Tiles tiles, int nu1f, int nu2f) {
  opt.nu1 = nu1;
  opt.nu2 = nu2;
  opt.nu1f = nu1f;
  opt.nu2f = nu2f;
  vs.nu1 = nu1f > 0 ? nu1f : nu1;
  vs.nu2 = nu2f > 0 ? nu2f : nu2;
  opt.n_sor = vs.n_sor = n_sor;
  opt.tiles = tiles;
  prepare_tail();
}

// Layout of the cluster-resident tail for the current schedule.  Needs the
// mixed path, a separable coarsest level, a cluster size C (16, or the
// coarsest level's polar cell count when smaller) that divides every level
// into slabs of an even number of rows (one row or more on the coarsest
// level), radial lines of at most 256 cells, polar segments (own rows plus
// h = 2 n_sor halo rows each side) of at most 24 cells, and a shared-memory
// layout within the SM's 227 KB.
size_t tail_tables(const std::vector<int>& nr, const std::vector<int>& nt, TailArgs& t) {
  size_t tab = 0;
  for (size_t l = 0; l < nr.size() && l < 8; ++l) {
    tab = (tab + 1) / 2 * 2 + 1;   // odd offset: pairs of table entries are aligned vector loads
    t.lv[l].tab = int(tab);
    tab += size_t(RT_N) * (nr[l] + 2) + size_t(TT_N) * (nt[l] + 2) + nr[l] + nt[l];
  }
  tab = (tab + 3) / 4 * 4;
  t.tab_stride = int(tab);
  return tab;
}

size_t tail_layout(const std::vector<int>& nr, const std::vector<int>& nt, int n_sor, bool separable,
                   TailArgs& t) {
  const int nl = int(nr.size());
  if (!separable || nl < 2 || nl > 8) return 0;
  const int h = 2 * n_sor;
  const int ntc = nt[nl - 1], nrc = nr[nl - 1];
  int C = 16;
  while (C > ntc) C /= 2;
  if (C < 2 || ntc % C) return 0;
  t.nlev = nl;
  t.C = C;
  t.h = h;
  t.n_sor = n_sor;
  tail_tables(nr, nt, t);
  size_t off = 0;   // complex FP32 elements
  for (int l = 0; l < nl; ++l) {
    const int s = nt[l] / C;
    if (nt[l] % C || s < 1 || nr[l] > 256 || (nr[l] & 1)) return 0;
    if (l < nl - 1 && (s < 2 || (s & 1) || s + 2 * h > 24 || nr[l] < 16)) return 0;
    TailLevel& q = t.lv[l];
    const size_t halo = size_t(2 * h) * nr[l];
    q.s = s;
    q.eo = int(off); off += size_t(s) * nr[l];
    q.eh[0] = int(off); off += halo;
    if (l < nl - 1) {   // smoothed levels: a second halo buffer and the right-hand side
      q.eh[1] = int(off); off += halo;
      q.fo = int(off); off += size_t(s + 2 * h) * nr[l];
    } else {            // the coarsest level's right-hand side is gathered whole (g_off)
      q.eh[1] = q.eh[0];
      q.fo = q.eo;
    }
  }
  t.g_off = int(off * sizeof(float2));
  off += size_t(ntc) * nrc;
  size_t bytes = (off * sizeof(float2) + 15) / 16 * 16;
  t.z_off = int(bytes);
  bytes += size_t(ntc) * nrc * sizeof(double2);
  t.zl_off = int(bytes);
  bytes += size_t(ntc / C) * nrc * sizeof(double2);
  t.u_off = int(bytes);
  bytes += size_t(2) * nr[0] * sizeof(double2);   // the FP64 solution's two halo rows
  t.part_off = int(bytes);
  bytes += size_t(C) * 32;
  t.tab_off = int(bytes);
  bytes += size_t(t.tab_stride) * sizeof(float);
  bytes = (bytes + 15) / 16 * 16;
  t.smem_bytes = bytes;
  return bytes <= kTailSmemMax ? bytes : 0;
}

// Layout of the cluster-resident tail for the current schedule (see
// tail_layout): the mixed path only.
bool MGSolver::prepare_tail() {
  tail_planes = 0;
  if (!opt.precision || tail_cap == 0 || !d_tail_tabs) return false;
  const int nl = int(lv.size());
  std::vector<int> nr(nl), nt(nl);
  for (int l = 0; l < nl; ++l) { nr[l] = lv[l].nr; nt[l] = lv[l].nt; }
  TailArgs t = tl;
  if (!tail_layout(nr, nt, opt.n_sor, H.sep_stride > 0 && !H.large, t)) return false;
  for (int l = 0; l < nl; ++l) {
    TailLevel& q = t.lv[l];
    q.L = lv[l];
    const bool fused = l >= first;
    q.nu1 = fused ? vs.nu1 : opt.nu1;
    q.nu2 = fused ? vs.nu2 : opt.nu2;
  }
  t.ctab = d_ctab;
  t.sep = d_sep;
  t.sep_stride = H.sep_stride;
  t.sep_sym = H.sep_sym;
  t.tabs = d_tail_tabs;
  if (!t.cinv) return false;
  const int fit = tail_max_clusters(t);
  if (fit < 1) return false;
  tl = t;
  tail_planes = std::min(std::min(fit, 8), max_planes);
  if (tail_cap > 0) tail_planes = std::min(tail_planes, tail_cap);
  return true;
}

void MGSolver::tail(const double2* ff, double2* u, double tol, cudaStream_t st) {
  if (tail_planes <= 0) return;
  TailArgs t = tl;
  t.tol = tol;
  t.max_cycles = opt.max_cycles;
  t.stagnation = opt.stagnation;
  launch_tail(t, batch, S, ff, u, tail_planes, st);
}

void MGSolver::init_loop(cudaStream_t st) { launch_init_active(d_act, d_nact, max_planes, S, st); }

void MGSolver::loop_body(const double2* ff, double2* u, double tol, cudaStream_t st, int use_cond,
                         unsigned long long cond) {
  residual(ff, u, tol, st, use_cond, cond);
  if (vcycle(st, u)) return;
  if (opt.precision)
    launch_update<float>(lv[0], batch, u, (const float2*)e[0], st);
  else
    launch_update<double>(lv[0], batch, u, (const double2*)e[0], st);
}

int MGSolver::eager_solve(const double2* ff, double2* u, double tol, cudaStream_t st,
                          std::string& err) {
  init_loop(st);
  for (int it = 0; it <= opt.max_cycles + 1; ++it) {
    residual(ff, u, tol, st, 0, 0);
    cudaMemcpyAsync(h_cont, d_cont, sizeof(int), cudaMemcpyDeviceToHost, st);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t se = cudaStreamSynchronize(st);
    if (le != cudaSuccess || se != cudaSuccess) {
      err = std::string("multigrid iteration: ") + cudaGetErrorString(le != cudaSuccess ? le : se);
      return -2;
    }
    if (!*h_cont) return 0;
    if (!vcycle(st, u)) {
      if (opt.precision)
        launch_update<float>(lv[0], batch, u, (const float2*)e[0], st);
      else
        launch_update<double>(lv[0], batch, u, (const double2*)e[0], st);
    }
    if (*h_cont == 2) {   // at most tail_planes remain: the tail kernel finishes them
      tail(ff, u, tol, st);
      return 0;
    }
  }
  return 0;
}

}  // namespace ps
