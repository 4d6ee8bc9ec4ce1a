// Batched per-mode multigrid solver on the device (host-side orchestration).
#pragma once
#include <string>
#include <vector>

#include "kernels.h"

namespace ps {

// Device memory owner with optional user allocation hooks.
struct Arena {
  void* (*alloc_fn)(size_t, void*) = nullptr;
  void (*free_fn)(void*, void*) = nullptr;
  void* user = nullptr;
  std::vector<void*> blocks;
  size_t bytes = 0;
  void* get(size_t n);
  void release_all();
};

struct MGOptions {
  int precision = 1;   // 0 FP64, 1 mixed (FP32 V-cycles inside FP64 refinement)
  int nu1 = 2, nu2 = 2, n_sor = 2;
  int nu1f = 0, nu2f = 0;   // smoothing cycles of the fused (shared-memory) levels; 0: nu1 / nu2
  Tiles tiles;         // tile shapes of the level-wide smoothing passes
  int max_cycles = 100;
  int stagnation = 0;  // retire planes whose residual stops falling
  int coarsest_size = 1;   // coarsest-level rule (psolve_desc.coarsest_size; 1: small)
};

// Shared-memory layout of the cluster-resident tail (k_tail.cu) for levels of
// nr[l] x nt[l] cells and n_sor SOR sweeps: fills t's cluster size, rows per
// CTA, offsets and table layout; returns the bytes per CTA, or 0 when the
// plan does not allow the tail (a coarsest level without the separable form,
// cluster slabs that do not divide the levels, radial lines above 256 cells
// (or below 16 on a smoothed level),
// polar segments above 24 cells, or more than kTailSmemMax bytes).
constexpr size_t kTailSmemMax = 224 * 1024;
size_t tail_layout(const std::vector<int>& nr, const std::vector<int>& nt, int n_sor, bool separable,
                   TailArgs& t);
size_t tail_tables(const std::vector<int>& nr, const std::vector<int>& nt, TailArgs& t);

class MGSolver {
 public:
  // fine: plane geometry; modes[s]: azimuthal mode number of slot s;
  // plane_slot (size max_planes, may be empty = identity); neumann: inner
  // radial face carries a prescribed flux (zero coefficient on all levels).
  bool init(Arena& A, const PlaneGeo& fine, bool neumann, const std::vector<int>& modes,
            const std::vector<int>& plane_slot, int max_planes, const MGOptions& o,
            std::string& err);
  // Solve L u = f for all planes (u holds the initial guess).  Enqueued on
  // st; with cond_handle (use_cond) the loop is a graph WHILE body; in eager
  // mode the host reads the continue flag each iteration.
  void init_loop(cudaStream_t st);
  void loop_body(const double2* f, double2* u, double tol, cudaStream_t st, int use_cond,
                 unsigned long long cond);
  int eager_solve(const double2* f, double2* u, double tol, cudaStream_t st, std::string& err);
  // One V-cycle; with u, the refinement's update u += e rides on the last
  // smoothing pass when the schedule post-smooths level 0 with the
  // level-wide passes (returns true then; else the caller updates).
  bool vcycle(cudaStream_t st, double2* u = nullptr);
  // Change the smoothing schedule and tile shapes of later V-cycles (a
  // captured solve must be captured again).
  void set_schedule(int nu1, int nu2, int n_sor, Tiles tiles, int nu1f, int nu2f);
  // results (device arrays, per plane)
  int* d_cycles = nullptr;
  int* d_status = nullptr;
  double2* d_nf2 = nullptr;
  double2* d_nr2 = nullptr;
  int* d_iter = nullptr;
  int* d_cont = nullptr;
  int* h_cont = nullptr;   // pinned
  Hierarchy H;
  std::vector<LevelDev> lv;
  Batch batch{};
  MGOptions opt;
  int max_planes = 0;
  // level buffers (T2 of the precision): e[l], f[l]
  std::vector<void*> e, f;
  void* tmp = nullptr;             // ping-pong buffer of the global-memory smoother
  int first = 0;                   // first level handled by the shared-memory kernel
  int zero_guess = 0;              // the next solve starts from u = 0 (set by the caller)
  VSmemArgs vs{};
  // stage helpers on explicit buffers
  // u: the last pass adds e to u instead of storing it (see launch_smooth)
  void smooth(int level, void* e, const void* f, int cycles, bool zero_init, cudaStream_t st,
              double2* u = nullptr);
  void restrict_(int level, const void* e, const void* f, void* fc, cudaStream_t st);
  void prolong(int level, void* e, const void* ec, cudaStream_t st);
  void fused(cudaStream_t st);   // levels first .. coarsest in shared memory
  void residual(const double2* f, const double2* u, double tol, cudaStream_t st, int use_cond,
                unsigned long long cond);
  // the defect alone into r (tolerance 0: no plane retires)
  void residual_to(const double2* f, const double2* u, void* r, cudaStream_t st);
  int* d_act = nullptr;
  int* d_nact = nullptr;
  int* d_slot = nullptr;
  int* d_mode = nullptr;
  double* d_s2 = nullptr;
  float* d_s2f = nullptr;
  double* d_inv = nullptr;
  double* d_blk = nullptr;
  double* d_sep = nullptr;
  double* d_ctab = nullptr;   // level-0 per-cell FP64 products [4][nt][nr]
  double* d_dtab = nullptr;   // level-0 diagonal of each mode slot [slots][nt][nr]
  SqPart* d_part = nullptr;
  Sum4* d_psum = nullptr;
  int* d_cnt = nullptr;
  int* d_gcnt = nullptr;
  double* d_fmax2 = nullptr;
  RetireState S{};
  // cluster-resident tail (k_tail.cu): the last tail_planes active planes
  // (0: disabled) are finished by one launch, one cluster per plane
  TailArgs tl{};
  float* d_tail_tabs = nullptr;   // per-slot packed FP32 tables of every level
  int tail_planes = 0;
  int tail_cap = -1;              // -1: as many as can be resident; 0: off; n: at most n
  bool prepare_tail();            // layout for the current schedule; false when unsupported
  void tail(const double2* f, double2* u, double tol, cudaStream_t st);
  int precision_of_buffers = 1;
  size_t vbytes() const { return opt.precision ? sizeof(float2) : sizeof(double2); }
};

}  // namespace ps
