// Device-resident N-GMRES solve (one CUDA graph per precision phase); used
// synchronously by cp_solve and concurrently by the request server.
#pragma once

#include <chrono>

#include "cp_internal.cuh"
#include "linesearch.cuh"

namespace cpg {

// Control block written by the graph's control kernels.
struct SolveCtl {
  int iters, fg_evals, als_sweeps, restarts, ls_failures;
  int mixed_iters, fp64_iters;
  int ls_evals, accepts;
  int stop;          // 0 running, 1 tol met, 2 maxit, 3 mixed phase stalled, 4 non-finite
  int restart_now;   // this iteration restarted (the tail resets the window)
  int since_best;
  double gn, best, f;
};

// Kernels per graph stretch (captured once), to count replayed launches.
struct KernelCounts {
  unsigned long long top = 0, head = 0, restart = 0, ls_fixed = 0, ls_eval = 0, accept = 0, reject = 0;
};

struct SolverMem {
  double *u, *g, *ubar, *gbar, *uhat, *d, *x, *gx, *work, *M, *grams, *scal, *poly, *U, *G;
  // M^(1) of u, ubar and x (the next ALS sweep starts from u's), M^(N) of
  // the swept point and of ubar, and the line-search variant MTTKRPs of the
  // last mode
  double *M0, *M0bar, *M0x, *Ml, *Mlbar, *Mv;
  // the line search's Grams (ubar^T ubar, ubar^T d, d^T d per mode), from
  // which those of the accepted point follow
  double* Gls;
  float *u32, *ubar32, *d32;
  // Grams of u and ubar (N x R x R); inverses of Gammabar^(1) of u, ubar and
  // x with their ok flags (R*R + 2 doubles each)
  double *Gu, *Gbar, *Xi0, *Xi0bar, *Xi0x;
  int* win;
  MTState* st;
  SolveCtl* ctl;
};

// Streams, event, status word and pinned buffers of one solve; reusable by a
// server slot so that admitting a request allocates no host-pinned memory
// and creates no streams.
struct SolverRes {
  cudaStream_t stream = nullptr;
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};   // capture streams of nested bodies
  cudaEvent_t ev = nullptr;
  int* d_status = nullptr;
  unsigned* d_counter = nullptr;
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // one aux stream and event pair per nested capture level (a stream that
  // joined a capture stays in it until that capture ends)
  cudaStream_t aux_side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork_side[3] = {nullptr, nullptr, nullptr}, join_side[3] = {nullptr, nullptr, nullptr};
  double* h_pinned = nullptr;
  int* h_pinned_i = nullptr;
  SolveCtl* hctl = nullptr;
  cp_status create();
  void destroy();
};

struct Solver {
  cp_ctx sub;                       // device, the slot's stream, status word, pinned scratch, arena
  SolverRes own;                    // used when no slot resources are given
  SolverRes* res = nullptr;
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t done_ev = nullptr;
  cp_tensor* t = nullptr;
  cp_solve_opts o{};
  Layout L;
  int64_t P = 0;
  void* base = nullptr;
  void* arena = nullptr;
  SolverMem m{};
  SolveCtl* hctl = nullptr;         // pinned mirror, written at the end of each phase
  SolveCtl ctl_before{};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};   // [0] FP64, [1] mixed
  KernelCounts kcount, phase_counts[2];
  cp_precision cur = CP_FP64;
  bool polish_pending = false;
  int phase = 0;
  bool finished = false;
  bool converged = false;
  cp_status result = CP_OK;
  cp_solve_report rep{};
  std::chrono::steady_clock::time_point t0;

  ~Solver();
  void release();
  cp_status setup(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts& opts, SolverRes* r);
  cp_status capture_phase(cp_precision pr, bool first, cudaGraph_t* out);
  cp_status build_phase(cp_precision pr, bool first);
  cp_status launch_phase(cp_precision pr, bool first);
  void account_phase();
  cp_status start(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts& opts, const double* u0, bool on_device,
                  SolverRes* r = nullptr);
  bool poll(bool block);
  void rep_fill();
  cp_status copy_out(double* u_user, bool on_device);
};

}  // namespace cpg
