// The N-GMRES optimisation algorithm (Algorithm 1, Steps I-III of Section
// 2.1) with ALS as the one-step process M(.) (Section 2.3), windowed start-up
// and window size w (Section 2.1), the restart rule of Section 2.1 and the
// delta I regularisation with eps = 1e-12 (Section 2.4).
//
// The whole iteration runs on the device.  Each precision phase of a solve is
// ONE CUDA graph built from conditional nodes:
//
//   start   f, g at u (with u's Grams, M^(1) and Gammabar^(1) inverse);
//           window <- {(u, g(u))}; ||g||; set `outer`
//   WHILE outer:
//     head      Step I: the ALS sweep on u (its first mode from the carried
//               M^(1) and inverse), normalised into ubar (the sweep's last
//               MTTKRP and the Grams follow); f and g at ubar; Step II
//               (window dots, normal equations, uhat, normalised);
//               d = uhat - ubar, slope = g(ubar)^T d;
//               set `restart` = (slope >= 0)
//     IF restart:  u = ubar (with its f, g, M^(1), Grams and inverse)
//     ELSE:        Step III: the polynomial phi(beta) = f(ubar + beta d)
//                  from one MTTKRP launch (Khatri-Rao variants) and the
//                  Grams of ubar and d, the More-Thuente search on it;
//                  set `accept`
//                  IF accept: x = ubar + beta d; f, g at x from the
//                             variants; u = normalise(x)
//                  ELSE:      u = ubar
//     tail      push (u, g) to the window (reset it after a restart),
//               ||g||, counters, stopping test; set `outer`
//
// The host launches one graph per phase and reads a small control block at
// its end.  Workspace inside the graph comes from a bump arena (sized by a
// first, measuring capture), so every conditional body holds kernel nodes only.
//
// Mixed precision: the bf16x3 phase stops at ||g||/P < tol * mixed_tol_factor
// or after 50 iterations without a new best ||g||; then the FP64 phase (the
// polish) restarts the window from the FP64 gradient and runs to tol.
#include <chrono>
#include <cmath>
#include <functional>
#include <vector>

#include "cp_internal.cuh"
#include "linesearch.cuh"
#include "norm_dev.cuh"
#include "solver.cuh"

namespace cpg {

namespace {

enum { F = 0, FBAR = 1, SLOPE = 3, GD = 4, GG = 5, NSCAL = 8 };
enum { STOP_RUN = 0, STOP_TOL = 1, STOP_MAXIT = 2, STOP_STALL = 3, STOP_NONFINITE = 4 };

// Iterations of the mixed phase without a new smallest ||g|| before the FP64
// phase takes over (the safeguard for a tolerance below the mixed-precision
// noise floor).  On collinear problems N-GMRES's ||g|| plateaus for long
// stretches, and a handover that comes too early leaves most of the solve to
// the FP64 phase (a 174 x 164 x 48, R = 18, c = 0.9 request: 115 mixed + 1024
// FP64 iterations after a false stall at 50, against 325 mixed iterations).
// Over the first 128 requests of the serving stream, solved alone: 7.0 s in
// total at 50, 4.2 s at 200, 3.6 s at 400, 3.5 s at 800 (no false stall left).
constexpr int kMixedStallDefault = 800;

// Dense tensors with fewer entries solve in FP64 when mixed precision is
// asked for (cp_solve_opts.mixed_min_entries).
constexpr int64_t kMixedMinEntriesDefault = 4096;

// Stopping test on ||g||/P (shared by the phase start and the loop tail).
__device__ void ctl_eval(SolveCtl* c, const double* scal, double P, double tol, int maxit, int mixed,
                         int stall, cudaGraphConditionalHandle outer) {
  const double gn = sqrt(scal[GG]) / P;
  c->gn = gn;
  c->f = scal[F];
  int stop = STOP_RUN;
  if (!isfinite(gn))
    stop = STOP_NONFINITE;
  else if (gn < tol)
    stop = STOP_TOL;
  else if (c->iters >= maxit)
    stop = STOP_MAXIT;
  else if (mixed) {
    if (gn < c->best) {
      c->best = gn;
      c->since_best = 0;
    } else if (++c->since_best >= stall) {
      stop = STOP_STALL;
    }
  }
  c->stop = stop;
  cudaGraphSetConditional(outer, stop == STOP_RUN ? 1u : 0u);
}

// Up to eight copies in one launch (the branches that make ubar the iterate).
struct CopySeg {
  const double* src[8];
  double* dst[8];
  int64_t n[8];
  int nseg;
};

__global__ void copy_multi_kernel(const CopySeg c) {
  CP_PDL_ENTRY();
  for (int s = 0; s < c.nseg; ++s)
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < c.n[s]; k += (int64_t)gridDim.x * blockDim.x)
      c.dst[s][k] = c.src[s][k];
}

// Block sum of one value per thread (fixed order); thread 0 returns it.
__device__ double block_sum(double v, double* red8) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red8[w];
  return s;
}

__device__ bool is_last_block(unsigned* counter, bool* flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *flag = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (*flag) __threadfence();
  return *flag;
}

// Sum of the per-block partials, in block order, by warp 0 (result in lane 0).
__device__ double sum_blocks(const double* blk, int nb) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += __ldcg(&blk[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// After the N-GMRES combination (Section 2.1 Step II): normalise uhat with
// the scales from the combine pass's column sums (R6), d = uhat - ubar, the
// slope s = g(ubar)^T d, and the restart decision s >= 0 (R7).
__global__ void __launch_bounds__(256) uhat_finish_kernel(Layout L, const double* __restrict__ uhat,
                                                          const double* __restrict__ ubar,
                                                          const double* __restrict__ gbar,
                                                          const double* __restrict__ colsq, int S,
                                                          double* __restrict__ d, double* blk, unsigned* counter,
                                                          SolveCtl* c, double* scal, cudaGraphConditionalHandle restart,
                                                          int* status, float* __restrict__ d32, F32Off o32) {
  CP_PDL_ENTRY();
  __shared__ NormShared sh;
  __shared__ double red8[8];
  __shared__ bool is_last;
  norm_prologue(L, colsq, S, nullptr, nullptr, status, sh);
  const int R = L.R;
  const int64_t P = L.off[L.N];
  double part = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
    int n = 0;
    while (n + 1 < L.N && e >= L.off[n + 1]) ++n;
    const int64_t within = e - L.off[n];
    const int64_t i = within / R;
    const int p = (int)(within - i * R);
    const int q = sh.order[p];
    const double v = uhat[L.off[n] + i * R + q] * sh.scale[n * R + q];
    const double dv = v - ubar[e];
    d[e] = dv;
    if (d32) d32[o32.off[n] + i * o32.rs + p] = (float)dv;
    part = fma(gbar[e], dv, part);
  }
  const double bs = block_sum(part, red8);
  if (threadIdx.x == 0) blk[blockIdx.x] = bs;
  if (!is_last_block(counter, &is_last)) return;
  if (threadIdx.x < 32) {
    const double slope = sum_blocks(blk, gridDim.x);
    if (threadIdx.x == 0) {
      scal[SLOPE] = slope;
      c->als_sweeps += 1;
      c->fg_evals += 1;
      const bool r = !(slope < 0.0);
      c->restart_now = r ? 1 : 0;
      if (r) c->restarts += 1;
      cudaGraphSetConditional(restart, r ? 1u : 0u);
      *counter = 0u;
    }
  }
}

// End of an iteration (or start of a phase): push (u, g) into the window ring
// (reset to {(u, g)} at a phase start or after a restart), ||g||^2, and the
// stopping test that sets the WHILE condition.
__global__ void __launch_bounds__(256) tail_kernel(const double* __restrict__ u, const double* __restrict__ g,
                                                   double* __restrict__ U, double* __restrict__ G, int* win, int cap,
                                                   int64_t P, SolveCtl* c, double* scal, double Pd, double tol,
                                                   int maxit, int mixed, int stall,
                                                   cudaGraphConditionalHandle outer, double* blk, unsigned* counter,
                                                   int begin) {
  CP_PDL_ENTRY();
  __shared__ double red8[8];
  __shared__ bool is_last;
  const int reset = begin ? 1 : c->restart_now;
  const int start = win[0], m = win[1];
  const int slot = reset ? 0 : (m < cap ? (start + m) % cap : start);
  double part = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const double gk = g[k];
    U[(int64_t)slot * P + k] = u[k];
    G[(int64_t)slot * P + k] = gk;
    part = fma(gk, gk, part);
  }
  const double bs = block_sum(part, red8);
  if (threadIdx.x == 0) blk[blockIdx.x] = bs;
  if (!is_last_block(counter, &is_last)) return;
  if (threadIdx.x < 32) {
    const double gg = sum_blocks(blk, gridDim.x);
    if (threadIdx.x == 0) {
      scal[GG] = gg;
      if (reset) {
        win[0] = 0;
        win[1] = 1;
      } else if (win[1] < cap) {
        win[1] += 1;
      } else {
        win[0] = (win[0] + 1) % cap;
      }
      if (begin) {
        c->best = INFINITY;
        c->since_best = 0;
        c->fg_evals += 1;
      } else {
        c->iters += 1;
        if (mixed)
          c->mixed_iters += 1;
        else
          c->fp64_iters += 1;
      }
      c->restart_now = 0;
      ctl_eval(c, scal, Pd, tol, maxit, mixed, stall, outer);
      *counter = 0u;
    }
  }
}

int64_t grid_for(cp_ctx* ctx, int64_t n) {
  const int64_t b = std::min<int64_t>((n + 255) / 256, 8 * (int64_t)ctx->num_sms);
  return std::max<int64_t>(b, 1);
}

cp_status dcopy_multi(cp_ctx* ctx, const CopySeg& c) {
  int64_t nmax = 1;
  for (int s = 0; s < c.nseg; ++s) nmax = std::max(nmax, c.n[s]);
  (void)launch_pdl(copy_multi_kernel, dim3((unsigned)grid_for(ctx, nmax)), dim3(256), 0, ctx->stream, c);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

// Append a conditional node after the capture frontier of `s`; body i is
// captured on stream `bs` by fill(i).  The graph that owns the node is the
// one `s` is capturing into.
cp_status add_conditional(cudaStream_t s, cudaStream_t bs, cudaGraphConditionalHandle h,
                          cudaGraphConditionalNodeType type, unsigned size,
                          const std::function<cp_status(int)>& fill) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CP_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps));
  cudaGraphNodeParams prm{};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = size;
  cudaGraphNode_t node;
  CP_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &prm));
  for (unsigned i = 0; i < size; ++i) {
    CP_CUDA(cudaStreamBeginCaptureToGraph(bs, prm.conditional.phGraph_out[i], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed));
    const cp_status st = fill((int)i);
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(bs, &out);
    CP_TRY(st);
    CP_CUDA(e);
  }
  CP_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return CP_OK;
}

cp_status new_handle(cudaStream_t s, unsigned dflt, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  CP_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  CP_CUDA(cudaGraphConditionalHandleCreate(h, g, dflt, cudaGraphCondAssignDefault));
  return CP_OK;
}

}  // namespace

cp_status SolverRes::create() {
  CP_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
  for (auto& s : side) CP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  CP_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CP_CUDA(cudaMalloc(&d_status, sizeof(int)));
  CP_CUDA(cudaMemset(d_status, 0, sizeof(int)));
  CP_CUDA(cudaMalloc(&d_counter, 4 * sizeof(unsigned)));
  CP_CUDA(cudaMemset(d_counter, 0, 4 * sizeof(unsigned)));
  CP_CUDA(cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking));
  CP_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
  CP_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
  for (int i = 0; i < 3; ++i) {
    CP_CUDA(cudaStreamCreateWithFlags(&aux_side[i], cudaStreamNonBlocking));
    CP_CUDA(cudaEventCreateWithFlags(&fork_side[i], cudaEventDisableTiming));
    CP_CUDA(cudaEventCreateWithFlags(&join_side[i], cudaEventDisableTiming));
  }
  CP_CUDA(cudaMallocHost(&h_pinned, sizeof(double) * 64));
  CP_CUDA(cudaMallocHost(&h_pinned_i, sizeof(int) * 64));
  CP_CUDA(cudaMallocHost(&hctl, sizeof(SolveCtl)));
  return CP_OK;
}

void SolverRes::destroy() {
  if (stream) cudaStreamSynchronize(stream);
  for (auto& s : side)
    if (s) cudaStreamDestroy(s);
  if (stream) cudaStreamDestroy(stream);
  if (ev) cudaEventDestroy(ev);
  if (d_status) cudaFree(d_status);
  if (d_counter) cudaFree(d_counter);
  if (aux) cudaStreamDestroy(aux);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  for (int i = 0; i < 3; ++i) {
    if (aux_side[i]) cudaStreamDestroy(aux_side[i]);
    if (fork_side[i]) cudaEventDestroy(fork_side[i]);
    if (join_side[i]) cudaEventDestroy(join_side[i]);
  }
  if (h_pinned) cudaFreeHost(h_pinned);
  if (h_pinned_i) cudaFreeHost(h_pinned_i);
  if (hctl) cudaFreeHost(hctl);
  *this = SolverRes();
}

Solver::~Solver() { release(); }

// Frees in stream order on the solver's stream; no device-wide sync.
void Solver::release() {
  for (auto& e : exec)
    if (e) {
      cudaGraphExecDestroy(e);
      e = nullptr;
    }
  if (base && sub.stream) cudaFreeAsync(base, sub.stream);
  base = nullptr;
  if (arena && sub.stream) cudaFreeAsync(arena, sub.stream);
  arena = nullptr;
  if (res == &own) own.destroy();
  res = nullptr;
  sub.stream = nullptr;
}

cp_status Solver::setup(cp_ctx* ctx, const cp_tensor* t_in, const cp_solve_opts& opts, SolverRes* r) {
  t = const_cast<cp_tensor*>(t_in);
  o = opts;
  // small dense tensors: FP64 throughout (the bf16x3 noise in f costs more
  // iterations than the tensor cores save: a 9 x 8 x 7, R = 3 solve took 81
  // mixed iterations against 13 in FP64; every request of the serving stream,
  // from 58 176 entries up, was faster mixed)
  const int64_t min_entries = o.mixed_min_entries > 0 ? o.mixed_min_entries
                              : o.mixed_min_entries == 0 ? kMixedMinEntriesDefault : 0;
  if (o.prec != CP_FP64 && t->kind == 0 && t->K < min_entries) o.prec = CP_FP64;
  L.set(t->N, t->dims, o.R);
  P = L.P();
  if (r) {
    res = r;
  } else {
    res = &own;
    CP_TRY(own.create());
  }
  sub = cp_ctx();
  sub.device = ctx->device;
  sub.num_sms = ctx->num_sms;
  sub.stream = res->stream;
  for (int i = 0; i < 3; ++i) side[i] = res->side[i];
  done_ev = res->ev;
  sub.d_status = res->d_status;
  sub.d_counter = res->d_counter;
  sub.aux = res->aux;
  sub.ev_fork = res->ev_fork;
  sub.ev_join = res->ev_join;
  sub.h_pinned = res->h_pinned;
  sub.h_pinned_i = res->h_pinned_i;
  hctl = res->hctl;
  *hctl = SolveCtl{};
  CP_CUDA(cudaMemsetAsync(sub.d_status, 0, sizeof(int), sub.stream));
  int64_t Imax = 1;
  for (int n = 0; n < L.N; ++n) Imax = std::max(Imax, L.dims[n]);
  const size_t RR = (size_t)o.R * o.R;
  const int cap = o.w;
  const size_t n0 = (size_t)L.dims[0] * o.R;                                  // M^(1) of u, ubar, x
  const size_t nl = (size_t)L.dims[L.N - 1] * o.R;                           // M^(N) of the swept point, ubar
  int64_t acc32 = 0;
  (void)f32_layout(L, &acc32);
  // doubles per FP32 copy, a multiple of 128 bytes: the copies start 128-byte
  // aligned (the tensor-core kernel bulk-copies and vector-loads them)
  const size_t n32 = ((size_t)acc32 + 31) / 32 * 16;
  const size_t nmv = ((size_t)1 << (L.N - 1)) * (size_t)P;                   // line-search variants, every mode
  const size_t bytes = sizeof(double) * (9 * (size_t)P + 2 * (size_t)cap * P + (size_t)Imax * o.R +
                                         (size_t)L.N * RR + 16 + 40 + 3 * n0 + 2 * nl + nmv + 5 * (size_t)L.N * RR + 3 * n32 + 16 +
                                         3 * (RR + 2)) +
                       sizeof(MTState) + sizeof(SolveCtl) + 512;
  CP_CUDA(cudaMallocAsync(&base, bytes, sub.stream));
  double* p = (double*)base;
  m.u = p; p += P;
  m.g = p; p += P;
  m.ubar = p; p += P;
  m.gbar = p; p += P;
  m.uhat = p; p += P;
  m.d = p; p += P;
  m.x = p; p += P;
  m.gx = p; p += P;
  m.work = p; p += P;
  m.U = p; p += (size_t)cap * P;
  m.G = p; p += (size_t)cap * P;
  m.M = p; p += (size_t)Imax * o.R;
  m.grams = p; p += (size_t)L.N * RR;
  m.scal = p; p += 16;
  m.poly = p; p += 40;
  m.M0 = p; p += n0;
  m.M0bar = p; p += n0;
  m.M0x = p; p += n0;
  m.Ml = p; p += nl;
  m.Mlbar = p; p += nl;
  m.Gls = p; p += 3 * (size_t)L.N * RR;
  // padded FP32 copies of u, ubar and d for the tensor-core MTTKRPs (the
  // padding columns stay zero)
  p = (double*)(((uintptr_t)p + 127) & ~(uintptr_t)127);
  m.u32 = (float*)p; p += n32;
  m.ubar32 = (float*)p; p += n32;
  m.d32 = (float*)p; p += n32;
  m.Mv = p; p += nmv;
  m.Gu = p; p += (size_t)L.N * RR;
  m.Gbar = p; p += (size_t)L.N * RR;
  m.Xi0 = p; p += RR + 2;
  m.Xi0bar = p; p += RR + 2;
  m.Xi0x = p; p += RR + 2;
  m.win = (int*)p; p += 8;
  uintptr_t q = ((uintptr_t)p + 63) & ~(uintptr_t)63;
  m.st = (MTState*)q;
  q = (q + sizeof(MTState) + 63) & ~(uintptr_t)63;
  m.ctl = (SolveCtl*)q;
  CP_CUDA(cudaMemsetAsync(m.ctl, 0, sizeof(SolveCtl), sub.stream));
  CP_CUDA(cudaMemsetAsync(m.u32, 0, 3 * n32 * sizeof(double), sub.stream));
  if (o.prec != CP_FP64) CP_TRY(prepare_mixed(&sub, t));
  // dimension tree for the mixed phase of 3-way dense solves: on request, or
  // by default from 2^21 tensor entries up (256^3, R = 16: the pair of
  // MTTKRPs in 40 instead of 66 us, 316 against 326 us per iteration)
  sub.dimtree = o.prec == CP_MIXED_BF16X3 && t->kind == 0 && t->N == 3 &&
                (o.dimtree > 0 || (o.dimtree < 0 && t->K >= ((int64_t)1 << 21)));
  if (sub.dimtree) CP_TRY(prepare_dimtree(&sub, t));
  return CP_OK;
}

// Capture one phase graph on the solver's stream.  first: the phase starts
// from the user's (normalised) initial guess.
cp_status Solver::capture_phase(cp_precision pr, bool first, cudaGraph_t* out) {
  cp_ctx* ctx = &sub;
  cudaStream_t s0 = sub.stream;
  const bool mixed = pr != CP_FP64 && o.polish;
  // the tensor-core MTTKRPs read FP32 copies of u, ubar and d, kept beside them
  const bool want32 = pr == CP_MIXED_BF16X3 && t->kind == 0;
  int64_t acc32 = 0;
  const F32Off o32 = f32_layout(L, &acc32);
  const double tol = mixed ? o.tol * (o.mixed_tol_factor > 0 ? o.mixed_tol_factor : 1.0) : o.tol;
  const int maxit = o.maxit;
  const int stall = o.mixed_stall > 0 ? o.mixed_stall : kMixedStallDefault;
  const double Pd = (double)P;
  const int cap = o.w;
  cp_ls_opts lso = o.ls;
  if (pr != CP_FP64 && o.mixed_maxfev > 0 && o.mixed_maxfev < lso.maxfev) lso.maxfev = o.mixed_maxfev;
  unsigned long long k0 = g_launches.load();
  kcount = KernelCounts();
  auto with_stream = [&](cudaStream_t st, const std::function<cp_status()>& f) -> cp_status {
    const cp_ctx keep = *ctx;
    ctx->stream = st;
    for (int i = 0; i < 3; ++i)
      if (side[i] == st) {
        ctx->aux = res->aux_side[i];
        ctx->ev_fork = res->fork_side[i];
        ctx->ev_join = res->join_side[i];
      }
    const cp_status r = f();
    ctx->stream = keep.stream;
    ctx->aux = keep.aux;
    ctx->ev_fork = keep.ev_fork;
    ctx->ev_join = keep.ev_join;
    return r;
  };
  auto counted = [&](unsigned long long* slot, const std::function<cp_status()>& f) -> cp_status {
    const unsigned long long a = g_launches.load();
    const cp_status r = f();
    *slot += g_launches.load() - a;
    return r;
  };
  // ubar becomes the iterate: u, g, f, M^(1), Grams and Gammabar^(1) inverse follow
  CopySeg ubar_state{};
  ubar_state.nseg = 6;
  ubar_state.src[0] = m.ubar;
  ubar_state.dst[0] = m.u;
  ubar_state.n[0] = P;
  ubar_state.src[1] = m.gbar;
  ubar_state.dst[1] = m.g;
  ubar_state.n[1] = P;
  ubar_state.src[2] = m.scal + FBAR;
  ubar_state.dst[2] = m.scal + F;
  ubar_state.n[2] = 1;
  ubar_state.src[3] = m.M0bar;
  ubar_state.dst[3] = m.M0;
  ubar_state.n[3] = (int64_t)L.dims[0] * L.R;
  ubar_state.src[4] = m.Gbar;
  ubar_state.dst[4] = m.Gu;
  ubar_state.n[4] = (int64_t)L.N * L.R * L.R;
  ubar_state.src[5] = m.Xi0bar;
  ubar_state.dst[5] = m.Xi0;
  ubar_state.n[5] = (int64_t)L.R * L.R + 2;
  if (want32) {
    ubar_state.nseg = 7;
    ubar_state.src[6] = (const double*)m.ubar32;
    ubar_state.dst[6] = (double*)m.u32;
    ubar_state.n[6] = (acc32 + 1) / 2;
  }
  const unsigned vec_blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, 2 * (int64_t)sub.num_sms));
  auto tail = [&](cudaStream_t st, cudaGraphConditionalHandle h, int begin) -> cp_status {
    double* blk = nullptr;
    CP_TRY(ws_alloc(ctx, (void**)&blk, sizeof(double) * vec_blocks));
    (void)launch_pdl(tail_kernel, dim3(vec_blocks), dim3(256), 0, st, m.u, m.g, m.U, m.G, m.win, cap, P, m.ctl, m.scal, Pd, tol, maxit,
                                            mixed ? 1 : 0, stall, h, blk, ctx->d_counter, begin);
    CP_LAUNCH_CHECK();
    ws_free(ctx, blk);
    return CP_OK;
  };
  CP_CUDA(cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed));
  cp_status st = [&]() -> cp_status {
    cudaGraphConditionalHandle h_outer;
    CP_TRY(new_handle(s0, 0, &h_outer));
    CP_TRY(counted(&kcount.top, [&]() -> cp_status {
      if (first) CP_TRY(normalize_into(ctx, L, m.work, m.u, nullptr, nullptr, nullptr));
      if (want32) CP_TRY(f32_copy(ctx, L, m.u, o32, acc32, m.u32));
      CP_TRY(fg_eval_ex(ctx, t, L, m.u, nullptr, nullptr, nullptr, m.scal + F, m.g, pr, nullptr, m.Gu, m.M0,
                        nullptr, nullptr, m.Xi0, nullptr, want32 ? m.u32 : nullptr));
      // window <- {(u, g)}, ||g||^2, the stopping test
      return tail(s0, h_outer, 1);
    }));
    CP_TRY(add_conditional(s0, side[0], h_outer, cudaGraphCondTypeWhile, 1, [&](int) -> cp_status {
      return with_stream(side[0], [&]() -> cp_status {
        cudaGraphConditionalHandle h_restart;
        CP_TRY(new_handle(side[0], 0, &h_restart));
        CP_TRY(counted(&kcount.head, [&]() -> cp_status {
          // Step I on u in place (u itself is already in the window); u's
          // Grams, M^(1) and Gammabar^(1) inverse were carried over from the
          // point u was made from
          // (the sweep's last MTTKRP is M^(N) of the swept point: it follows
          // the normalisation and stands in for that mode's pass at ubar)
          CP_TRY(als_sweep_v2(ctx, t, L, m.u, pr, m.Gu, true, m.M0, m.Xi0, m.Ml, want32 ? m.u32 : nullptr));
          CP_TRY(normalize_into(ctx, L, m.u, m.ubar, nullptr, nullptr, nullptr, m.Gu, nullptr, nullptr, m.Gbar,
                                nullptr, nullptr, m.Ml, m.Mlbar, want32 ? m.ubar32 : nullptr));
          MGiven mg_bar;
          mg_bar.m[L.N - 1] = m.Mlbar;
          CP_TRY(fg_eval_ex(ctx, t, L, m.ubar, nullptr, nullptr, nullptr, m.scal + FBAR, m.gbar, pr, nullptr,
                            nullptr, m.M0bar, &mg_bar, m.Gbar, m.Xi0bar, nullptr, want32 ? m.ubar32 : nullptr));
          // Step II, then normalise uhat, d = uhat - ubar, slope, restart test
          double* colsq = nullptr;
          double* blk = nullptr;
          int S = 1;
          CP_TRY(ws_alloc(ctx, (void**)&colsq, sizeof(double) * (size_t)L.N * (2 * sub.num_sms + 2) * L.R));
          CP_TRY(ws_alloc(ctx, (void**)&blk, sizeof(double) * vec_blocks));
          CP_TRY(ngmres_core(ctx, P, m.win, cap, m.U, m.G, m.ubar, m.gbar, o.eps, m.work, nullptr, &L, colsq, &S));
          (void)launch_pdl(uhat_finish_kernel, dim3(vec_blocks), dim3(256), 0, side[0], L, m.work, m.ubar, m.gbar, colsq, S, m.d, blk,
                                                              ctx->d_counter, m.ctl, m.scal, h_restart,
                                                              ctx->d_status, want32 ? m.d32 : nullptr, o32);
          CP_LAUNCH_CHECK();
          ws_free(ctx, blk);
          ws_free(ctx, colsq);
          return CP_OK;
        }));
        CP_TRY(add_conditional(side[0], side[1], h_restart, cudaGraphCondTypeIf, 2, [&](int br) -> cp_status {
          return with_stream(side[1], [&]() -> cp_status {
            if (br == 0) {
              // restart: u = ubar (the tail resets the window to {(ubar, g(ubar))})
              return counted(&kcount.restart, [&]() -> cp_status { return dcopy_multi(ctx, ubar_state); });
            }
            // Step III: More-Thuente on the polynomial phi(beta) (one MTTKRP
            // pass), which also sets `accept`
            cudaGraphConditionalHandle h_acc;
            CP_TRY(new_handle(side[1], 0, &h_acc));
            bool ls_all = false;
            CP_TRY(counted(&kcount.ls_fixed, [&]() -> cp_status {
              return ls_poly(ctx, t, L, m.ubar, m.d, pr, lso, m.st, m.poly, m.ctl, h_acc, 1, m.Mv, &ls_all, m.Gls,
                             want32 ? m.ubar32 : nullptr, want32 ? m.d32 : nullptr);
            }));
            return add_conditional(side[1], side[2], h_acc, cudaGraphCondTypeIf, 2, [&](int ab) -> cp_status {
              return with_stream(side[2], [&]() -> cp_status {
                return counted(ab == 0 ? &kcount.accept : &kcount.reject, [&]() -> cp_status {
                  if (ab == 0) {
                    // x = ubar + beta d, f and g there (the last mode's M,
                    // or every mode's, from the line-search variants)
                    MGiven mg_x;
                    mg_x.nvar = 1 << (L.N - 1);
                    mg_x.beta = &m.st->stp_eval;
                    for (int n = ls_all ? 0 : L.N - 1; n < L.N; ++n) mg_x.m[n] = m.Mv + (size_t)mg_x.nvar * L.off[n];
                    // (f(x) goes straight to the iterate's f: nothing reads that in between)
                    CP_TRY(fg_eval_ex(ctx, t, L, m.ubar, m.d, &m.st->stp_eval, m.x, m.scal + F, m.gx, pr,
                                      nullptr, m.grams, m.M0x, &mg_x, nullptr, m.Xi0x, m.Gls));
                    return normalize_into(ctx, L, m.x, m.u, m.gx, m.g, nullptr, m.grams, m.M0x, m.M0, m.Gu,
                                          m.Xi0x, m.Xi0, nullptr, nullptr, want32 ? m.u32 : nullptr);
                  }
                  return dcopy_multi(ctx, ubar_state);
                });
              });
            });
          });
        }));
        // window push (or reset after a restart), ||g||^2, stopping test
        return counted(&kcount.head, [&]() { return tail(side[0], h_outer, 0); });
      });
    }));
    CP_CUDA(cudaMemcpyAsync(hctl, m.ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s0));
    return CP_OK;
  }();
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s0, &g);
  g_launches.fetch_sub(g_launches.load() - k0);   // captured, not launched
  if (st != CP_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  CP_CUDA(e);
  *out = g;
  return CP_OK;
}

cp_status Solver::build_phase(cp_precision pr, bool first) {
  const int slot = pr == CP_FP64 ? 0 : 1;
  if (exec[slot] && !first) return CP_OK;
  if (exec[slot]) {
    cudaGraphExecDestroy(exec[slot]);
    exec[slot] = nullptr;
  }
  // measuring capture: size of the workspace arena
  sub.arena_on = true;
  sub.arena_measure = true;
  sub.arena_off = 0;
  cudaGraph_t g = nullptr;
  cp_status st = capture_phase(pr, first, &g);
  if (g) cudaGraphDestroy(g);
  const size_t need = sub.arena_off + 4096;
  sub.arena_measure = false;
  if (st != CP_OK) {
    sub.arena_on = false;
    return st;
  }
  if (need > sub.arena_cap) {
    if (arena) cudaFreeAsync(arena, sub.stream);
    arena = nullptr;
    cudaError_t e = cudaMallocAsync(&arena, need, sub.stream);
    if (e != cudaSuccess) {
      sub.arena_on = false;
      return cuda_fail(e, "cudaMalloc(arena)", __FILE__, __LINE__);
    }
    sub.arena_base = (char*)arena;
    sub.arena_cap = need;
  }
  sub.arena_off = 0;
  g = nullptr;
  st = capture_phase(pr, first, &g);
  sub.arena_on = false;
  if (st != CP_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  const cudaError_t ei = cudaGraphInstantiate(&exec[slot], g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
  phase_counts[slot] = kcount;
  return CP_OK;
}

cp_status Solver::launch_phase(cp_precision pr, bool first) {
  CP_TRY(build_phase(pr, first));
  cur = pr;
  const int slot = pr == CP_FP64 ? 0 : 1;
  ctl_before = *hctl;   // counters before this phase (for the launch count)
  CP_CUDA(cudaGraphLaunch(exec[slot], sub.stream));
  CP_CUDA(cudaEventRecord(done_ev, sub.stream));
  return CP_OK;
}

void Solver::account_phase() {
  const KernelCounts& k = phase_counts[cur == CP_FP64 ? 0 : 1];
  const SolveCtl& a = ctl_before;
  const SolveCtl& b = *hctl;
  const unsigned long long iters = (unsigned long long)(b.iters - a.iters);
  const unsigned long long restarts = (unsigned long long)(b.restarts - a.restarts);
  const unsigned long long lsrch = iters - restarts;
  const unsigned long long evals = (unsigned long long)(b.ls_evals - a.ls_evals);
  const unsigned long long acc = (unsigned long long)(b.accepts - a.accepts);
  g_launches.fetch_add(k.top + iters * k.head + restarts * k.restart + lsrch * k.ls_fixed + evals * k.ls_eval +
                       acc * k.accept + (lsrch - acc) * k.reject);
}

cp_status Solver::start(cp_ctx* ctx, const cp_tensor* t_in, const cp_solve_opts& opts, const double* u0,
                        bool u0_on_device, SolverRes* r) {
  t0 = std::chrono::steady_clock::now();
  CP_TRY(setup(ctx, t_in, opts, r));
  CP_CUDA(cudaMemcpyAsync(m.work, u0, sizeof(double) * P,
                          u0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, sub.stream));
  polish_pending = (o.prec != CP_FP64) && o.polish;
  phase = 1;
  return launch_phase(o.prec, true);
}

// Non-blocking: advance when the running phase has finished.  Returns true
// when the solve is complete (result holds the status).
bool Solver::poll(bool block) {
  if (finished) return true;
  cudaError_t q = block ? cudaEventSynchronize(done_ev) : cudaEventQuery(done_ev);
  if (q == cudaErrorNotReady) return false;
  auto finish = [&](cp_status s) {
    result = s;
    finished = true;
    rep_fill();
    return true;
  };
  if (q != cudaSuccess) return finish(cuda_fail(q, "solve phase", __FILE__, __LINE__));
  account_phase();
  {
    const cp_status s = read_status(&sub);
    if (s != CP_OK) return finish(s);
  }
  const SolveCtl& c = *hctl;
  if (c.stop == STOP_NONFINITE) {
    set_error("cp_solve: non-finite gradient");
    return finish(CP_ERR_NONFINITE);
  }
  if (cur != CP_FP64 && polish_pending && (c.stop == STOP_TOL || c.stop == STOP_STALL)) {
    polish_pending = false;
    phase = 2;
    const cp_status s = launch_phase(CP_FP64, false);
    if (s != CP_OK) return finish(s);
    return false;
  }
  converged = c.stop == STOP_TOL;
  return finish(CP_OK);
}

void Solver::rep_fill() {
  const SolveCtl& c = *hctl;
  rep = cp_solve_report{};
  rep.iters = c.iters;
  rep.fg_evals = c.fg_evals;
  rep.als_sweeps = c.als_sweeps;
  rep.restarts = c.restarts;
  rep.ls_failures = c.ls_failures;
  rep.converged = converged ? 1 : 0;
  rep.mixed_iters = c.mixed_iters;
  rep.fp64_iters = c.fp64_iters;
  rep.f = c.f;
  rep.gnorm_over_P = c.gn;
  rep.normT2 = t ? t->norm2 : 0.0;
  rep.ls_trials = c.ls_evals;
  rep.t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

cp_status Solver::copy_out(double* u_user, bool on_device) {
  CP_CUDA(cudaMemcpyAsync(u_user, m.u, sizeof(double) * P, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          sub.stream));
  CP_CUDA(cudaStreamSynchronize(sub.stream));
  return CP_OK;
}

cp_status solve_impl(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts* o, double* u_user, bool user_on_device,
                     cp_solve_report* rep) {
  // order after the caller's earlier work on the context stream
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  Solver s;
  cp_status st = s.start(ctx, t, *o, u_user, user_on_device);
  if (st == CP_OK) {
    while (!s.poll(true)) {
    }
    st = s.result;
  }
  if (st == CP_OK) st = s.copy_out(u_user, user_on_device);
  if (s.finished || st != CP_OK) {
    s.rep_fill();
    if (rep) *rep = s.rep;
  }
  if (st == CP_OK && !s.converged) {
    set_error("cp_solve: tol not met after %d iterations (||g||/P = %.3e)", s.rep.iters, s.rep.gnorm_over_P);
    return CP_ERR_MAXIT;
  }
  return st;
}

}  // namespace cpg
