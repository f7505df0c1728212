// The N-GMRES optimisation algorithm (Algorithm 1, Steps I-III of Section
// 2.1) with ALS as the one-step process M(.) (Section 2.3), windowed start-up
// and window size w (Section 2.1), the restart rule of Section 2.1 and the
// delta I regularisation with eps = 1e-12 (Section 2.4).
//
// All state (iterates, gradients, the window ring and its indices, the line
// search) lives on the device.  Each stretch of work between two host
// decisions is captured once as a CUDA graph and replayed:
//   head     Step I (ALS sweep, normalise), f and g at ubar, Step II (window
//            dots, normal equations, uhat, normalise), d = uhat - ubar,
//            slope = g(ubar)^T d, line-search start
//   ls_eval  x = ubar + stp d, f and g at x, phi'(stp) = g(x)^T d, one
//            More-Thuente update
//   accept   u = normalise(x) with the gradient rescaled, push to the window
//   reject   u = ubar (line search without sufficient decrease), push
//   restart  u = ubar, window reset to {(ubar, g(ubar))}
// The host reads a few pinned scalars after each replay (the slope, the line
// search's done flag, ||g||) to choose the next graph.
//
// Mixed precision: iterations run with bf16x3 MTTKRPs until ||g||/P drops
// below tol * mixed_tol_factor (or stops improving for 50 iterations); then
// the window is reset and FP64 iterations continue until the FP64 gradient
// meets tol (the polish).
#include <chrono>
#include <cmath>
#include <functional>

#include "cp_internal.cuh"
#include "linesearch.cuh"

namespace cpg {

// One ALS sweep in place on u (grams must hold the Grams of u on entry and
// hold those of the result on exit); M is I_max x R scratch.
cp_status als_sweep_inplace(cp_ctx* ctx, const cp_tensor* t, const Layout& L, double* u,
                            double* grams, double* M, cp_precision prec) {
  for (int n = 0; n < L.N; ++n) {
    CP_TRY(mttkrp_any(ctx, t, L, u, n, M, prec));
    CP_TRY(als_mode_solve(ctx, L, u, n, M, grams));
  }
  return CP_OK;
}

namespace {

struct Graph {
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;
  ~Graph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

cp_status capture(cp_ctx* ctx, const std::function<cp_status()>& body, Graph& out) {
  const unsigned long long before = g_launches.load();
  cudaGraph_t graph = nullptr;
  CP_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  const cp_status st = body();
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
  const unsigned long long n = g_launches.load() - before;
  g_launches.fetch_sub(n);   // captured, not launched
  if (st != CP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  const cudaError_t ei = cudaGraphInstantiate(&out.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
  out.kernels = n;
  return CP_OK;
}

cp_status replay(cp_ctx* ctx, const Graph& g) {
  CP_CUDA(cudaGraphLaunch(g.exec, ctx->stream));
  g_launches.fetch_add(g.kernels);
  return CP_OK;
}

struct Mem {
  double *u, *g, *ubar, *gbar, *uhat, *d, *x, *gx, *work, *M, *grams, *scal, *U, *G;
  int* win;
  MTState* st;
  void* base = nullptr;
};

// Scalars (device scal[] and its pinned mirror).
enum { F = 0, FBAR = 1, FX = 2, SLOPE = 3, GD = 4, GG = 5, NSCAL = 8 };

struct PrecGraphs {
  Graph head, ls_eval, accept, reject, restart;
  bool ready = false;
};

}  // namespace

cp_status solve_impl(cp_ctx* ctx, const cp_tensor* t_in, const cp_solve_opts* o, double* u_user,
                     bool user_on_device, cp_solve_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  cp_tensor* t = const_cast<cp_tensor*>(t_in);
  Layout L;
  L.set(t->N, t->dims, o->R);
  const int64_t P = L.P();
  int64_t Imax = 1;
  for (int n = 0; n < L.N; ++n) Imax = std::max(Imax, L.dims[n]);
  const size_t RR = (size_t)o->R * o->R;
  const int cap = o->w;

  // The solve runs on a private capturable stream ordered after the
  // context stream's earlier work.
  cudaStream_t user_stream = ctx->stream;
  cudaStream_t ss = nullptr;
  cudaEvent_t ev = nullptr;
  CP_CUDA(cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking));
  CP_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CP_CUDA(cudaEventRecord(ev, user_stream));
  CP_CUDA(cudaStreamWaitEvent(ss, ev, 0));
  ctx->stream = ss;

  Mem s;
  double* h = ctx->h_pinned;                       // NSCAL doubles
  MTState* hst = (MTState*)(ctx->h_pinned + 16);   // line-search state mirror
  cp_solve_report r{};
  r.normT2 = t->norm2;
  cp_precision prec = o->prec;
  bool polish_pending = (o->prec != CP_FP64) && o->polish;
  const double tol_mixed = o->tol * (o->mixed_tol_factor > 0 ? o->mixed_tol_factor : 1.0);
  constexpr int kMixedStall = 50;   // mixed iterations without a new best ||g|| before FP64
  double best_mixed = INFINITY;
  int since_best = 0;
  PrecGraphs graphs[2];

  auto body = [&]() -> cp_status {
    const size_t bytes = sizeof(double) * (9 * (size_t)P + 2 * (size_t)cap * P + (size_t)Imax * o->R +
                                           (size_t)L.N * RR + 16) +
                         sizeof(MTState) + 256 + 64;
    CP_CUDA(cudaMallocAsync(&s.base, bytes, ctx->stream));
    double* p = (double*)s.base;
    s.u = p; p += P;
    s.g = p; p += P;
    s.ubar = p; p += P;
    s.gbar = p; p += P;
    s.uhat = p; p += P;
    s.d = p; p += P;
    s.x = p; p += P;
    s.gx = p; p += P;
    s.work = p; p += P;
    s.U = p; p += (size_t)cap * P;
    s.G = p; p += (size_t)cap * P;
    s.M = p; p += (size_t)Imax * o->R;
    s.grams = p; p += (size_t)L.N * RR;
    s.scal = p; p += 16;
    s.win = (int*)p; p += 8;
    s.st = (MTState*)(((uintptr_t)p + 63) & ~(uintptr_t)63);
    if (o->prec != CP_FP64) CP_TRY(prepare_mixed(ctx, t));

    auto to_host = [&]() -> cp_status {
      CP_CUDA(cudaMemcpyAsync(h, s.scal, sizeof(double) * NSCAL, cudaMemcpyDeviceToHost, ctx->stream));
      return CP_OK;
    };
    auto st_to_host = [&]() -> cp_status {
      CP_CUDA(cudaMemcpyAsync(hst, s.st, sizeof(MTState), cudaMemcpyDeviceToHost, ctx->stream));
      return CP_OK;
    };
    auto sync = [&]() -> cp_status {
      CP_CUDA(cudaStreamSynchronize(ctx->stream));
      return CP_OK;
    };
    auto build = [&](cp_precision pr) -> cp_status {
      PrecGraphs& G = graphs[pr == CP_FP64 ? 0 : 1];
      if (G.ready) return CP_OK;
      CP_TRY(capture(ctx, [&]() -> cp_status {
        CP_CUDA(cudaMemcpyAsync(s.work, s.u, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
        CP_TRY(grams_all(ctx, L, s.work, s.grams));
        CP_TRY(als_sweep_inplace(ctx, t, L, s.work, s.grams, s.M, pr));
        CP_TRY(normalize_into(ctx, L, s.work, s.ubar, nullptr, nullptr, nullptr));
        CP_TRY(fg_eval(ctx, t, L, s.ubar, s.scal + FBAR, s.gbar, pr));
        CP_TRY(ngmres_core(ctx, P, s.win, cap, s.U, s.G, s.ubar, s.gbar, o->eps, s.work, nullptr));
        CP_TRY(normalize_into(ctx, L, s.work, s.uhat, nullptr, nullptr, nullptr));
        CP_TRY(sub(ctx, P, s.uhat, s.ubar, s.d));
        CP_TRY(dot(ctx, P, s.gbar, s.d, s.scal + SLOPE));
        cp_ls_opts lso = o->ls;
        if (pr != CP_FP64 && o->mixed_maxfev > 0 && o->mixed_maxfev < lso.maxfev) lso.maxfev = o->mixed_maxfev;
        CP_TRY(mt_start(ctx, s.st, s.scal + FBAR, s.scal + SLOPE, lso));
        CP_TRY(to_host());
        return st_to_host();
      }, G.head));
      CP_TRY(capture(ctx, [&]() -> cp_status {
        CP_TRY(axpy_scalar(ctx, P, s.ubar, s.d, &s.st->stp, s.x));
        CP_TRY(fg_eval(ctx, t, L, s.x, s.scal + FX, s.gx, pr));
        CP_TRY(dot(ctx, P, s.gx, s.d, s.scal + GD));
        CP_TRY(mt_iterate(ctx, s.st, s.scal + FX, s.scal + GD));
        return st_to_host();
      }, G.ls_eval));
      CP_TRY(capture(ctx, [&]() -> cp_status {
        CP_TRY(normalize_into(ctx, L, s.x, s.u, s.gx, s.g, nullptr));
        CP_CUDA(cudaMemcpyAsync(s.scal + F, s.scal + FX, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CP_TRY(window_update(ctx, s.win, cap, false, P, s.u, s.g, s.U, s.G));
        CP_TRY(dot(ctx, P, s.g, s.g, s.scal + GG));
        return to_host();
      }, G.accept));
      for (int reset = 0; reset < 2; ++reset) {
        CP_TRY(capture(ctx, [&]() -> cp_status {
          CP_CUDA(cudaMemcpyAsync(s.u, s.ubar, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
          CP_CUDA(cudaMemcpyAsync(s.g, s.gbar, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
          CP_CUDA(cudaMemcpyAsync(s.scal + F, s.scal + FBAR, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
          CP_TRY(window_update(ctx, s.win, cap, reset != 0, P, s.u, s.g, s.U, s.G));
          CP_TRY(dot(ctx, P, s.g, s.g, s.scal + GG));
          return to_host();
        }, reset ? G.restart : G.reject));
      }
      G.ready = true;
      return CP_OK;
    };
    // start-up: u0 normalised, f and g at u0, window {(u0, g0)}
    auto start = [&](cp_precision pr, bool from_user) -> cp_status {
      if (from_user) {
        CP_CUDA(cudaMemcpyAsync(s.work, u_user, sizeof(double) * P,
                                user_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
        CP_TRY(normalize_into(ctx, L, s.work, s.u, nullptr, nullptr, nullptr));
      }
      CP_TRY(fg_eval(ctx, t, L, s.u, s.scal + F, s.g, pr));
      CP_TRY(window_update(ctx, s.win, cap, true, P, s.u, s.g, s.U, s.G));
      CP_TRY(dot(ctx, P, s.g, s.g, s.scal + GG));
      CP_TRY(to_host());
      return sync();
    };

    CP_TRY(start(prec, true));
    r.fg_evals++;
    CP_TRY(build(prec));
    for (;;) {
      CP_TRY(read_status(ctx));
      const double gn = std::sqrt(h[GG]) / (double)P;
      r.f = h[F];
      r.gnorm_over_P = gn;
      if (!std::isfinite(gn)) {
        set_error("cp_solve: non-finite gradient");
        return CP_ERR_NONFINITE;
      }
      const bool mixed_phase = prec != CP_FP64 && polish_pending;
      bool stalled = false;
      if (mixed_phase) {
        if (gn < best_mixed) {
          best_mixed = gn;
          since_best = 0;
        } else if (++since_best >= kMixedStall) {
          stalled = true;
        }
      }
      if (mixed_phase && (gn < tol_mixed || stalled)) {
        // polish: exact FP64 gradient at u, fresh window, FP64 graphs
        prec = CP_FP64;
        polish_pending = false;
        CP_TRY(start(prec, false));
        r.fg_evals++;
        CP_TRY(build(prec));
        continue;
      }
      if (gn < o->tol && (prec == CP_FP64 || !o->polish)) {
        r.converged = 1;
        break;
      }
      if (r.iters >= o->maxit) break;
      PrecGraphs& G = graphs[prec == CP_FP64 ? 0 : 1];
      CP_TRY(replay(ctx, G.head));
      CP_TRY(sync());
      r.als_sweeps++;
      r.fg_evals++;
      if (!(h[SLOPE] < 0.0)) {
        r.restarts++;
        CP_TRY(replay(ctx, G.restart));
        CP_TRY(sync());
      } else {
        for (int k = 0; k <= o->ls.maxfev && !hst->done; ++k) {
          CP_TRY(replay(ctx, G.ls_eval));
          CP_TRY(sync());
        }
        const MTState ms = *hst;
        r.fg_evals += ms.nfev;
        if (ms.info != 1) r.ls_failures++;
        const bool accept = ms.nfev > 0 && (ms.info == 1 || ms.f <= ms.f0 + ms.ftol * ms.stp_eval * ms.g0);
        CP_TRY(replay(ctx, accept ? G.accept : G.reject));
        CP_TRY(sync());
      }
      r.iters++;
      if (prec == CP_FP64)
        r.fp64_iters++;
      else
        r.mixed_iters++;
    }
    CP_CUDA(cudaMemcpyAsync(u_user, s.u, sizeof(double) * P,
                            user_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CP_TRY(sync());
    return read_status(ctx);
  };
  cp_status result = body();
  if (s.base) cudaFreeAsync(s.base, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  ctx->stream = user_stream;
  cudaEventDestroy(ev);
  cudaStreamDestroy(ss);
  r.t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rep) *rep = r;
  if (result == CP_OK && !r.converged) {
    set_error("cp_solve: tol not met after %d iterations (||g||/P = %.3e)", r.iters, r.gnorm_over_P);
    return CP_ERR_MAXIT;
  }
  return result;
}

}  // namespace cpg
