// The N-GMRES optimisation algorithm (Algorithm 1, Steps I-III of Section
// 2.1) with ALS as the one-step process M(.) (Section 2.3), windowed start-up
// and window size w (Section 2.1), the restart rule of Section 2.1 and the
// delta I regularisation with eps = 1e-12 (Section 2.4).
//
// Every vector stays on the device; per iteration the host reads three kinds
// of scalars to steer control flow: ||g||, the slope g(ubar)^T d, and the
// line search's "done" flag after each evaluation.
//
// Mixed precision: iterations run with bf16x3 MTTKRPs until ||g||/P drops
// below tol * mixed_tol_factor; then the window is reset and FP64 iterations
// continue until the FP64 gradient meets tol (the polish).
#include <chrono>
#include <cmath>

#include "cp_internal.cuh"
#include "linesearch.cuh"

namespace cpg {

namespace {

struct Window {
  double* U = nullptr;
  double* G = nullptr;
  int cap = 0, start = 0, m = 0;
};

cp_status window_reset(cp_ctx* ctx, Window& w, int64_t P, const double* u, const double* g) {
  w.start = 0;
  w.m = 1;
  CP_CUDA(cudaMemcpyAsync(w.U, u, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
  CP_CUDA(cudaMemcpyAsync(w.G, g, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
  return CP_OK;
}

cp_status window_push(cp_ctx* ctx, Window& w, int64_t P, const double* u, const double* g) {
  int slot;
  if (w.m < w.cap) {
    slot = (w.start + w.m) % w.cap;
    ++w.m;
  } else {
    slot = w.start;
    w.start = (w.start + 1) % w.cap;
  }
  CP_CUDA(cudaMemcpyAsync(w.U + (int64_t)slot * P, u, sizeof(double) * P, cudaMemcpyDeviceToDevice,
                          ctx->stream));
  CP_CUDA(cudaMemcpyAsync(w.G + (int64_t)slot * P, g, sizeof(double) * P, cudaMemcpyDeviceToDevice,
                          ctx->stream));
  return CP_OK;
}

}  // namespace

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

struct SolveMem {
  double *u, *g, *ubar, *gbar, *uhat, *d, *x, *gx, *work, *M, *grams, *scal;
  MTState* st;
  Window w;
  void* base = nullptr;
};

cp_status solve_impl(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts* o, double* u_user,
                     bool user_on_device, cp_solve_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  Layout L;
  L.set(t->N, t->dims, o->R);
  const int64_t P = L.P();
  int64_t Imax = 1;
  for (int n = 0; n < L.N; ++n) Imax = std::max(Imax, L.dims[n]);
  const size_t RR = (size_t)o->R * o->R;
  // one allocation for all solver state
  const size_t nvec = 9;
  size_t bytes = sizeof(double) * (nvec * (size_t)P + 2 * (size_t)o->w * P + (size_t)Imax * o->R +
                                   (size_t)L.N * RR + 16) +
                 sizeof(MTState) + 256;
  SolveMem s;
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
  s.w.U = p; p += (size_t)o->w * P;
  s.w.G = p; p += (size_t)o->w * P;
  s.w.cap = o->w;
  s.M = p; p += (size_t)Imax * o->R;
  s.grams = p; p += (size_t)L.N * RR;
  s.scal = p; p += 16;
  s.st = (MTState*)(((uintptr_t)p + 63) & ~(uintptr_t)63);
  double* f = s.scal + 0;
  double* fbar = s.scal + 1;
  double* fx = s.scal + 2;
  double* slope = s.scal + 3;
  double* gd = s.scal + 4;
  double* gg = s.scal + 5;
  double* h = ctx->h_pinned;
  MTState* host_st = (MTState*)(ctx->h_pinned + 16);

  cp_solve_report r{};
  r.normT2 = t->norm2;
  cp_status result = CP_OK;
  cp_precision prec = o->prec;
  bool polish_pending = (o->prec != CP_FP64) && o->polish;
  const double tol_now_mixed = o->tol * (o->mixed_tol_factor > 0 ? o->mixed_tol_factor : 1.0);
  constexpr int kMixedStall = 50;   // mixed iterations without a new best ||g|| before FP64
  double best_mixed = INFINITY;
  int since_best = 0;

  auto body = [&]() -> cp_status {
    CP_CUDA(cudaMemcpyAsync(s.work, u_user, sizeof(double) * P,
                            user_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            ctx->stream));
    CP_TRY(normalize_into(ctx, L, s.work, s.u, nullptr, nullptr, nullptr));
    CP_TRY(fg_eval(ctx, t, L, s.u, f, s.g, prec));
    r.fg_evals++;
    CP_TRY(window_reset(ctx, s.w, P, s.u, s.g));
    for (;;) {
      CP_TRY(dot(ctx, P, s.g, s.g, gg));
      CP_CUDA(cudaMemcpyAsync(h, s.scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, ctx->stream));
      CP_CUDA(cudaStreamSynchronize(ctx->stream));
      CP_TRY(read_status(ctx));
      const double gn = std::sqrt(h[5]) / (double)P;
      r.f = h[0];
      r.gnorm_over_P = gn;
      if (!std::isfinite(gn)) return CP_ERR_NONFINITE;
      const double tol_now = (prec != CP_FP64 && polish_pending) ? tol_now_mixed : o->tol;
      // a mixed phase that stops improving hands over to FP64 early
      if (prec != CP_FP64 && polish_pending) {
        if (gn < best_mixed) {
          best_mixed = gn;
          since_best = 0;
        } else if (++since_best >= kMixedStall) {
          best_mixed = 0.0;   // forces the switch below
        }
      }
      if (gn < tol_now || (prec != CP_FP64 && polish_pending && best_mixed == 0.0)) {
        if (prec != CP_FP64 && polish_pending) {
          // switch to FP64: exact gradient at u, fresh window
          prec = CP_FP64;
          polish_pending = false;
          CP_TRY(fg_eval(ctx, t, L, s.u, f, s.g, prec));
          r.fg_evals++;
          CP_TRY(window_reset(ctx, s.w, P, s.u, s.g));
          continue;
        }
        if (prec == CP_FP64 || !o->polish) {
          r.converged = 1;
          break;
        }
      }
      if (r.iters >= o->maxit) break;
      // Step I: ubar = normalise(ALS(u))
      CP_CUDA(cudaMemcpyAsync(s.work, s.u, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
      CP_TRY(grams_all(ctx, L, s.work, s.grams));
      CP_TRY(als_sweep_inplace(ctx, t, L, s.work, s.grams, s.M, prec));
      r.als_sweeps++;
      CP_TRY(normalize_into(ctx, L, s.work, s.ubar, nullptr, nullptr, nullptr));
      CP_TRY(fg_eval(ctx, t, L, s.ubar, fbar, s.gbar, prec));
      r.fg_evals++;
      // Step II: uhat from the window, normalised; d = uhat - ubar
      CP_TRY(ngmres_core(ctx, P, s.w.m, s.w.U, s.w.G, s.w.start, s.w.cap, s.ubar, s.gbar, o->eps,
                         s.work, nullptr));
      CP_TRY(normalize_into(ctx, L, s.work, s.uhat, nullptr, nullptr, nullptr));
      CP_TRY(sub(ctx, P, s.uhat, s.ubar, s.d));
      CP_TRY(dot(ctx, P, s.gbar, s.d, slope));
      CP_CUDA(cudaMemcpyAsync(h, s.scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, ctx->stream));
      CP_CUDA(cudaStreamSynchronize(ctx->stream));
      const double sl = h[3];
      if (!(sl < 0.0)) {
        // restart: u_{i+1} = ubar, window {(ubar, g(ubar))}
        r.restarts++;
        CP_CUDA(cudaMemcpyAsync(s.u, s.ubar, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
        CP_CUDA(cudaMemcpyAsync(s.g, s.gbar, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
        CP_CUDA(cudaMemcpyAsync(f, fbar, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CP_TRY(window_reset(ctx, s.w, P, s.u, s.g));
      } else {
        // Step III: line search along d from ubar
        CP_TRY(run_linesearch(ctx, t, L, s.ubar, fbar, slope, s.d, o->ls, s.x, fx, s.gx, gd, s.st,
                              prec, host_st));
        const MTState& ms = *host_st;
        r.fg_evals += ms.nfev;
        if (ms.info != 1) r.ls_failures++;
        const bool accept =
            ms.nfev > 0 && (ms.info == 1 || ms.f <= ms.f0 + ms.ftol * ms.stp_eval * ms.g0);
        if (accept) {
          CP_TRY(normalize_into(ctx, L, s.x, s.u, s.gx, s.g, nullptr));
          CP_CUDA(cudaMemcpyAsync(f, fx, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        } else {
          CP_CUDA(cudaMemcpyAsync(s.u, s.ubar, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
          CP_CUDA(cudaMemcpyAsync(s.g, s.gbar, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
          CP_CUDA(cudaMemcpyAsync(f, fbar, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        }
        CP_TRY(window_push(ctx, s.w, P, s.u, s.g));
      }
      r.iters++;
      if (prec == CP_FP64 && o->prec != CP_FP64)
        r.fp64_iters++;
      else if (prec != CP_FP64)
        r.mixed_iters++;
      else
        r.fp64_iters++;
    }
    CP_CUDA(cudaMemcpyAsync(u_user, s.u, sizeof(double) * P,
                            user_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            ctx->stream));
    CP_CUDA(cudaStreamSynchronize(ctx->stream));
    return read_status(ctx);
  };
  result = body();
  cudaFreeAsync(s.base, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  r.t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rep) *rep = r;
  if (result == CP_OK && !r.converged) {
    set_error("cp_solve: tol not met after %d iterations (||g||/P = %.3e)", r.iters, r.gnorm_over_P);
    return CP_ERR_MAXIT;
  }
  return result;
}

}  // namespace cpg
