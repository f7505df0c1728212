// Step III of N-GMRES (Section 2.1, Eq. linesearch, Eq. new) with the
// More-Thuente line search the paper uses (Section 2.4 parameters; method of
// J. J. More and D. J. Thuente, ACM TOMS 20(3), 1994).
//
// The search state lives in device memory and is advanced by a one-thread
// kernel after each evaluation of phi(beta) = f(x0 + beta d) and
// phi'(beta) = g(x0 + beta d)^T d, so the iterate never leaves the GPU; the
// host only learns whether another evaluation is wanted.
//
// Algorithm (as published):
//  * sufficient decrease  phi(a) <= phi(0) + ftol a phi'(0),
//    curvature            |phi'(a)| <= gtol |phi'(0)|;
//  * stage 1 works on psi(a) = phi(a) - phi(0) - ftol a phi'(0) until a trial
//    has psi <= 0 and phi' >= min(ftol, gtol) phi'(0);
//  * trial selection by the four cases of cubic / quadratic / secant
//    interpolation, the interval update rules, extrapolation into
//    [a_t + 1.1 (a_t - a_l), a_t + 4 (a_t - a_l)] while unbracketed, and
//    bisection when a bracketed interval fails to shrink by 0.66 in two trials.
#include <cmath>

#include "cp_internal.cuh"
#include "linesearch.cuh"
#include "mt_device.cuh"

namespace cpg {

namespace {

__global__ void mt_start_kernel(MTState* st, const double* f0, const double* g0, cp_ls_opts o) {
  MTState s;
  s.ftol = o.ftol;
  s.gtol = o.gtol;
  s.xtol = o.xtol;
  s.stpmin = o.stpmin;
  s.stpmax = o.stpmax;
  s.maxfev = o.maxfev;
  s.f0 = *f0;
  s.g0 = *g0;
  s.nfev = 0;
  s.info = 0;
  s.done = 0;
  s.brackt = 0;
  s.stage = 1;
  s.lo_a = 0.0; s.lo_f = s.f0; s.lo_g = s.g0;
  s.hi_a = 0.0; s.hi_f = s.f0; s.hi_g = s.g0;
  s.width = o.stpmax - o.stpmin;
  s.width1 = 2.0 * s.width;
  s.stp = fmin(fmax(o.stp0, o.stpmin), o.stpmax);
  s.imin = 0.0;
  s.imax = s.stp + 4.0 * s.stp;
  s.stp_eval = s.stp;
  s.f = s.f0;
  s.g = s.g0;
  if (!(s.g0 < 0.0)) {
    s.info = -1;
    s.done = 1;
    s.stp_eval = 0.0;
  }
  *st = s;
}

// Consume phi(stp), phi'(stp); decide termination or the next trial.
__global__ void mt_iterate_kernel(MTState* st, const double* fval, const double* gval) {
  mtdev::mt_advance(st, fval, gval);
}

// The same step inside a graph: the enclosing WHILE node repeats the
// evaluation while the search is not done.
__global__ void mt_iterate_cond_kernel(MTState* st, const double* fval, const double* gval,
                                       cudaGraphConditionalHandle h) {
  mtdev::mt_advance(st, fval, gval);
  cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

}  // namespace

cp_status mt_start(cp_ctx* ctx, MTState* st, const double* f0, const double* g0,
                   const cp_ls_opts& o) {
  mt_start_kernel<<<1, 1, 0, ctx->stream>>>(st, f0, g0, o);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

cp_status mt_iterate(cp_ctx* ctx, MTState* st, const double* f, const double* g) {
  mt_iterate_kernel<<<1, 1, 0, ctx->stream>>>(st, f, g);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

cp_status mt_iterate_cond(cp_ctx* ctx, MTState* st, const double* f, const double* g,
                          cudaGraphConditionalHandle h) {
  mt_iterate_cond_kernel<<<1, 1, 0, ctx->stream>>>(st, f, g, h);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

// Runs the search: x = x0 + stp d, f and g at x, phi' = g . d.  The last
// evaluated point is left in x, fx, gx.  Host reads one flag per evaluation.
cp_status run_linesearch(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* x0,
                         const double* f0, const double* slope, const double* d,
                         const cp_ls_opts& o, double* x, double* fx, double* gx, double* gd,
                         MTState* st, cp_precision prec, MTState* host_out) {
  const int64_t P = L.P();
  CP_TRY(mt_start(ctx, st, f0, slope, o));
  for (int it = 0; it < o.maxfev + 1; ++it) {
    CP_CUDA(cudaMemcpyAsync(host_out, st, sizeof(MTState), cudaMemcpyDeviceToHost, ctx->stream));
    CP_CUDA(cudaStreamSynchronize(ctx->stream));
    if (host_out->done) break;
    CP_TRY(axpy_scalar(ctx, P, x0, d, &st->stp, x));
    CP_TRY(fg_eval(ctx, t, L, x, fx, gx, prec));
    CP_TRY(dot(ctx, P, gx, d, gd));
    CP_TRY(mt_iterate(ctx, st, fx, gd));
  }
  return CP_OK;
}

}  // namespace cpg
