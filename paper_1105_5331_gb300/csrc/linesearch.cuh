// Device-resident state of the More-Thuente line search (Step III).
#pragma once

#include "cp_internal.cuh"

namespace cpg {

struct MTState {
  double f0, g0;                  // phi(0), phi'(0)
  double stp;                     // next trial step
  double stp_eval;                // step of the last evaluation
  double f, g;                    // phi, phi' at stp_eval
  double lo_a, lo_f, lo_g;        // best point (a_l)
  double hi_a, hi_f, hi_g;        // other end of the interval (a_u)
  double width, width1, imin, imax;
  double ftol, gtol, xtol, stpmin, stpmax;
  int maxfev, nfev, info, done, brackt, stage;
};

struct SolveCtl;
// Line search on the polynomial phi(beta) = f(base + beta d) (degree 2N):
// one MTTKRP pass for its coefficients (Grams on ctx->aux), then the whole
// More-Thuente search in one thread.  st receives the final state (stp_eval,
// f = phi there, nfev, info); poly the 2N + 1 coefficients.  With ctl the
// solver counters are updated, and with use_h the graph condition h is set to
// "accept" (info 1, or sufficient decrease at the last trial).  mv_out
// (nullable, 2^(N-1) x P doubles; mode n's block of 2^(N-1) x I_n x R at
// 2^(N-1) L.off[n]): the variant MTTKRPs M_v of the last mode, and, where
// one tensor-core launch can make them alongside (dense, mixed precision),
// those of every other mode too; *all_modes (nullable) tells which.
// grams_out (nullable, 3 x N x R x R): keeps the Grams the polynomial is
// built from, base^T base, base^T d and d^T d per mode (in that order).
// base32 / d32 (nullable): padded FP32 copies of base and d (f32_layout),
// used instead of making them.
cp_status ls_poly(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* base, const double* d,
                  cp_precision prec, const cp_ls_opts& o, MTState* st, double* poly, SolveCtl* ctl,
                  cudaGraphConditionalHandle h, int use_h, double* mv_out = nullptr, bool* all_modes = nullptr,
                  double* grams_out = nullptr, const float* base32 = nullptr, const float* d32_in = nullptr);


}  // namespace cpg
