// Normalisation scales and term order (Section 2.3), computed by every block
// that applies them: nu[n][r] = ||a_r^(n)||, lambda_r = prod_n nu,
// scale = lambda^(1/N) / nu, order = stable sort by decreasing lambda.  The
// column sums of squares come from the Gram diagonals (grams) or from
// per-chunk partial sums part[n][S][R].
//
// FP64 divides, square roots and pow are slow, serial chains on this GPU
// (pow about 5800 cycles, a divide or sqrt about 650), and every block waits
// for this prologue.  So y = 1/nu comes from Newton's iteration for
// 1/sqrt(s) (rsqrt_nr), nu = s y, scale = lambda^(1/N) y, and lambda^(1/N)
// is cbrt / sqrt for N = 3, 2, 4 (pow otherwise).
#pragma once

#include "cp_internal.cuh"
#include "newton.cuh"
#include "reduce.cuh"

namespace cpg {

struct NormShared {
  double nu[CP_MAX_N * CP_MAX_R];
  double scale[CP_MAX_N * CP_MAX_R];
  double key[CP_MAX_R];
  double lam[CP_MAX_R];
  int order[CP_MAX_R];
};

__device__ inline void norm_prologue(const Layout& L, const double* __restrict__ part, int S,
                                     const double* __restrict__ grams, double* __restrict__ lambda_out, int* status,
                                     NormShared& sh) {
  const int N = L.N, R = L.R;
  for (int t = threadIdx.x; t < N * R; t += blockDim.x) {
    const int n = t / R, r = t - (t / R) * R;
    double s;
    if (grams) {
      s = grams[(int64_t)n * R * R + r * R + r];
    } else {
      s = strided_sum(part + (int64_t)n * S * R + r, 0, S, 1, (int64_t)R);
    }
    const double y = s > 0.0 ? rsqrt_nr(s) : 0.0;
    sh.nu[t] = s * y;
    sh.scale[t] = y;   // 1 / nu for now
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double l = 1.0;
    bool zero = false;
    for (int n = 0; n < N; ++n) {
      l *= sh.nu[n * R + r];
      if (sh.nu[n * R + r] == 0.0) zero = true;
    }
    if (zero) l = 0.0;
    const double root = N == 3 ? cbrt(l) : N == 2 ? sqrt(l) : N == 4 ? sqrt(sqrt(l)) : pow(l, 1.0 / N);
    for (int n = 0; n < N; ++n) sh.scale[n * R + r] = zero ? 1.0 : root * sh.scale[n * R + r];
    sh.lam[r] = l;
    sh.key[r] = isnan(l) ? -INFINITY : l;
    if (!isfinite(l) && blockIdx.x == 0) record_status(status, CP_ERR_NONFINITE);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    int rank = 0;
    for (int s = 0; s < R; ++s)
      if (sh.key[s] > sh.key[r] || (sh.key[s] == sh.key[r] && s < r)) ++rank;
    sh.order[rank] = r;
    if (lambda_out && blockIdx.x == 0) lambda_out[rank] = sh.lam[r];
  }
  __syncthreads();
}

}  // namespace cpg
