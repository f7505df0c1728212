// Normalisation scales and term order (Section 2.3), computed by every block
// that applies them: nu[n][r] = ||a_r^(n)||, lambda_r = prod_n nu,
// scale = lambda^(1/N) / nu, order = stable sort by decreasing lambda.  The
// column sums of squares come from the Gram diagonals (grams) or from
// per-chunk partial sums part[n][S][R].
#pragma once

#include "cp_internal.cuh"
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
    sh.nu[t] = sqrt(s);
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
    const double root = pow(l, 1.0 / N);
    for (int n = 0; n < N; ++n) sh.scale[n * R + r] = zero ? 1.0 : root / sh.nu[n * R + r];
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
