// Small dense FP64 linear algebra executed by one thread block.
#pragma once

namespace cpg {

// In-place lower Cholesky of the R x R row-major matrix S in shared memory
// (right-looking, all threads of the block).  Returns false if a pivot is
// not positive and finite.
__device__ inline bool chol_block(double* S, int R, int* flag) {
  for (int k = 0; k < R; ++k) {
    if (threadIdx.x == 0) {
      const double d = S[k * R + k];
      if (!(d > 0.0) || !isfinite(d))
        *flag = 1;
      else
        S[k * R + k] = sqrt(d);
    }
    __syncthreads();
    if (*flag) return false;
    const double piv = S[k * R + k];
    for (int i = k + 1 + threadIdx.x; i < R; i += blockDim.x) S[i * R + k] /= piv;
    __syncthreads();
    const int rem = R - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      if (j <= i) S[i * R + j] -= S[i * R + k] * S[j * R + k];
    }
    __syncthreads();
  }
  return true;
}

}  // namespace cpg
