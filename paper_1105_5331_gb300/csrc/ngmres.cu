// N-GMRES Step II (Section 2.1, Eq. accel, Eq. linearize, Eq. normal): from a
// window of m previous iterates u_j and gradients g(u_j), and the preliminary
// iterate ubar with gradient gbar,
//     p_j = gbar - g(u_j),  (P^T P + delta I) alpha = -P^T gbar,
//     delta = eps * max_j (P^T P)_jj,  uhat = ubar + sum_j alpha_j (ubar - u_j).
// One pass over the window computes every p_j . p_l and p_j . gbar (the p_j
// are formed per element, never stored); one block reduces the per-CTA sums in
// a fixed order, factors the m x m system by Cholesky and solves for alpha; a
// last pass forms uhat.
#include <algorithm>

#include "cp_internal.cuh"
#include "dev_linalg.cuh"

namespace cpg {

namespace {

constexpr int kTile = 32;
constexpr int kMaxOutPerThread = 9;   // (64*65/2 + 64) / 256 rounded up

__device__ __forceinline__ void pair_of(int o, int m, int* j, int* l) {
  // o enumerates (j, l), j <= l, row by row: (0,0),(0,1),...,(0,m-1),(1,1),...
  int jj = 0, base = 0;
  while (o >= base + (m - jj)) {
    base += m - jj;
    ++jj;
  }
  *j = jj;
  *l = jj + (o - base);
}

__global__ void ngmres_dots_kernel(const double* __restrict__ G, int start, int wcap, int m,
                                   int64_t P, const double* __restrict__ gbar, int64_t chunk,
                                   double* __restrict__ part) {
  __shared__ double pt[CP_MAX_W * (kTile + 1)];
  __shared__ double gt[kTile];
  const int npairs = m * (m + 1) / 2;
  const int nout = npairs + m;
  int oj[kMaxOutPerThread], ol[kMaxOutPerThread];
  double acc[kMaxOutPerThread];
#pragma unroll
  for (int q = 0; q < kMaxOutPerThread; ++q) {
    const int o = threadIdx.x + q * blockDim.x;
    acc[q] = 0.0;
    oj[q] = -1;
    ol[q] = -1;
    if (o < npairs) {
      pair_of(o, m, &oj[q], &ol[q]);
    } else if (o < nout) {
      oj[q] = o - npairs;
      ol[q] = -1;   // right-hand side entry
    }
  }
  const int64_t kb = (int64_t)blockIdx.x * chunk;
  const int64_t ke = min(P, kb + chunk);
  for (int64_t k0 = kb; k0 < ke; k0 += kTile) {
    const int kt = (int)min((int64_t)kTile, ke - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kt; e += blockDim.x) gt[e] = gbar[k0 + e];
    for (int e = threadIdx.x; e < m * kt; e += blockDim.x) {
      const int j = e / kt, kk = e - (e / kt) * kt;
      const int slot = (start + j) % wcap;
      pt[j * (kTile + 1) + kk] = gbar[k0 + kk] - G[(int64_t)slot * P + k0 + kk];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxOutPerThread; ++q) {
      if (oj[q] < 0) continue;
      const double* a = pt + oj[q] * (kTile + 1);
      const double* b = ol[q] >= 0 ? pt + ol[q] * (kTile + 1) : gt;
      double s = acc[q];
      for (int kk = 0; kk < kt; ++kk) s = fma(a[kk], b[kk], s);
      acc[q] = s;
    }
  }
#pragma unroll
  for (int q = 0; q < kMaxOutPerThread; ++q) {
    const int o = threadIdx.x + q * blockDim.x;
    if (o < nout) part[(int64_t)blockIdx.x * nout + o] = acc[q];
  }
}

__global__ void ngmres_solve_kernel(const double* __restrict__ part, int nparts, int m, double eps,
                                    double* __restrict__ alpha, int* status) {
  __shared__ double H[CP_MAX_W * CP_MAX_W];
  __shared__ double rhs[CP_MAX_W];
  __shared__ double dmax;
  __shared__ int flag;
  const int npairs = m * (m + 1) / 2;
  const int nout = npairs + m;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * nout + o];
    if (o < npairs) {
      int j, l;
      pair_of(o, m, &j, &l);
      H[j * m + l] = s;
      H[l * m + j] = s;
    } else {
      rhs[o - npairs] = -s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int j = 0; j < m; ++j) d = fmax(d, H[j * m + j]);
    dmax = d;
    flag = 0;
    if (d > 0.0)
      for (int j = 0; j < m; ++j) H[j * m + j] += eps * d;
  }
  __syncthreads();
  if (!(dmax > 0.0)) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) alpha[j] = 0.0;
    return;
  }
  if (!chol_block(H, m, &flag)) {
    if (threadIdx.x == 0) record_status(status, CP_ERR_NOT_SPD);
    for (int j = threadIdx.x; j < m; j += blockDim.x) alpha[j] = 0.0;
    return;
  }
  if (threadIdx.x == 0) {
    double y[CP_MAX_W];
    for (int r = 0; r < m; ++r) {
      double v = rhs[r];
      for (int s = 0; s < r; ++s) v -= H[r * m + s] * y[s];
      y[r] = v / H[r * m + r];
    }
    for (int r = m - 1; r >= 0; --r) {
      double v = y[r];
      for (int s = r + 1; s < m; ++s) v -= H[s * m + r] * y[s];
      y[r] = v / H[r * m + r];
    }
    for (int r = 0; r < m; ++r) alpha[r] = y[r];
  }
}

__global__ void ngmres_combine_kernel(const double* __restrict__ U, int start, int wcap, int m,
                                      int64_t P, const double* __restrict__ ubar,
                                      const double* __restrict__ alpha, double* __restrict__ uhat) {
  __shared__ double a[CP_MAX_W];
  for (int j = threadIdx.x; j < m; j += blockDim.x) a[j] = alpha[j];
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double ub = ubar[k];
    double acc = 0.0;
    for (int j = 0; j < m; ++j) {
      const int slot = (start + j) % wcap;
      acc += a[j] * (ub - U[(int64_t)slot * P + k]);
    }
    uhat[k] = ub + acc;
  }
}

}  // namespace

cp_status ngmres_core(cp_ctx* ctx, int64_t P, int m, const double* U, const double* G, int start,
                      int wcap, const double* ubar, const double* gbar, double eps, double* uhat,
                      double* alpha) {
  if (m < 1 || m > CP_MAX_W) {
    set_error("ngmres: window size %d outside [1, %d]", m, CP_MAX_W);
    return CP_ERR_ARG;
  }
  const int nout = m * (m + 1) / 2 + m;
  int64_t nb = std::min<int64_t>((P + 255) / 256, 2 * (int64_t)ctx->num_sms);
  nb = std::max<int64_t>(nb, 1);
  const int64_t chunk = (P + nb - 1) / nb;
  nb = (P + chunk - 1) / chunk;
  if (nb < 1) nb = 1;
  double* part = nullptr;
  double* a = alpha;
  CP_TRY(ws_alloc(ctx, (void**)&part, sizeof(double) * ((size_t)nb * nout + CP_MAX_W)));
  if (!a) a = part + (size_t)nb * nout;
  ngmres_dots_kernel<<<(unsigned)nb, 256, 0, ctx->stream>>>(G, start, wcap, m, P, gbar, chunk, part);
  CP_LAUNCH_CHECK();
  ngmres_solve_kernel<<<1, 256, 0, ctx->stream>>>(part, (int)nb, m, eps, a, ctx->d_status);
  CP_LAUNCH_CHECK();
  int64_t cb = std::min<int64_t>((P + 255) / 256, 8 * (int64_t)ctx->num_sms);
  ngmres_combine_kernel<<<(unsigned)std::max<int64_t>(cb, 1), 256, 0, ctx->stream>>>(
      U, start, wcap, m, P, ubar, a, uhat);
  CP_LAUNCH_CHECK();
  ws_free(ctx, part);
  return CP_OK;
}

}  // namespace cpg
