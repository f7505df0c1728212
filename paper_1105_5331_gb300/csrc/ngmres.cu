// N-GMRES Step II (Section 2.1, Eq. accel, Eq. linearize, Eq. normal): from a
// window of m previous iterates u_j and gradients g(u_j), and the preliminary
// iterate ubar with gradient gbar,
//     p_j = gbar - g(u_j),  (P^T P + delta I) alpha = -P^T gbar,
//     delta = eps * max_j (P^T P)_jj,  uhat = ubar + sum_j alpha_j (ubar - u_j).
// One pass over the window computes every p_j . p_l and p_j . gbar (the p_j
// are formed per element, never stored); one block reduces the per-CTA sums in
// a fixed order, factors the m x m system by Cholesky and solves for alpha; a
// last pass forms uhat.
//
// The window is a ring of `cap` slots in device memory; its state
// win = {start, m} also lives in device memory (window row j, oldest first, is
// slot (start + j) % cap), so the whole step can be replayed from a CUDA graph
// while the window grows and rotates (window size w of Section 2.1).
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

__global__ void ngmres_dots_kernel(const double* __restrict__ G, const int* __restrict__ win, int cap,
                                   int64_t P, const double* __restrict__ gbar, int64_t chunk,
                                   int nout_max, double* __restrict__ part) {
  __shared__ double pt[CP_MAX_W * (kTile + 1)];
  __shared__ double gt[kTile];
  const int start = win[0];
  const int m = win[1];
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
      const int slot = (start + j) % cap;
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
    if (o < nout) part[(int64_t)blockIdx.x * nout_max + o] = acc[q];
  }
}

__global__ void ngmres_solve_kernel(const double* __restrict__ part, int nparts, int nout_max,
                                    const int* __restrict__ win, double eps, double* __restrict__ alpha,
                                    int* status) {
  __shared__ double H[CP_MAX_W * CP_MAX_W];
  __shared__ double rhs[CP_MAX_W];
  __shared__ double dmax;
  __shared__ int flag;
  const int m = win[1];
  const int npairs = m * (m + 1) / 2;
  const int nout = npairs + m;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * nout_max + o];
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

__global__ void ngmres_combine_kernel(const double* __restrict__ U, const int* __restrict__ win, int cap,
                                      int64_t P, const double* __restrict__ ubar,
                                      const double* __restrict__ alpha, double* __restrict__ uhat) {
  __shared__ double a[CP_MAX_W];
  const int start = win[0];
  const int m = win[1];
  for (int j = threadIdx.x; j < m; j += blockDim.x) a[j] = alpha[j];
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double ub = ubar[k];
    double acc = 0.0;
    for (int j = 0; j < m; ++j) {
      const int slot = (start + j) % cap;
      acc += a[j] * (ub - U[(int64_t)slot * P + k]);
    }
    uhat[k] = ub + acc;
  }
}

// Copy (u, g) into the slot the window update will use; win is read only.
__global__ void window_copy_kernel(const int* __restrict__ win, int cap, int reset, int64_t P,
                                   const double* __restrict__ u, const double* __restrict__ g,
                                   double* __restrict__ U, double* __restrict__ G) {
  const int start = win[0], m = win[1];
  const int slot = reset ? 0 : (m < cap ? (start + m) % cap : start);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    U[(int64_t)slot * P + k] = u[k];
    G[(int64_t)slot * P + k] = g[k];
  }
}

// Window bookkeeping after the copy: reset -> {0, 1}; push grows to cap,
// then drops the oldest.
__global__ void window_index_kernel(int* win, int cap, int reset) {
  if (reset) {
    win[0] = 0;
    win[1] = 1;
  } else if (win[1] < cap) {
    win[1] += 1;
  } else {
    win[0] = (win[0] + 1) % cap;
  }
}

}  // namespace

cp_status ngmres_core(cp_ctx* ctx, int64_t P, const int* win, int cap, const double* U, const double* G,
                      const double* ubar, const double* gbar, double eps, double* uhat, double* alpha) {
  if (cap < 1 || cap > CP_MAX_W) {
    set_error("ngmres: window capacity %d outside [1, %d]", cap, CP_MAX_W);
    return CP_ERR_ARG;
  }
  const int nout_max = cap * (cap + 1) / 2 + cap;
  int64_t nb = std::min<int64_t>((P + 255) / 256, 2 * (int64_t)ctx->num_sms);
  nb = std::max<int64_t>(nb, 1);
  const int64_t chunk = (P + nb - 1) / nb;
  nb = std::max<int64_t>((P + chunk - 1) / chunk, 1);
  double* part = nullptr;
  double* a = alpha;
  CP_TRY(ws_alloc(ctx, (void**)&part, sizeof(double) * ((size_t)nb * nout_max + CP_MAX_W)));
  if (!a) a = part + (size_t)nb * nout_max;
  ngmres_dots_kernel<<<(unsigned)nb, 256, 0, ctx->stream>>>(G, win, cap, P, gbar, chunk, nout_max, part);
  CP_LAUNCH_CHECK();
  ngmres_solve_kernel<<<1, 256, 0, ctx->stream>>>(part, (int)nb, nout_max, win, eps, a, ctx->d_status);
  CP_LAUNCH_CHECK();
  int64_t cb = std::min<int64_t>((P + 255) / 256, 8 * (int64_t)ctx->num_sms);
  ngmres_combine_kernel<<<(unsigned)std::max<int64_t>(cb, 1), 256, 0, ctx->stream>>>(U, win, cap, P, ubar, a,
                                                                                      uhat);
  CP_LAUNCH_CHECK();
  ws_free(ctx, part);
  return CP_OK;
}

cp_status window_update(cp_ctx* ctx, int* win, int cap, bool reset, int64_t P, const double* u,
                        const double* g, double* U, double* G) {
  int64_t cb = std::min<int64_t>((P + 255) / 256, 8 * (int64_t)ctx->num_sms);
  window_copy_kernel<<<(unsigned)std::max<int64_t>(cb, 1), 256, 0, ctx->stream>>>(win, cap, reset ? 1 : 0, P, u,
                                                                                   g, U, G);
  CP_LAUNCH_CHECK();
  window_index_kernel<<<1, 1, 0, ctx->stream>>>(win, cap, reset ? 1 : 0);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

}  // namespace cpg
