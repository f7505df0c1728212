// FP64 R x R algebra around the MTTKRP: factor Grams and their Hadamard
// products (Eq. Gamma), the ALS mode solve (Section 2.3, Eq. foopt), the
// objective/gradient assembly (Eq. fA, Eq. Gn) and the normalisation and
// reordering of rank-one terms (Section 2.3).
//
// FP64 throughput is low on this part, so every O(I R^2) step is spread over
// many CTAs (row chunks) and reduced in a fixed order (deterministic).
#include <algorithm>

#include "cp_internal.cuh"
#include "dev_linalg.cuh"

namespace cpg {

cp_status reduce_partials(cp_ctx* ctx, const double* partial, int nparts, int64_t n, double* out);

namespace {

constexpr int kGramRows = 16;   // rows staged per tile

// Partial Gram of rows [chunk) of mode m = mode_lo + blockIdx.y.
// part layout: [mode][S][R*R].
__global__ void gram_partial_kernel(FactorPtrs F, int mode_lo, int S, double* __restrict__ part) {
  __shared__ double tile[kGramRows * CP_MAX_R];
  const int m = mode_lo + blockIdx.y;
  const int R = F.R;
  const int64_t I = F.I[m];
  const int64_t chunk = (I + S - 1) / S;
  const int64_t rb = (int64_t)blockIdx.x * chunk;
  const int64_t re = min(I, rb + chunk);
  const int RR = R * R;
  double acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  const double* A = F.A[m];
  for (int64_t r0 = rb; r0 < re; r0 += kGramRows) {
    const int nr = (int)min((int64_t)kGramRows, re - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * R; e += blockDim.x) tile[e] = A[r0 * R + e];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int e = threadIdx.x + k * blockDim.x;
      if (e < RR) {
        const int r = e / R, s = e - (e / R) * R;
        double a = acc[k];
        for (int q = 0; q < nr; ++q) a = fma(tile[q * R + r], tile[q * R + s], a);
        acc[k] = a;
      }
    }
  }
  double* out = part + ((int64_t)blockIdx.y * S + blockIdx.x) * RR;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int e = threadIdx.x + k * blockDim.x;
    if (e < RR) out[e] = acc[k];
  }
}

// grams[(mode_lo + y) * RR + e] = sum_s part[y][s][e]
__global__ void gram_reduce_kernel(const double* __restrict__ part, int S, int RR, int nmodes,
                                   int mode_lo, double* __restrict__ grams) {
  const int total = nmodes * RR;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int y = idx / RR, e = idx - (idx / RR) * RR;
    double s = 0.0;
    for (int c = 0; c < S; ++c) s += part[((int64_t)y * S + c) * RR + e];
    grams[(int64_t)(mode_lo + y) * RR + e] = s;
  }
}

// Gammabar^(n) = Hadamard product of grams[m], m != n (n = -1: all modes).
__device__ void build_gamma(const double* __restrict__ grams, int N, int R, int n, double* S) {
  const int RR = R * R;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) v *= grams[(int64_t)m * RR + e];
    S[e] = v;
  }
}

// Factor Gammabar^(n) with one ridge retry; false if both attempts fail.
__device__ bool factor_gamma_bar(const double* grams, int N, int R, int n, double* S, int* flag) {
  build_gamma(grams, N, R, n, S);
  if (threadIdx.x == 0) *flag = 0;
  __syncthreads();
  if (chol_block(S, R, flag)) return true;
  __syncthreads();
  build_gamma(grams, N, R, n, S);
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int r = 0; r < R; ++r) tr += S[r * R + r];
    const double ridge = 1e-12 * tr / R;
    for (int r = 0; r < R; ++r) S[r * R + r] += ridge;
    *flag = 0;
  }
  __syncthreads();
  return chol_block(S, R, flag);
}

// A_n[rows] = M[rows] Gammabar^-1 via L L^T: one thread per row.
__global__ void als_solve_kernel(double* __restrict__ An, const double* __restrict__ M, int64_t I,
                                 const double* __restrict__ grams, int N, int R, int n, int S,
                                 int* status) {
  __shared__ double L[CP_MAX_R * CP_MAX_R];
  __shared__ int flag;
  if (!factor_gamma_bar(grams, N, R, n, L, &flag)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) record_status(status, CP_ERR_NOT_SPD);
    return;
  }
  const int64_t chunk = (I + S - 1) / S;
  const int64_t rb = (int64_t)blockIdx.x * chunk;
  const int64_t re = min(I, rb + chunk);
  for (int64_t i = rb + threadIdx.x; i < re; i += blockDim.x) {
    double y[CP_MAX_R];
    const double* m = M + i * R;
    for (int r = 0; r < R; ++r) {
      double v = m[r];
      for (int s = 0; s < r; ++s) v -= L[r * R + s] * y[s];
      y[r] = v / L[r * R + r];
    }
    for (int r = R - 1; r >= 0; --r) {
      double v = y[r];
      for (int s = r + 1; s < R; ++s) v -= L[s * R + r] * y[s];
      y[r] = v / L[r * R + r];
    }
    double* a = An + i * R;
    for (int r = 0; r < R; ++r) a[r] = y[r];
  }
}

// g^(n)[i, r] = -M^(n)[i, r] + sum_s A^(n)[i, s] Gammabar^(n)[s, r]
__global__ void grad_kernel(const double* __restrict__ A, const double* __restrict__ M,
                            double* __restrict__ g, int64_t I, const double* __restrict__ grams,
                            int N, int R, int n) {
  __shared__ double Gb[CP_MAX_R * CP_MAX_R];
  build_gamma(grams, N, R, n, Gb);
  __syncthreads();
  const int64_t total = I * R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / R;
    const int r = (int)(e - i * R);
    const double* a = A + i * R;
    double v = 0.0;
    for (int s = 0; s < R; ++s) v = fma(a[s], Gb[s * R + r], v);
    g[e] = v - M[e];
  }
}

// f = 1/2 (||T||^2 - 2 inner + sum Gamma).
__global__ void f_finalize_kernel(const double* __restrict__ grams, int N, int R, double norm2,
                                  const double* __restrict__ inner, double* __restrict__ f,
                                  int* status) {
  __shared__ double sh[256];
  const int RR = R * R;
  double acc = 0.0;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m) v *= grams[(int64_t)m * RR + e];
    acc += v;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = 0.5 * (norm2 - 2.0 * (*inner) + sh[0]);
    *f = v;
    if (!isfinite(v)) record_status(status, CP_ERR_NONFINITE);
  }
}

// Deterministic dot product, stage 1.
__global__ void dot_partial_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                   int64_t n, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[k], y[k], acc);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void dot_final_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) acc += part[k];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void axpy_scalar_kernel(int64_t n, const double* __restrict__ x0,
                                   const double* __restrict__ d, const double* __restrict__ stp,
                                   double* __restrict__ x) {
  const double a = *stp;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    x[k] = x0[k] + a * d[k];
}

__global__ void sub_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = a[k] - b[k];
}

// Column sums of squares, partial over row chunks: part[mode][S][R].
__global__ void colsq_partial_kernel(FactorPtrs F, int S, double* __restrict__ part) {
  const int m = blockIdx.y;
  const int R = F.R;
  const int64_t I = F.I[m];
  const int64_t chunk = (I + S - 1) / S;
  const int64_t rb = (int64_t)blockIdx.x * chunk;
  const int64_t re = min(I, rb + chunk);
  __shared__ double sh[256];
  // threads: r = tid % R, lane group = tid / R strides over rows
  const int groups = blockDim.x / R;
  const int r = threadIdx.x % R;
  const int gidx = threadIdx.x / R;
  double acc = 0.0;
  if (gidx < groups)
    for (int64_t i = rb + gidx; i < re; i += groups) {
      const double v = F.A[m][i * R + r];
      acc = fma(v, v, acc);
    }
  sh[threadIdx.x] = (gidx < groups) ? acc : 0.0;
  __syncthreads();
  if ((int)threadIdx.x < R) {
    double s = 0.0;
    for (int q = 0; q < groups; ++q) s += sh[q * R + threadIdx.x];
    part[((int64_t)m * S + blockIdx.x) * R + threadIdx.x] = s;
  }
}

// Scales and term order (Section 2.3): nu[n][r] = ||a_r^(n)||, lambda_r =
// prod_n nu, scale = lambda^(1/N) / nu; stable order by decreasing lambda.
// meta layout: scale[N*R] doubles followed by order[R] ints (as doubles).
__global__ void norm_finalize_kernel(const double* __restrict__ part, int S, int N, int R,
                                     double* __restrict__ scale, int* __restrict__ order,
                                     double* __restrict__ lambda_out, int* status) {
  __shared__ double lam[CP_MAX_R];
  __shared__ double key[CP_MAX_R];
  const int r = threadIdx.x;
  if (r < R) {
    double nu[CP_MAX_N];
    double l = 1.0;
    bool zero = false;
    for (int n = 0; n < N; ++n) {
      double s = 0.0;
      for (int c = 0; c < S; ++c) s += part[((int64_t)n * S + c) * R + r];
      nu[n] = sqrt(s);
      l *= nu[n];
      if (nu[n] == 0.0) zero = true;
    }
    if (zero) l = 0.0;
    const double root = pow(l, 1.0 / N);
    for (int n = 0; n < N; ++n) scale[n * R + r] = zero ? 1.0 : root / nu[n];
    lam[r] = l;
    key[r] = isnan(l) ? -INFINITY : l;
    if (!isfinite(l)) record_status(status, CP_ERR_NONFINITE);
  }
  __syncthreads();
  if (r < R) {
    int rank = 0;
    for (int s = 0; s < R; ++s)
      if (key[s] > key[r] || (key[s] == key[r] && s < r)) ++rank;
    order[rank] = r;
    if (lambda_out) lambda_out[rank] = lam[r];
  }
}

// dst[n][i][p] = src[n][i][order[p]] * scale[n][order[p]] (and g / scale).
__global__ void norm_apply_kernel(Layout L, const double* __restrict__ src, double* __restrict__ dst,
                                  const double* __restrict__ gsrc, double* __restrict__ gdst,
                                  const double* __restrict__ scale, const int* __restrict__ order) {
  const int64_t P = L.off[L.N];
  const int R = L.R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P;
       e += (int64_t)gridDim.x * blockDim.x) {
    int n = 0;
    while (n + 1 < L.N && e >= L.off[n + 1]) ++n;
    const int64_t within = e - L.off[n];
    const int64_t i = within / R;
    const int p = (int)(within - i * R);
    const int q = order[p];
    const int64_t srcidx = L.off[n] + i * R + q;
    const double s = scale[n * R + q];
    dst[e] = src[srcidx] * s;
    if (gdst) gdst[e] = gsrc[srcidx] / s;
  }
}

inline int grid_for(cp_ctx* ctx, int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  b = std::min<int64_t>(b, 8 * (int64_t)ctx->num_sms);
  return (int)std::max<int64_t>(b, 1);
}

// Row chunks for an O(I R^2) step: about 16 rows per CTA, at most 2 x SMs CTAs.
inline int chunks_for(cp_ctx* ctx, int64_t I) {
  int64_t s = (I + 15) / 16;
  s = std::min<int64_t>(s, 2 * (int64_t)ctx->num_sms);
  return (int)std::max<int64_t>(s, 1);
}

}  // namespace

cp_status grams_modes(cp_ctx* ctx, const Layout& L, const double* u, int mode_lo, int nmodes,
                      double* grams) {
  const FactorPtrs F = factor_ptrs(L, u);
  int64_t Imax = 1;
  for (int m = mode_lo; m < mode_lo + nmodes; ++m) Imax = std::max(Imax, L.dims[m]);
  const int S = chunks_for(ctx, Imax);
  const int RR = L.R * L.R;
  double* part = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&part, sizeof(double) * (size_t)nmodes * S * RR));
  gram_partial_kernel<<<dim3(S, nmodes), 256, 0, ctx->stream>>>(F, mode_lo, S, part);
  CP_LAUNCH_CHECK();
  gram_reduce_kernel<<<grid_for(ctx, (int64_t)nmodes * RR, 256), 256, 0, ctx->stream>>>(
      part, S, RR, nmodes, mode_lo, grams);
  CP_LAUNCH_CHECK();
  ws_free(ctx, part);
  return CP_OK;
}

cp_status grams_all(cp_ctx* ctx, const Layout& L, const double* u, double* grams) {
  return grams_modes(ctx, L, u, 0, L.N, grams);
}

cp_status als_mode_solve(cp_ctx* ctx, const Layout& L, double* u, int mode, const double* M,
                         double* grams) {
  const int64_t I = L.dims[mode];
  const int S = chunks_for(ctx, I);
  als_solve_kernel<<<S, 128, 0, ctx->stream>>>(u + L.off[mode], M, I, grams, L.N, L.R, mode, S,
                                               ctx->d_status);
  CP_LAUNCH_CHECK();
  return grams_modes(ctx, L, u, mode, 1, grams);
}

cp_status dot(cp_ctx* ctx, int64_t n, const double* x, const double* y, double* out) {
  const int threads = 256;
  int nb = (int)std::min<int64_t>((n + threads - 1) / threads, 2 * ctx->num_sms);
  if (nb < 1) nb = 1;
  double* part = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&part, sizeof(double) * nb));
  dot_partial_kernel<<<nb, threads, 0, ctx->stream>>>(x, y, n, part);
  CP_LAUNCH_CHECK();
  dot_final_kernel<<<1, 256, 0, ctx->stream>>>(part, nb, out);
  CP_LAUNCH_CHECK();
  ws_free(ctx, part);
  return CP_OK;
}

cp_status fg_assemble(cp_ctx* ctx, const Layout& L, const double* u, const double* M_all,
                      const double* grams, double norm2, double* f, double* g) {
  if (g) {
    for (int n = 0; n < L.N; ++n) {
      const int64_t I = L.dims[n];
      grad_kernel<<<grid_for(ctx, I * L.R, 256), 256, 0, ctx->stream>>>(
          u + L.off[n], M_all + L.off[n], g + L.off[n], I, grams, L.N, L.R, n);
      CP_LAUNCH_CHECK();
    }
  }
  double* inner = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&inner, sizeof(double)));
  const int last = L.N - 1;
  CP_TRY(dot(ctx, L.dims[last] * L.R, u + L.off[last], M_all + L.off[last], inner));
  f_finalize_kernel<<<1, 256, 0, ctx->stream>>>(grams, L.N, L.R, norm2, inner, f, ctx->d_status);
  CP_LAUNCH_CHECK();
  ws_free(ctx, inner);
  return CP_OK;
}

cp_status normalize_into(cp_ctx* ctx, const Layout& L, const double* src, double* dst,
                         const double* gsrc, double* gdst, double* lambda) {
  const FactorPtrs F = factor_ptrs(L, src);
  int64_t Imax = 1;
  for (int m = 0; m < L.N; ++m) Imax = std::max(Imax, L.dims[m]);
  const int S = chunks_for(ctx, Imax);
  const int R = L.R;
  double* part = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&part, sizeof(double) * ((size_t)L.N * S * R + (size_t)L.N * R + R)));
  double* scale = part + (size_t)L.N * S * R;
  int* order = (int*)(scale + (size_t)L.N * R);
  const int threads = std::max(32, (256 / R) * R);
  colsq_partial_kernel<<<dim3(S, L.N), threads, 0, ctx->stream>>>(F, S, part);
  CP_LAUNCH_CHECK();
  norm_finalize_kernel<<<1, 64, 0, ctx->stream>>>(part, S, L.N, R, scale, order, lambda,
                                                  ctx->d_status);
  CP_LAUNCH_CHECK();
  norm_apply_kernel<<<grid_for(ctx, L.P(), 256), 256, 0, ctx->stream>>>(L, src, dst, gsrc, gdst,
                                                                        scale, order);
  CP_LAUNCH_CHECK();
  ws_free(ctx, part);
  return CP_OK;
}

cp_status axpy_scalar(cp_ctx* ctx, int64_t n, const double* x0, const double* d, const double* stp,
                      double* x) {
  axpy_scalar_kernel<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(n, x0, d, stp, x);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

cp_status sub_vec(cp_ctx* ctx, int64_t n, const double* a, const double* b, double* out) {
  sub_kernel<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(n, a, b, out);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

cp_status mttkrp_any(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, int mode,
                     double* out, cp_precision prec) {
  if (t->kind == 1) return mttkrp_sparse(ctx, t, L, u, mode, out, prec);
  if (prec == CP_MIXED_BF16X3)
    return mttkrp_dense_mixed(ctx, const_cast<cp_tensor*>(t), L, u, mode, out);
  return mttkrp_dense_f64(ctx, t, L, u, mode, out);
}

cp_status fg_eval(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, double* f,
                  double* g, cp_precision prec) {
  // prep (Grams, FP32 copy) -> MTTKRP partial sums -> fused finish
  return fg_eval_ex(ctx, t, L, u, nullptr, nullptr, nullptr, f, g, prec, nullptr, nullptr,
                    cudaGraphConditionalHandle{}, 0);
}

}  // namespace cpg
