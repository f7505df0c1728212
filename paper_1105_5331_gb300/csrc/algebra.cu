// Vector kernels of the solve (dot products, axpy, differences) and the
// normalisation and reordering of rank-one terms (Section 2.3).
//
// FP64 throughput is low on this part, so every O(I R) step is spread over
// many CTAs and reduced in a fixed order (deterministic).
#include <algorithm>

#include "cp_internal.cuh"
#include "norm_dev.cuh"

namespace cpg {

cp_status reduce_partials(cp_ctx* ctx, const double* partial, int nparts, int64_t n, double* out);

namespace {

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
  CP_PDL_ENTRY();
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

// Normalisation and term order (Section 2.3): nu[n][r] = ||a_r^(n)||,
// lambda_r = prod_n nu, scale = lambda^(1/N) / nu, stable order by decreasing
// lambda; then dst[n][i][p] = src[n][i][order[p]] * scale[n][order[p]] (and
// g / scale).  Every block derives the R scales itself (a few FP64 ops per
// rank) from the column sums of squares: the diagonals of the factor Grams
// when they are known, else the colsq partials (S per mode and rank).
__global__ void __launch_bounds__(256) norm_apply_kernel(Layout L, const double* __restrict__ src,
                                                         double* __restrict__ dst, const double* __restrict__ gsrc,
                                                         double* __restrict__ gdst, const double* __restrict__ part,
                                                         int S, const double* __restrict__ grams,
                                                         double* __restrict__ lambda_out, int* status,
                                                         const double* __restrict__ m0_src,
                                                         double* __restrict__ m0_dst,
                                                         double* __restrict__ grams_out,
                                                         const double* __restrict__ xi_src,
                                                         double* __restrict__ xi_dst,
                                                         const double* __restrict__ ml_src,
                                                         double* __restrict__ ml_dst, float* __restrict__ dst32,
                                                         F32Off o32) {
  CP_PDL_ENTRY();
  __shared__ NormShared sh;
  norm_prologue(L, part, S, grams, lambda_out, status, sh);
  const double* scale = sh.scale;
  const int* order = sh.order;
  const int N = L.N, R = L.R;
  const int64_t P = L.off[L.N];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P;
       e += (int64_t)gridDim.x * blockDim.x) {
    int n = 0;
    while (n + 1 < L.N && e >= L.off[n + 1]) ++n;
    const int64_t within = e - L.off[n];
    const int64_t i = within / R;
    const int p = (int)(within - i * R);
    const int q = order[p];
    const int64_t srcidx = L.off[n] + i * R + q;
    const double sc = scale[n * R + q];
    const double v = src[srcidx] * sc;
    dst[e] = v;
    if (dst32) dst32[o32.off[n] + i * o32.rs + p] = (float)v;
    if (gdst) gdst[e] = gsrc[srcidx] / sc;
  }
  if (m0_dst) {
    // M^(1)[i][p] of the normalised point: column order[p] of src's M^(1)
    // times the scales of modes 2..N of that column
    const int64_t n0 = L.dims[0] * R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n0; e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = e / R;
      const int pcol = (int)(e - i * R);
      const int q = order[pcol];
      double sc = 1.0;
      for (int n = 1; n < N; ++n) sc *= scale[n * R + q];
      m0_dst[e] = m0_src[i * R + q] * sc;
    }
  }
  if (ml_dst) {
    // M^(N) likewise, with the scales of modes 1..N-1
    const int64_t nl = L.dims[N - 1] * R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl; e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = e / R;
      const int pcol = (int)(e - i * R);
      const int q = order[pcol];
      double sc = 1.0;
      for (int n = 0; n + 1 < N; ++n) sc *= scale[n * R + q];
      ml_dst[e] = ml_src[i * R + q] * sc;
    }
  }
  if (blockIdx.x == 0 && grams_out) {
    // Grams of dst: G'[n][p][q] = G[n][o_p][o_q] s_n[o_p] s_n[o_q]
    for (int e = threadIdx.x; e < N * R * R; e += blockDim.x) {
      const int n = e / (R * R), pq = e - n * R * R;
      const int pr = pq / R, qr = pq - (pq / R) * R;
      const int op = order[pr], oq = order[qr];
      grams_out[e] = grams[(int64_t)n * R * R + op * R + oq] * scale[n * R + op] * scale[n * R + oq];
    }
  }
  if (blockIdx.x == 0 && xi_dst) {
    // inverse of Gammabar^(1) of dst: Xi'[p][q] = Xi[o_p][o_q] / (S[o_p] S[o_q]),
    // S[r] = prod_{n >= 2} s_n[r]; the ok flag follows
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
      const int pr = e / R, qr = e - (e / R) * R;
      const int op = order[pr], oq = order[qr];
      double sp = 1.0, sq = 1.0;
      for (int n = 1; n < N; ++n) {
        sp *= scale[n * R + op];
        sq *= scale[n * R + oq];
      }
      xi_dst[e] = xi_src[op * R + oq] / (sp * sq);
    }
    if (threadIdx.x == 0) *(int*)(xi_dst + R * R) = *(const int*)(xi_src + R * R);
  }
}

// w = the iterate whose factor m is d's when m != mode and bit j(m) of v is
// set (j(m): m's index among the modes other than `mode`), else u's.
__global__ void mix_for_mode_kernel(Layout L, const double* __restrict__ u, const double* __restrict__ d, int mode,
                                    int v, double* __restrict__ w) {
  CP_PDL_ENTRY();
  const int64_t P = L.off[L.N];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
    int n = 0;
    while (n + 1 < L.N && e >= L.off[n + 1]) ++n;
    const int j = n < mode ? n : n - 1;
    w[e] = (n != mode && ((v >> j) & 1)) ? d[e] : u[e];
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

cp_status normalize_into(cp_ctx* ctx, const Layout& L, const double* src, double* dst,
                         const double* gsrc, double* gdst, double* lambda, const double* grams,
                         const double* m0_src, double* m0_dst, double* grams_out, const double* xi_src,
                         double* xi_dst, const double* ml_src, double* ml_dst, float* dst32) {
  const int R = L.R;
  double* part = nullptr;
  int S = 1;
  if (!grams) {
    const FactorPtrs F = factor_ptrs(L, src);
    int64_t Imax = 1;
    for (int m = 0; m < L.N; ++m) Imax = std::max(Imax, L.dims[m]);
    S = chunks_for(ctx, Imax);
    CP_TRY(ws_alloc(ctx, (void**)&part, sizeof(double) * (size_t)L.N * S * R));
    const int threads = std::max(32, (256 / R) * R);
    (void)launch_pdl(colsq_partial_kernel, dim3(dim3(S, L.N)), dim3(threads), 0, ctx->stream, F, S, part);
    CP_LAUNCH_CHECK();
  }
  (void)launch_pdl(norm_apply_kernel, dim3(grid_for(ctx, L.P(), 256)), dim3(256), 0, ctx->stream, L, src, dst, gsrc, gdst, part, S, grams,
                                                                        lambda, ctx->d_status, m0_src, m0_dst,
                                                                        grams ? grams_out : nullptr, xi_src, xi_dst,
                                                                        ml_src, ml_dst, dst32, [&]() { int64_t a; return f32_layout(L, &a); }());
  CP_LAUNCH_CHECK();
  if (part) ws_free(ctx, part);
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

cp_status mttkrp_variants_any(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, const double* d,
                              const int* modes, int nmodes, double* out, cp_precision prec) {
  if (t->kind == 0 && prec == CP_MIXED_BF16X3 && tc_variants_supported(L))
    return mttkrp_dense_mixed_variants(ctx, const_cast<cp_tensor*>(t), L, u, d, modes, nmodes, out);
  // one MTTKRP per variant, of the mixed iterate
  const int nvar = 1 << (L.N - 1);
  double* w = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&w, sizeof(double) * (size_t)L.P()));
  size_t off = 0;
  for (int k = 0; k < nmodes; ++k) {
    const int mode = modes[k];
    for (int v = 0; v < nvar; ++v) {
      (void)launch_pdl(mix_for_mode_kernel, dim3(grid_for(ctx, L.P(), 256)), dim3(256), 0, ctx->stream, L, u, d,
                       mode, v, w);
      CP_LAUNCH_CHECK();
      CP_TRY(mttkrp_any(ctx, t, L, w, mode, out + off, prec));
      off += (size_t)L.dims[mode] * L.R;
    }
  }
  ws_free(ctx, w);
  return CP_OK;
}

cp_status fg_eval(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, double* f,
                  double* g, cp_precision prec) {
  // prep (Grams, FP32 copy) -> MTTKRP partial sums -> fused finish
  return fg_eval_ex(ctx, t, L, u, nullptr, nullptr, nullptr, f, g, prec, nullptr);
}

}  // namespace cpg
