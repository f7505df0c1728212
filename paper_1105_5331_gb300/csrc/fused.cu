// Fused f / grad f evaluation (Eq. fA, Eq. Gn, Eq. Gamma) in three steps:
//
//   prep     x = base (+ stp d for a point on a search line) and its FP32
//            copy for the tensor-core MTTKRP (unless one is given); the
//            factor Grams on the aux stream beside the MTTKRPs (unless given,
//            or formed from a line search's Grams), and the inverse of
//            Gammabar^(1) when asked for
//   MTTKRP   per mode whose M is not supplied, split-K partial sums
//            (tcgen05 / FP64 / sparse)
//   finish   per 32 gradient entries: M = the sum of the partials in a fixed
//            order (or the supplied M, or sum_v beta^popc(v) M_v from a line
//            search's Khatri-Rao variants), G = A Gammabar - M;
//            <A^(N), M^(N)> and g . d as block partials; the last block forms
//            f = 1/2(||T||^2 - 2<T,A> + sum Gamma) and g . d.
//
// "Last block" reductions: each block writes its partial, fences, and bumps a
// per-stream counter; the block that sees the final count reads all partials
// in index order and resets the counter.  Results do not depend on timing.
#include <algorithm>

#include "cp_internal.cuh"
#include "reduce.cuh"

namespace cpg {

cp_status mttkrp_tc_parts(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* u32, const F32Off& o, int mode,
                          Parts* out);
cp_status mttkrp_f64_parts(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, int mode,
                           Parts* out);

namespace {

__device__ __forceinline__ bool last_block(unsigned* counter, unsigned nblocks, bool* flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *flag = atomicAdd(counter, 1u) == nblocks - 1;
  __syncthreads();
  if (*flag) __threadfence();
  return *flag;
}

// x = base + (*stp) d (written when d is given) and its padded FP32 copy
// (when x32 is given), one pass over the FP32 layout.
__global__ void __launch_bounds__(256) xprep_kernel(Layout L, const double* __restrict__ base,
                                                    const double* __restrict__ d, const double* __restrict__ stp,
                                                    double* __restrict__ x, float* __restrict__ x32, F32Off o,
                                                    int64_t total) {
  CP_PDL_ENTRY();
  const double a = d ? *stp : 0.0;
  const int R = L.R;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int n = 0;
    while (n + 1 < L.N && q >= o.off[n + 1]) ++n;
    const int64_t within = q - o.off[n];
    const int64_t i = within / o.rs;
    const int r = (int)(within - i * o.rs);
    float v32 = 0.f;
    if (r < R) {
      const int64_t e = L.off[n] + i * R + r;
      double v = base[e];
      if (d) {
        v = fma(a, d[e], v);
        x[e] = v;
      }
      v32 = (float)v;
    }
    if (x32) x32[q] = v32;
  }
}

// Grams of x = base + beta d from those of base and d (per mode: base^T base,
// base^T d, d^T d):  X^T X = B^T B + beta (B^T D + D^T B) + beta^2 D^T D.
__global__ void grams_from_ls_kernel(int N, int R, const double* __restrict__ ls, const double* __restrict__ stp,
                                     double* __restrict__ out) {
  CP_PDL_ENTRY();
  const double b = *stp;
  const int RR = R * R;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * RR; e += gridDim.x * blockDim.x) {
    const int n = e / RR, k = e - n * RR;
    const int r = k / R, s = k - r * R;
    const double* ad = ls + (int64_t)(N + n) * RR;
    const double cross = ad[r * R + s] + ad[s * R + r];
    out[e] = fma(b, fma(b, ls[(int64_t)(2 * N + n) * RR + k], cross), ls[(int64_t)n * RR + k]);
  }
}

struct FinishParams {
  Layout L;
  Parts parts[CP_MAX_N];
  int64_t chunk_off[CP_MAX_N + 1];   // prefix of 32-entry chunks per mode
  const double* u;
  const double* grams;
  double norm2;
  double* g;              // nullable
  double* f;
  const double* d;        // nullable: also g . d
  double* gd;
  double* m0_out;         // nullable: M^(1) (mode 0) of the evaluation point
  // per mode, nullable: M given (mv_nvar = 1) or from the line-search
  // variants, M = sum_v beta^popc(v) mv[n][v I_n R + .] (x = base + beta d
  // is multilinear in beta)
  const double* mv[CP_MAX_N];
  int mv_nvar;
  const double* mv_beta;
  double* blk;            // 2 x gridDim.x block partials
  unsigned* counter;
  int* status;
};

__global__ void __launch_bounds__(256) fg_finish_kernel(const FinishParams p) {
  CP_PDL_ENTRY();
  __shared__ double Gb[CP_MAX_R * CP_MAX_R];
  __shared__ double sh[8][33];
  __shared__ double tr[3][8];
  __shared__ bool is_last;
  const int R = p.L.R, N = p.L.N, RR = R * R;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t chunk = blockIdx.x;
  int n = 0;
  while (n + 1 < N && chunk >= p.chunk_off[n + 1]) ++n;
  const int64_t nel = p.L.dims[n] * R;
  const int64_t e = (chunk - p.chunk_off[n]) * 32 + lane;
  for (int k = threadIdx.x; k < RR; k += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != n) v *= p.grams[(int64_t)m * RR + k];
    Gb[k] = v;
  }
  const Parts pt = p.parts[n];
  double s = 0.0;
  if (e < nel) {
    if (pt.f32) {
      // FP32 partial sums of the mixed MTTKRP are added in FP32
      s = (double)strided_sum((const float*)pt.p + e, w, pt.count, 8, nel);
    } else {
      s = strided_sum((const double*)pt.p + e, w, pt.count, 8, nel);
    }
  }
  sh[w][lane] = s;
  __syncthreads();
  if (w == 0) {
    double inner = 0.0, gdv = 0.0;
    if (e < nel) {
      double mval = 0.0;
      const double* mv = p.mv[n];
      if (mv && p.mv_nvar == 1) {
        mval = mv[e];
      } else if (mv) {
        const double beta = *p.mv_beta;
        double pw[CP_MAX_N];
        pw[0] = 1.0;
        for (int k = 1; k < N; ++k) pw[k] = pw[k - 1] * beta;
        for (int v = 0; v < p.mv_nvar; ++v) mval = fma(pw[__popc(v)], mv[(int64_t)v * nel + e], mval);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) mval += sh[q][lane];
      }
      if (p.m0_out && n == 0) p.m0_out[e] = mval;
      const int64_t off = p.L.off[n];
      const int64_t i = e / R;
      const int r = (int)(e - i * R);
      const double* A = p.u + off + i * R;
      // (A Gammabar)[i][r] in four interleaved chains (FP64 FMA latency)
      double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
      int t = 0;
      for (; t + 3 < R; t += 4) {
        v0 = fma(A[t], Gb[t * R + r], v0);
        v1 = fma(A[t + 1], Gb[(t + 1) * R + r], v1);
        v2 = fma(A[t + 2], Gb[(t + 2) * R + r], v2);
        v3 = fma(A[t + 3], Gb[(t + 3) * R + r], v3);
      }
      for (; t < R; ++t) v0 = fma(A[t], Gb[t * R + r], v0);
      const double gval = ((v0 + v1) + (v2 + v3)) - mval;
      if (p.g) p.g[off + e] = gval;
      if (n == N - 1) inner = p.u[off + e] * mval;
      if (p.d) gdv = gval * p.d[off + e];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      inner += __shfl_xor_sync(0xffffffffu, inner, o);
      gdv += __shfl_xor_sync(0xffffffffu, gdv, o);
    }
    if (lane == 0) {
      p.blk[blockIdx.x] = inner;
      p.blk[gridDim.x + blockIdx.x] = gdv;
    }
  }
  if (!last_block(p.counter, gridDim.x, &is_last)) return;
  double a = 0.0, b = 0.0, gs = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    a += __ldcg(&p.blk[k]);
    b += __ldcg(&p.blk[gridDim.x + k]);
  }
  for (int k = threadIdx.x; k < RR; k += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < N; ++m) v *= p.grams[(int64_t)m * RR + k];
    gs += v;
  }
  // the three sums: warp shuffles, then the eight warp sums in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    gs += __shfl_xor_sync(0xffffffffu, gs, o);
  }
  if (lane == 0) {
    tr[0][w] = a;
    tr[1][w] = b;
    tr[2][w] = gs;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double inner_sum = 0.0, gd_sum = 0.0, gsum = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      inner_sum += tr[0][q];
      gd_sum += tr[1][q];
      gsum += tr[2][q];
    }
    const double fv = 0.5 * (p.norm2 - 2.0 * inner_sum + gsum);
    *p.f = fv;
    if (!isfinite(fv)) record_status(p.status, CP_ERR_NONFINITE);
    if (p.d && p.gd) *p.gd = gd_sum;
    *p.counter = 0u;
  }
}

}  // namespace

cp_status mttkrp_parts(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u, const float* u32,
                       const F32Off& o32, int mode, cp_precision prec, Parts* out) {
  if (t->kind == 1) {
    double* M = nullptr;
    CP_TRY(ws_alloc(ctx, (void**)&M, sizeof(double) * (size_t)L.dims[mode] * L.R));
    CP_TRY(mttkrp_sparse(ctx, t, L, u, mode, M, prec));
    *out = Parts{M, 1, 0};
    return CP_OK;
  }
  if (prec == CP_MIXED_BF16X3) return mttkrp_tc_parts(ctx, t, L, u32, o32, mode, out);
  return mttkrp_f64_parts(ctx, t, L, u, mode, out);
}

// The MTTKRPs of several modes, one launch per mode.  (One tensor-core
// launch shared among the modes streams T faster when timed alone, but in
// the solve's stream of launches the next MTTKRP's CTAs already start on each
// SM as the previous one's finish, programmatic dependent launch overlapping
// their start-up, and the shared launch measured slower per iteration.)
static cp_status mttkrp_parts_multi(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u, const float* u32,
                                    const F32Off& o32, const int* modes, int nmodes, cp_precision prec, Parts* out) {
  if (ctx->dimtree && t->kind == 0 && t->N == 3 && prec == CP_MIXED_BF16X3 && u32 && nmodes == 2 && modes[0] == 0 &&
      modes[1] == 1) {
    // M^(1) and M^(2) from one pass: W = T x_3 A^(3), then one contraction each
    Parts W;
    CP_TRY(dimtree_w(ctx, t, L, u32, o32, 2, &W));
    for (int k = 0; k < 2; ++k) {
      double* M = nullptr;
      CP_TRY(ws_alloc(ctx, (void**)&M, sizeof(double) * (size_t)L.dims[k] * L.R));
      CP_TRY(dimtree_contract(ctx, t, L, W, 2, k, u32, o32, M));
      out[k] = Parts{M, 1, 0};
    }
    ws_free(ctx, const_cast<void*>(W.p));
    return CP_OK;
  }
  for (int k = 0; k < nmodes; ++k) CP_TRY(mttkrp_parts(ctx, t, L, u, u32, o32, modes[k], prec, &out[k]));
  return CP_OK;
}

cp_status fg_eval_ex(cp_ctx* ctx, const cp_tensor* t_in, const Layout& L, const double* base, const double* d,
                     const double* stp, double* x, double* f, double* g, cp_precision prec, double* gd,
                     double* grams_out, double* m0_out, const MGiven* mg, const double* grams_in,
                     double* xi0_out, const double* grams_ls, const float* x32_in) {
  cp_tensor* t = const_cast<cp_tensor*>(t_in);
  const int R = L.R, N = L.N, RR = R * R;
  const double* u = d ? x : base;
  // MTTKRPs (all modes for g; the last one alone for f), less those supplied
  const int first = g || d ? 0 : N - 1;
  int modes[CP_MAX_N], nm = 0;
  for (int n = first; n < N; ++n)
    if (!(mg && mg->m[n])) modes[nm++] = n;
  const bool want_f32 = t->kind == 0 && prec == CP_MIXED_BF16X3 && nm > 0;
  // x and its FP32 copy on the main stream; the Grams of x on the aux
  // stream, overlapped with the MTTKRPs (which do not need them)
  int64_t acc32 = 0;
  const F32Off o32 = f32_layout(L, &acc32);
  float* x32 = nullptr;
  double* grams = nullptr;
  const bool own32 = want_f32 && !(x32_in && !d);
  if (want_f32 && !own32) x32 = const_cast<float*>(x32_in);
  if (own32) CP_TRY(ws_alloc(ctx, (void**)&x32, sizeof(float) * (size_t)acc32 + 64));
  if (grams_in)
    grams = const_cast<double*>(grams_in);
  else if (grams_out)
    grams = grams_out;
  else
    CP_TRY(ws_alloc(ctx, (void**)&grams, sizeof(double) * (size_t)N * RR));
  // the Grams of x from a line search's Grams (main stream), else from the
  // factors (aux stream, overlapped with the MTTKRPs)
  const bool grams_on_aux = !grams_in && !(grams_ls && d);
  if (!grams_in && !grams_on_aux) {
    (void)launch_pdl(grams_from_ls_kernel, dim3((unsigned)((N * RR + 255) / 256)), dim3(256), 0, ctx->stream, N, R,
                     grams_ls, stp, grams);
    CP_LAUNCH_CHECK();
  }
  CP_CUDA(cudaEventRecord(ctx->ev_fork, ctx->stream));
  CP_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
  if (grams_on_aux) {
    GramJob jobs[kMaxGramJobs];
    for (int n = 0; n < N; ++n) {
      jobs[n] = GramJob{base + L.off[n], base + L.off[n], L.dims[n], grams + (size_t)n * RR, 1};
      if (d) {
        jobs[n].D = d + L.off[n];
        jobs[n].stp = stp;
      }
    }
    CP_TRY(grams_jobs(ctx, ctx->aux, ctx->d_counter + 1, R, jobs, N));
  }
  if (xi0_out) CP_TRY(gram_inverse_launch(ctx, ctx->aux, grams, L, 0, xi0_out));
  CP_CUDA(cudaEventRecord(ctx->ev_join, ctx->aux));
  if (d || own32) {
    float* w32 = own32 ? x32 : nullptr;
    const int64_t total = w32 ? acc32 : L.P();
    const F32Off o = w32 ? o32 : [&]() { F32Off q{}; q.rs = R; for (int n = 0; n < N; ++n) q.off[n] = L.off[n]; return q; }();
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4 * ctx->num_sms));
    (void)launch_pdl(xprep_kernel, dim3(blocks), dim3(256), 0, ctx->stream, L, base, d, stp, x, w32, o, total);
    CP_LAUNCH_CHECK();
  }
  FinishParams fp{};
  {
    Parts pm[CP_MAX_N];
    CP_TRY(mttkrp_parts_multi(ctx, t, L, u, x32, o32, modes, nm, prec, pm));
    for (int k = 0; k < nm; ++k) fp.parts[modes[k]] = pm[k];
  }
  // finish
  fp.L = L;
  int64_t chunks = 0;
  for (int n = 0; n < N; ++n) {
    fp.chunk_off[n] = chunks;
    if (n >= first) chunks += (L.dims[n] * R + 31) / 32;
  }
  fp.chunk_off[N] = chunks;
  fp.u = u;
  fp.grams = grams;
  fp.norm2 = t->norm2;
  fp.g = g;
  fp.f = f;
  fp.d = gd ? d : nullptr;   // g . d only when asked for
  fp.gd = gd;
  fp.m0_out = m0_out;
  if (mg) {
    for (int n = 0; n < N; ++n) fp.mv[n] = mg->m[n];
    fp.mv_nvar = mg->nvar;
    fp.mv_beta = mg->beta;
  } else {
    fp.mv_nvar = 1;
  }
  fp.counter = ctx->d_counter;
  fp.status = ctx->d_status;
  CP_TRY(ws_alloc(ctx, (void**)&fp.blk, sizeof(double) * 2 * (size_t)chunks + 16));
  // the finish needs the Grams; the inverse alone may run on beside it
  if (grams_on_aux) CP_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  (void)launch_pdl(fg_finish_kernel, dim3((unsigned)chunks), dim3(256), 0, ctx->stream, fp);
  CP_LAUNCH_CHECK();
  if (!grams_on_aux) CP_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  ws_free(ctx, fp.blk);
  for (int k = 0; k < nm; ++k) ws_free(ctx, const_cast<void*>(fp.parts[modes[k]].p));
  if (!grams_out && !grams_in) ws_free(ctx, grams);
  if (own32) ws_free(ctx, x32);
  return CP_OK;
}

}  // namespace cpg
