// Fused f / grad f evaluation (Eq. fA, Eq. Gn, Eq. Gamma) in three steps:
//
//   prep     x = base (+ stp d for a line-search trial), its FP32 copy for the
//            tensor-core MTTKRP, and the factor Grams A_m^T A_m (per-block
//            partial sums; the last block to finish adds them in a fixed order)
//   MTTKRP   per mode, split-K partial sums (tcgen05 / FP64 / sparse)
//   finish   per 32 gradient entries: M = sum of the partials (fixed order),
//            G = A Gammabar - M; <A^(N), M^(N)> and g . d as block partials;
//            the last block forms f = 1/2(||T||^2 - 2<T,A> + sum Gamma) and g . d.
//
// "Last block" reductions: each block writes its partial, fences, and bumps a
// per-stream counter; the block that sees the final count reads all partials
// in index order and resets the counter.  Results do not depend on timing.
#include <algorithm>

#include "cp_internal.cuh"

namespace cpg {

cp_status mttkrp_tc_parts(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* u32, const F32Off& o, int mode,
                          Parts* out);
cp_status mttkrp_f64_parts(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, int mode,
                           Parts* out);

namespace {

constexpr int kPrepRows = 16;

__device__ __forceinline__ bool last_block(unsigned* counter, unsigned nblocks, bool* flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *flag = atomicAdd(counter, 1u) == nblocks - 1;
  __syncthreads();
  if (*flag) __threadfence();
  return *flag;
}

struct PrepParams {
  Layout L;
  const double* base;
  const double* d;        // nullable: x = base + (*stp) d
  const double* stp;
  double* x;              // written when d != nullptr
  float* x32;             // nullable
  F32Off o32;
  double* part;           // [N][S][R*R]
  double* grams;          // out, N x R*R
  int S;
  unsigned* counter;
};

__global__ void __launch_bounds__(256) prep_kernel(const PrepParams p) {
  __shared__ double tile[kPrepRows * CP_MAX_R];
  __shared__ bool is_last;
  const int m = blockIdx.y;
  const int R = p.L.R;
  const int RR = R * R;
  const int64_t I = p.L.dims[m];
  const int64_t chunk = (I + p.S - 1) / p.S;
  const int64_t rb = (int64_t)blockIdx.x * chunk;
  const int64_t re = min(I, rb + chunk);
  const double a = p.d ? *p.stp : 0.0;
  const int64_t off = p.L.off[m];
  double acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  for (int64_t r0 = rb; r0 < re; r0 += kPrepRows) {
    const int nr = (int)min((int64_t)kPrepRows, re - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * R; e += blockDim.x) {
      const int64_t gi = off + r0 * R + e;
      double v = p.base[gi];
      if (p.d) {
        v = v + a * p.d[gi];
        p.x[gi] = v;
      }
      if (p.x32) p.x32[p.o32.off[m] + (r0 + e / R) * p.o32.rs + e % R] = (float)v;
      tile[e] = v;
    }
    if (p.x32)   // zero padding of the FP32 rows
      for (int e = threadIdx.x; e < nr * (p.o32.rs - R); e += blockDim.x) {
        const int q = e / (p.o32.rs - R);
        p.x32[p.o32.off[m] + (r0 + q) * p.o32.rs + R + (e - q * (p.o32.rs - R))] = 0.f;
      }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int e = threadIdx.x + k * blockDim.x;
      if (e < RR) {
        const int r = e / R, s = e - (e / R) * R;
        double t = acc[k];
        for (int q = 0; q < nr; ++q) t = fma(tile[q * R + r], tile[q * R + s], t);
        acc[k] = t;
      }
    }
  }
  double* out = p.part + ((int64_t)m * p.S + blockIdx.x) * RR;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int e = threadIdx.x + k * blockDim.x;
    if (e < RR) out[e] = acc[k];
  }
  if (!last_block(p.counter, gridDim.x * gridDim.y, &is_last)) return;
  for (int idx = threadIdx.x; idx < p.L.N * RR; idx += blockDim.x) {
    const int mm = idx / RR, e = idx - (idx / RR) * RR;
    double s = 0.0;
    for (int c = 0; c < p.S; ++c) s += __ldcg(&p.part[((int64_t)mm * p.S + c) * RR + e]);
    p.grams[idx] = s;
  }
  if (threadIdx.x == 0) *p.counter = 0u;
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
  double* blk;            // 2 x gridDim.x block partials
  unsigned* counter;
  int* status;
};

__global__ void __launch_bounds__(256) fg_finish_kernel(const FinishParams p) {
  __shared__ double Gb[CP_MAX_R * CP_MAX_R];
  __shared__ double sh[8][33];
  __shared__ double tr[2][256];
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
      const float* q = (const float*)pt.p;
      float sf = 0.f;
#pragma unroll 4
      for (int c = w; c < pt.count; c += 8) sf += __ldcg(&q[(int64_t)c * nel + e]);
      s = (double)sf;
    } else {
      const double* q = (const double*)pt.p;
#pragma unroll 4
      for (int c = w; c < pt.count; c += 8) s += __ldcg(&q[(int64_t)c * nel + e]);
    }
  }
  sh[w][lane] = s;
  __syncthreads();
  if (w == 0) {
    double inner = 0.0, gdv = 0.0;
    if (e < nel) {
      double mval = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) mval += sh[q][lane];
      const int64_t off = p.L.off[n];
      const int64_t i = e / R;
      const int r = (int)(e - i * R);
      const double* A = p.u + off + i * R;
      double v = 0.0;
      for (int t = 0; t < R; ++t) v = fma(A[t], Gb[t * R + r], v);
      const double gval = v - mval;
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
  tr[0][threadIdx.x] = a;
  tr[1][threadIdx.x] = b;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) {
      tr[0][threadIdx.x] += tr[0][threadIdx.x + st];
      tr[1][threadIdx.x] += tr[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  const double inner_sum = tr[0][0], gd_sum = tr[1][0];
  __syncthreads();
  tr[0][threadIdx.x] = gs;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) tr[0][threadIdx.x] += tr[0][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double fv = 0.5 * (p.norm2 - 2.0 * inner_sum + tr[0][0]);
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

cp_status fg_eval_ex(cp_ctx* ctx, const cp_tensor* t_in, const Layout& L, const double* base, const double* d,
                     const double* stp, double* x, double* f, double* g, cp_precision prec, double* gd,
                     double* grams_out) {
  cp_tensor* t = const_cast<cp_tensor*>(t_in);
  const int R = L.R, N = L.N, RR = R * R;
  const double* u = d ? x : base;
  const bool want_f32 = t->kind == 0 && prec == CP_MIXED_BF16X3;
  // prep: x, FP32 copy, Grams
  int64_t acc32 = 0;
  const F32Off o32 = f32_layout(L, &acc32);
  int64_t Imax = 1;
  for (int n = 0; n < N; ++n) Imax = std::max(Imax, L.dims[n]);
  const int S = (int)std::max<int64_t>(1, std::min<int64_t>((Imax + 15) / 16, 2 * (int64_t)ctx->num_sms));
  float* x32 = nullptr;
  double* grams = nullptr;
  double* gpart = nullptr;
  if (want_f32) CP_TRY(ws_alloc(ctx, (void**)&x32, sizeof(float) * (size_t)acc32 + 64));
  if (grams_out)
    grams = grams_out;
  else
    CP_TRY(ws_alloc(ctx, (void**)&grams, sizeof(double) * (size_t)N * RR));
  CP_TRY(ws_alloc(ctx, (void**)&gpart, sizeof(double) * (size_t)N * S * RR));
  PrepParams pp;
  pp.L = L;
  pp.base = base;
  pp.d = d;
  pp.stp = stp;
  pp.x = x;
  pp.x32 = x32;
  pp.o32 = o32;
  pp.part = gpart;
  pp.grams = grams;
  pp.S = S;
  pp.counter = ctx->d_counter;
  prep_kernel<<<dim3(S, N), 256, 0, ctx->stream>>>(pp);
  CP_LAUNCH_CHECK();
  // MTTKRPs (all modes for g; the last one alone for f)
  FinishParams fp{};
  const int first = g || d ? 0 : N - 1;
  for (int n = first; n < N; ++n) CP_TRY(mttkrp_parts(ctx, t, L, u, x32, o32, n, prec, &fp.parts[n]));
  // finish
  fp.L = L;
  int64_t chunks = 0;
  for (int n = 0; n < N; ++n) {
    fp.chunk_off[n] = chunks;
    if (n >= first) chunks += (L.dims[n] * R + 31) / 32;
  }
  fp.chunk_off[N] = chunks;
  // modes before `first` own no chunks: point their offsets past them
  fp.u = u;
  fp.grams = grams;
  fp.norm2 = t->norm2;
  fp.g = g;
  fp.f = f;
  fp.d = gd ? d : nullptr;   // g . d only when asked for
  fp.gd = gd;
  fp.counter = ctx->d_counter;
  fp.status = ctx->d_status;
  CP_TRY(ws_alloc(ctx, (void**)&fp.blk, sizeof(double) * 2 * (size_t)chunks + 16));
  fg_finish_kernel<<<(unsigned)chunks, 256, 0, ctx->stream>>>(fp);
  CP_LAUNCH_CHECK();
  ws_free(ctx, fp.blk);
  for (int n = first; n < N; ++n) ws_free(ctx, const_cast<void*>(fp.parts[n].p));
  ws_free(ctx, gpart);
  if (!grams_out) ws_free(ctx, grams);
  if (x32) ws_free(ctx, x32);
  return CP_OK;
}

}  // namespace cpg
