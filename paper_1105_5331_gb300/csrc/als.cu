// ALS sweep (Section 2.3, Eq. foopt) and factor Grams, laid out for a GPU
// whose FP64 units are scarce: a dependent FP64 FMA costs ~64 clocks and a
// divide or square root ~650 on sm_103a, so no kernel here runs a long
// serial FP64 chain and no single block reduces a large FP64 sum.
//
//   Grams       one warp per (Gram, entry): lanes stride the rows, a
//               butterfly shuffle adds the lane sums; no cross-block
//               reduction unless a factor is taller than one row chunk.
//   inverse     Gammabar^(n) = Hadamard product of the other modes' Grams,
//               inverted by symmetric Gauss-Jordan elimination (no pivoting,
//               which is stable for SPD matrices and fails exactly when a
//               Cholesky factorisation would), one ridge retry; pivot
//               reciprocals by Newton's iteration from an FP32 seed.  It runs
//               on the context's aux stream, overlapped with the MTTKRP of
//               the same mode, which does not depend on it; one barrier per
//               pivot (double-buffered), the thread that forms the next
//               diagonal entry forming its reciprocal at once (look-ahead).
//   update      A_n = M Gammabar^-1: rows spread over blocks; M rows from the
//               MTTKRP partial sums (FP32 partials added in FP32, FP64 ones in
//               FP64, in a fixed order), then one FP64 dot per output; the
//               last mode's M can be kept (it is M^(N) of the swept point).
#include <algorithm>

#include "cp_internal.cuh"
#include "newton.cuh"
#include "reduce.cuh"

namespace cpg {

cp_status mttkrp_parts(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u, const float* u32,
                       const F32Off& o32, int mode, cp_precision prec, Parts* out);

namespace {

constexpr int kGramChunk = 4096;      // rows per warp item before the row range is split

struct GramParams {
  GramJob job[kMaxGramJobs];
  int64_t item_off[kMaxGramJobs + 1];  // prefix of (entries x chunks) per job
  int njobs;
  int R;
  double* partial;                     // [items] when any job is chunked
  int chunked;
  unsigned* counter;
};

__device__ __forceinline__ void upper_pair(int e, int R, int* r, int* s) {
  // e enumerates (r, s), r <= s, row by row
  int rr = 0, base = 0;
  while (e >= base + (R - rr)) {
    base += R - rr;
    ++rr;
  }
  *r = rr;
  *s = rr + (e - base);
}

__device__ __forceinline__ void job_entry(const GramParams& p, int64_t item, int* j, int* r, int* s, int64_t* chunk) {
  int jj = 0;
  while (jj + 1 < p.njobs && item >= p.item_off[jj + 1]) ++jj;
  const GramJob& g = p.job[jj];
  const int64_t nch = (g.I + kGramChunk - 1) / kGramChunk;
  const int64_t local = item - p.item_off[jj];
  const int64_t e = local / (nch > 0 ? nch : 1);
  *chunk = local - e * (nch > 0 ? nch : 1);
  if (g.sym) {
    upper_pair((int)e, p.R, r, s);
  } else {
    *r = (int)(e / p.R);
    *s = (int)(e - (e / p.R) * p.R);
  }
  *j = jj;
}

__global__ void __launch_bounds__(256) gram_kernel(const GramParams p) {
  CP_PDL_ENTRY();
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int64_t nitems = p.item_off[p.njobs];
  if (item < nitems) {
    int j, r, s;
    int64_t ch;
    job_entry(p, item, &j, &r, &s, &ch);
    const GramJob& g = p.job[j];
    const int R = p.R;
    const int64_t i0 = ch * kGramChunk, i1 = min(g.I, i0 + kGramChunk);
    const double a = g.D ? *g.stp : 0.0;
    // element of an operand, shifted by a D when the job has one (the same
    // fma as the kernel that forms x = base + stp d)
    auto xv = [&](const double* M, int64_t idx) { return g.D ? fma(a, g.D[idx], M[idx]) : M[idx]; };
    double a0 = 0.0, a1 = 0.0;
    int64_t i = i0 + lane;
    for (; i + 32 < i1; i += 64) {
      a0 = fma(xv(g.X, i * R + r), xv(g.Y, i * R + s), a0);
      a1 = fma(xv(g.X, (i + 32) * R + r), xv(g.Y, (i + 32) * R + s), a1);
    }
    if (i < i1) a0 = fma(xv(g.X, i * R + r), xv(g.Y, i * R + s), a0);
    double v = a0 + a1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
      if (p.chunked) {
        p.partial[item] = v;
      } else {
        g.out[r * R + s] = v;
        if (g.sym) g.out[s * R + r] = v;
      }
    }
  }
  if (!p.chunked) return;
  // chunked: the last block adds each entry's chunk sums in chunk order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(p.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const int R = p.R;
  for (int j = 0; j < p.njobs; ++j) {
    const GramJob& g = p.job[j];
    const int64_t nch = (g.I + kGramChunk - 1) / kGramChunk;
    const int ne = g.sym ? R * (R + 1) / 2 : R * R;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      double v = 0.0;
      for (int64_t c = 0; c < nch; ++c) v += __ldcg(&p.partial[p.item_off[j] + (int64_t)e * nch + c]);
      int r, s;
      if (g.sym) {
        upper_pair(e, R, &r, &s);
      } else {
        r = e / R;
        s = e - r * R;
      }
      g.out[r * R + s] = v;
      if (g.sym) g.out[s * R + r] = v;
    }
  }
  if (threadIdx.x == 0) *p.counter = 0u;
}

struct InvParams {
  const double* grams;   // N x R*R
  int N, R, n;
  double* Xinv;          // R*R out: Gammabar^(n)^-1
  int* ok;               // out: 1 on success
  int* status;
};

// In-place Gauss-Jordan inversion of the SPD matrix in A (B: a second buffer).
// One pivot step maps every entry from the old matrix to the new one, so the
// two buffers alternate with one barrier per pivot.  With p = 1 / S_kk:
//   S_ij -= S_ik p S_kj (i, j != k),  S_ik = -S_ik p,  S_kj = -S_kj p,
//   S_kk = -p;  after all pivots the buffer holds -S^-1.  The matrix stays
// symmetric, so only i <= j is computed (and mirrored), and the thread that
// computes the next diagonal entry forms its reciprocal at once (look-ahead),
// so the next pivot starts right after the barrier.
__device__ bool gj_inverse2(double* A, double* B, int R, double** out, double* piv2, int* flag) {
  if (threadIdx.x == 0) {
    const double d = A[0];
    if (!(d > 0.0) || !isfinite(d)) *flag = 1;
    else piv2[0] = recip_nr(d);
  }
  __syncthreads();
  double* src = A;
  double* dst = B;
  // this thread's entries e = tid, tid + blockDim, ... as (i, j), stepped
  // without divisions (the same entries at every pivot)
  const int i0 = (int)threadIdx.x / R, j0 = (int)threadIdx.x - ((int)threadIdx.x / R) * R;
  const int qi = (int)blockDim.x / R, qj = (int)blockDim.x - ((int)blockDim.x / R) * R;
  for (int k = 0; k < R; ++k) {
    if (*flag) return false;                     // uniform: read after a barrier
    const double pinv = piv2[k & 1];
    int i = i0, j = j0;
    for (int e = threadIdx.x; e < R * R; e += blockDim.x, i += qi, j += qj) {
      if (j >= R) {
        j -= R;
        ++i;
      }
      if (i > j) continue;
      double v;
      if (i == k && j == k)
        v = -pinv;
      else if (i == k)
        v = -src[k * R + j] * pinv;
      else if (j == k)
        v = -src[i * R + k] * pinv;
      else
        v = fma(-src[i * R + k] * pinv, src[k * R + j], src[i * R + j]);
      dst[i * R + j] = v;
      dst[j * R + i] = v;
      if (i == k + 1 && j == k + 1) {
        if (!(v > 0.0) || !isfinite(v)) *flag = 1;
        else piv2[(k + 1) & 1] = recip_nr(v);
      }
    }
    __syncthreads();
    double* t = src;
    src = dst;
    dst = t;
  }
  *out = src;
  return true;
}

// Dynamic shared memory: two R x R FP64 buffers.
__global__ void __launch_bounds__(256) gram_inverse_kernel(const InvParams p) {
  CP_PDL_ENTRY();
  extern __shared__ double dsm[];
  const int R = p.R, RR = R * R;
  double* A = dsm;
  double* B = dsm + RR;
  auto build = [&](double ridge) {
    for (int k = threadIdx.x; k < RR; k += blockDim.x) {
      double v = 1.0;
      for (int m = 0; m < p.N; ++m)
        if (m != p.n) v *= p.grams[(int64_t)m * RR + k];
      A[k] = v;
    }
    __syncthreads();
    if (ridge > 0.0) {
      double tr = 0.0;
      for (int r = 0; r < R; ++r) tr += A[r * R + r];
      __syncthreads();
      for (int r = threadIdx.x; r < R; r += blockDim.x) A[r * R + r] += ridge * tr / R;
      __syncthreads();
    }
  };
  __shared__ double piv2[2];
  __shared__ int flag;
  double* res = nullptr;
  if (threadIdx.x == 0) flag = 0;
  build(0.0);
  bool ok = gj_inverse2(A, B, R, &res, piv2, &flag);
  if (!ok) {
    __syncthreads();
    if (threadIdx.x == 0) flag = 0;
    build(1e-12);
    ok = gj_inverse2(A, B, R, &res, piv2, &flag);
  }
  for (int k = threadIdx.x; k < RR; k += blockDim.x) p.Xinv[k] = ok ? -res[k] : 0.0;
  if (threadIdx.x == 0) {
    *p.ok = ok ? 1 : 0;
    if (!ok) record_status(p.status, CP_ERR_NOT_SPD);
  }
}

size_t inverse_smem(int R) { return 2 * (size_t)R * R * sizeof(double); }

cp_status inverse_smem_attr() {
  static bool done = false;
  if (!done) {
    CP_CUDA(cudaFuncSetAttribute(gram_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)inverse_smem(CP_MAX_R)));
    done = true;
  }
  return CP_OK;
}

struct UpdParams {
  Parts parts;
  int64_t I;
  int R;
  int rows;              // rows per block
  const double* Xinv;
  const int* ok;
  double* An;            // I x R, updated in place
  float* An32;           // nullable: padded FP32 rows (stride rs)
  int rs;
  double* Mout;          // nullable: the summed M^(n) rows (I x R)
};

__global__ void __launch_bounds__(256) als_update_kernel(const UpdParams p) {
  CP_PDL_ENTRY();
  __shared__ double X[CP_MAX_R * CP_MAX_R];
  __shared__ double Mt[2 * CP_MAX_R];
  __shared__ float redf[8][33];
  __shared__ double redd[8][33];
  const int R = p.R, RR = R * R;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t rb = (int64_t)blockIdx.x * p.rows;
  const int nr = (int)min((int64_t)p.rows, p.I - rb);
  const int nout = nr * R;
  const int64_t nel = p.I * R;
  const bool ok = *p.ok != 0;
  if (!ok && !p.Mout) return;
  if (ok)
    for (int k = threadIdx.x; k < RR; k += blockDim.x) X[k] = p.Xinv[k];
  // M rows of this block: warp w adds partials c = w, w + 8, ... for 32
  // consecutive outputs; warp 0 adds the eight warp sums in order
  for (int e0 = 0; e0 < nout; e0 += 32) {
    const int64_t e = rb * R + e0 + lane;
    const bool in = e0 + lane < nout;
    if (p.parts.f32) {
      redf[w][lane] = in ? strided_sum((const float*)p.parts.p + e, w, p.parts.count, 8, nel) : 0.f;
    } else {
      redd[w][lane] = in ? strided_sum((const double*)p.parts.p + e, w, p.parts.count, 8, nel) : 0.0;
    }
    __syncthreads();
    if (w == 0 && in) {
      if (p.parts.f32) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += redf[q][lane];
        Mt[e0 + lane] = (double)t;
      } else {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += redd[q][lane];
        Mt[e0 + lane] = t;
      }
    }
    __syncthreads();
  }
  // M^(n) depends on the other modes only, so it is kept even when the
  // update itself is skipped (no inverse)
  if (p.Mout)
    for (int o = threadIdx.x; o < nout; o += blockDim.x) p.Mout[rb * R + o] = Mt[o];
  if (!ok) return;
  // a_i = m_i Gammabar^-1: one output per thread, two partial chains
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int q = o / R, r = o - (o / R) * R;
    const double* m = Mt + q * R;
    double s0 = 0.0, s1 = 0.0;
    int k = 0;
    for (; k + 1 < R; k += 2) {
      s0 = fma(m[k], X[k * R + r], s0);
      s1 = fma(m[k + 1], X[(k + 1) * R + r], s1);
    }
    if (k < R) s0 = fma(m[k], X[k * R + r], s0);
    const double a = s0 + s1;
    const int64_t idx = (rb + q) * R + r;
    p.An[idx] = a;
    if (p.An32) p.An32[(rb + q) * p.rs + r] = (float)a;
  }
}

// Padded FP32 copy: every float of the layout is written (padding as 0).
__global__ void f32_copy_kernel(Layout L, const double* __restrict__ u, F32Off o, int64_t total,
                                float* __restrict__ out) {
  CP_PDL_ENTRY();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int n = 0;
    while (n + 1 < L.N && q >= o.off[n + 1]) ++n;
    const int64_t within = q - o.off[n];
    const int64_t i = within / o.rs;
    const int r = (int)(within - i * o.rs);
    out[q] = r < L.R ? (float)u[L.off[n] + i * L.R + r] : 0.f;
  }
}

}  // namespace

cp_status gram_inverse_launch(cp_ctx* ctx, cudaStream_t s, const double* grams, const Layout& L, int n, double* xi) {
  CP_TRY(inverse_smem_attr());
  InvParams ip{grams, L.N, L.R, n, xi, (int*)(xi + (size_t)L.R * L.R), ctx->d_status};
  (void)launch_pdl(gram_inverse_kernel, dim3(1), dim3(256), inverse_smem(L.R), s, ip);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

cp_status f32_copy(cp_ctx* ctx, const Layout& L, const double* u, const F32Off& o, int64_t total, float* out) {
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4 * ctx->num_sms));
  (void)launch_pdl(f32_copy_kernel, dim3(blocks), dim3(256), 0, ctx->stream, L, u, o, total, out);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

cp_status grams_jobs(cp_ctx* ctx, cudaStream_t s, unsigned* counter, int R, const GramJob* jobs, int njobs) {
  if (njobs < 1 || njobs > kMaxGramJobs) {
    set_error("grams: %d jobs outside [1, %d]", njobs, kMaxGramJobs);
    return CP_ERR_ARG;
  }
  GramParams p{};
  p.njobs = njobs;
  p.R = R;
  int64_t items = 0;
  for (int j = 0; j < njobs; ++j) {
    p.job[j] = jobs[j];
    p.item_off[j] = items;
    const int64_t nch = std::max<int64_t>(1, (jobs[j].I + kGramChunk - 1) / kGramChunk);
    if (nch > 1) p.chunked = 1;
    items += (int64_t)(jobs[j].sym ? R * (R + 1) / 2 : R * R) * nch;
  }
  p.item_off[njobs] = items;
  p.counter = counter;
  if (p.chunked) {
    // chunked jobs need every job's item layout to carry its chunk count;
    // jobs that fit one chunk still index as nch = 1
    CP_TRY(ws_alloc_on(ctx, s, (void**)&p.partial, sizeof(double) * (size_t)items));
  }
  const unsigned blocks = (unsigned)std::max<int64_t>(1, (items + 7) / 8);
  (void)launch_pdl(gram_kernel, dim3(blocks), dim3(256), 0, s, p);
  CP_LAUNCH_CHECK();
  if (p.partial) ws_free_on(ctx, s, p.partial);
  return CP_OK;
}

cp_status grams_of(cp_ctx* ctx, cudaStream_t s, unsigned* counter, const Layout& L, const double* u, int mode_lo,
                   int nmodes, double* grams) {
  GramJob jobs[kMaxGramJobs];
  for (int k = 0; k < nmodes; ++k) {
    const int m = mode_lo + k;
    jobs[k] = GramJob{u + L.off[m], u + L.off[m], L.dims[m], grams + (size_t)m * L.R * L.R, 1};
  }
  return grams_jobs(ctx, s, counter, L.R, jobs, nmodes);
}

// One ALS sweep in place on u (Section 2.3): every mode n in turn takes
// A_n = M^(n) Gammabar^(n)^-1.  grams (N x R x R) receives the Grams of the
// updated factors; with grams_valid it already holds those of u on entry.
// With mlast_out the last mode's M^(N) (from the updated modes 1..N-1) is
// kept: it is M^(N) of the swept point as well.
cp_status als_sweep_v2(cp_ctx* ctx, const cp_tensor* t_in, const Layout& L, double* u, cp_precision prec,
                       double* grams, bool grams_valid, const double* m0, const double* xi0, double* mlast_out,
                       float* u32_io) {
  cp_tensor* t = const_cast<cp_tensor*>(t_in);
  const int R = L.R, N = L.N, RR = R * R;
  const bool want_f32 = t->kind == 0 && prec == CP_MIXED_BF16X3;
  int64_t acc32 = 0;
  const F32Off o32 = f32_layout(L, &acc32);
  float* u32 = nullptr;
  double* Xinv = nullptr;
  int* ok = nullptr;
  const bool own32 = want_f32 && !u32_io;
  if (want_f32) u32 = u32_io;
  if (own32) CP_TRY(ws_alloc(ctx, (void**)&u32, sizeof(float) * (size_t)acc32 + 64));
  CP_TRY(ws_alloc(ctx, (void**)&Xinv, sizeof(double) * (size_t)RR + 64));
  ok = (int*)(Xinv + RR);
  CP_TRY(inverse_smem_attr());
  if (own32) CP_TRY(f32_copy(ctx, L, u, o32, acc32, u32));
  if (!grams_valid) CP_TRY(grams_of(ctx, ctx->stream, ctx->d_counter, L, u, 0, N, grams));
  const int rows = std::max(1, 32 / R);
  const bool dtree = ctx->dimtree && want_f32 && N == 3;
  Parts W{};
  for (int n = 0; n < N; ++n) {
    // aux: (Gram of the mode updated last) -> inverse of Gammabar^(n),
    // overlapped with this mode's MTTKRP on the main stream; the first mode's
    // inverse may come precomputed (xi0)
    const bool pre = n == 0 && xi0;
    if (!pre) {
      CP_CUDA(cudaEventRecord(ctx->ev_fork, ctx->stream));
      CP_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
      if (n > 0) CP_TRY(grams_of(ctx, ctx->aux, ctx->d_counter + 1, L, u, n - 1, 1, grams));
      InvParams ip{grams, N, R, n, Xinv, ok, ctx->d_status};
      (void)launch_pdl(gram_inverse_kernel, dim3(1), dim3(256), inverse_smem(R), ctx->aux, ip);
      CP_LAUNCH_CHECK();
      CP_CUDA(cudaEventRecord(ctx->ev_join, ctx->aux));
    }
    Parts pt;
    if (n == 0 && m0) {
      pt = Parts{m0, 1, 0};
    } else if (dtree && n >= 1) {
      // M^(2) and M^(3) from W = T x_1 A^(1) (A^(1) just updated): M^(2)
      // with the old A^(3), M^(3) with the A^(2) updated in between
      if (n == 1) CP_TRY(dimtree_w(ctx, t, L, u32, o32, 0, &W));
      double* M = nullptr;
      CP_TRY(ws_alloc(ctx, (void**)&M, sizeof(double) * (size_t)L.dims[n] * R));
      CP_TRY(dimtree_contract(ctx, t, L, W, 0, n, u32, o32, M));
      pt = Parts{M, 1, 0};
    } else {
      CP_TRY(mttkrp_parts(ctx, t, L, u, u32, o32, n, prec, &pt));
    }
    if (!pre) CP_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    UpdParams up;
    up.parts = pt;
    up.I = L.dims[n];
    up.R = R;
    up.rows = rows;
    up.Xinv = pre ? xi0 : Xinv;
    up.ok = pre ? (const int*)(xi0 + RR) : ok;
    up.An = u + L.off[n];
    up.An32 = u32 ? u32 + o32.off[n] : nullptr;
    up.rs = o32.rs;
    up.Mout = n == N - 1 ? mlast_out : nullptr;
    (void)launch_pdl(als_update_kernel, dim3((unsigned)((L.dims[n] + rows - 1) / rows)), dim3(256), 0, ctx->stream, up);
    CP_LAUNCH_CHECK();
    if (!(n == 0 && m0)) ws_free(ctx, const_cast<void*>(pt.p));
  }
  if (W.p) ws_free(ctx, const_cast<void*>(W.p));
  CP_TRY(grams_of(ctx, ctx->stream, ctx->d_counter, L, u, N - 1, 1, grams));
  ws_free(ctx, Xinv);
  if (own32) ws_free(ctx, u32);
  return CP_OK;
}

}  // namespace cpg
