// Step III of N-GMRES (Section 2.1, Eq. linesearch) on the exact polynomial
// phi(beta) = f(ubar + beta d).
//
// The CP model is multilinear in the factors, so along the search line
//   phi(beta) = 1/2 ||T||^2 - C(beta) + 1/2 E(beta)
// with (Eq. fA written out along the line)
//   C(beta) = sum_r T x_1 (a1_r + beta d1_r) ... x_N (aN_r + beta dN_r)
//           = sum over subsets S of the modes of beta^|S| <T, rank-1 terms>,
//   E(beta) = sum_{r,s} prod_n (A_n^T A_n + beta (A_n^T D_n + D_n^T A_n)
//                               + beta^2 D_n^T D_n)[r, s],
// a polynomial of degree 2N whose coefficients need one pass over T: the
// MTTKRP of the last mode against the 2^(N-1) Khatri-Rao products in which
// every other mode contributes either its A or its D factor, contracted with
// A and D of the last mode, plus three Grams per mode.  Where the variant
// tiles are narrow, the same launch makes every other mode's variants too,
// from which M^(n)(ubar + beta d) of every mode, and so f and g at the
// accepted point, follow without another pass.  The More-Thuente
// search then evaluates phi and phi' = dphi/dbeta (= g(ubar + beta d) . d)
// by Horner's rule at no further cost per trial, in one thread.  Every trial
// sees the same function the paper's search sees; only the arithmetic that
// produces its values differs.
#include <algorithm>

#include "cp_internal.cuh"
#include "reduce.cuh"
#include "linesearch.cuh"
#include "mt_device.cuh"
#include "solver.cuh"

namespace cpg {


namespace {

constexpr int kMaxVar = 1 << (CP_MAX_N - 1);
constexpr int kMaxDeg = 2 * CP_MAX_N;

struct CoefParams {
  const void* pp[kMaxVar];      // partial sums of variant v
  int count[kMaxVar];
  int f32;
  int col_stride;               // columns per row of the partials
  int col_off[kMaxVar];         // first column of variant v
  int nvar;
  int64_t I;                    // rows of the last mode
  int64_t chunks;               // 32-output chunks per variant
  int R, N;
  const double* Alast;
  const double* Dlast;
  const double* epoly;          // 2N + 1 coefficients of E(beta)
  double norm2;
  double* blk;                  // [2][gridDim.x]
  double* poly;                 // 2N + 1 coefficients out
  double* mv_out;               // nullable: M_v (nvar x I x R, FP64)
  // the other modes' variants (tensor-core layout, like the last mode's),
  // summed into xout[k] (nvar x I x R, FP64) by the blocks past the last
  // mode's nvar x chunks
  int nx;
  const float* xpp[CP_MAX_N - 1];
  int xcount[CP_MAX_N - 1];
  int64_t xI[CP_MAX_N - 1];
  int64_t xblk_off[CP_MAX_N];   // prefix of nvar x chunks over those modes
  double* xout[CP_MAX_N - 1];
  MTState* st;
  cp_ls_opts o;
  SolveCtl* ctl;                // nullable: solver counters
  cudaGraphConditionalHandle h;
  int use_h;
  unsigned* counter;
  int* status;
};

// E(beta) coefficients: thread per (r, s), the product of the N quadratics
// of that entry; block sums, then the last block adds them in block order.
__global__ void __launch_bounds__(256) ls_epoly_kernel(const double* __restrict__ grams, int N, int R,
                                                       double* __restrict__ blk, double* __restrict__ e_out,
                                                       unsigned* counter) {
  CP_PDL_ENTRY();
  __shared__ double epart[8][kMaxDeg + 1];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int RR = R * R, D = 2 * N;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double c[kMaxDeg + 1];
#pragma unroll
  for (int q = 0; q <= kMaxDeg; ++q) c[q] = 0.0;
  if (k < RR) {
    const int rr = k / R, ss = k - (k / R) * R;
    c[0] = 1.0;
    int deg = 0;
    for (int n = 0; n < N; ++n) {
      const double q0 = grams[(int64_t)(0 * N + n) * RR + k];
      const double q1 = grams[(int64_t)(1 * N + n) * RR + k] + grams[(int64_t)(1 * N + n) * RR + ss * R + rr];
      const double q2 = grams[(int64_t)(2 * N + n) * RR + k];
      for (int q = deg + 2; q >= 0; --q) {
        double t = q <= deg ? c[q] * q0 : 0.0;
        if (q >= 1 && q - 1 <= deg) t = fma(c[q - 1], q1, t);
        if (q >= 2) t = fma(c[q - 2], q2, t);
        c[q] = t;
      }
      deg += 2;
    }
  }
  for (int q = 0; q <= D; ++q) {
    double s = c[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) epart[w][q] = s;
  }
  __syncthreads();
  if ((int)threadIdx.x <= D) {
    double s = 0.0;
    for (int ww = 0; ww < 8; ++ww) s += epart[ww][threadIdx.x];
    blk[(int64_t)blockIdx.x * (kMaxDeg + 1) + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if ((int)threadIdx.x <= D) {
    double s = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&blk[(int64_t)b * (kMaxDeg + 1) + threadIdx.x]);
    e_out[threadIdx.x] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

__global__ void __launch_bounds__(256) ls_coef_kernel(const CoefParams p) {
  CP_PDL_ENTRY();
  __shared__ float redf[8][33];
  __shared__ double redd[8][33];
  __shared__ double sums[2 * kMaxVar];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int R = p.R, N = p.N;
  if ((int64_t)blockIdx.x >= (int64_t)p.nvar * p.chunks) {
    // another mode's variants: sum the partials into xout (no coefficient)
    const int64_t b = (int64_t)blockIdx.x - (int64_t)p.nvar * p.chunks;
    int k = 0;
    while (k + 1 < p.nx && b >= p.xblk_off[k + 1]) ++k;
    const int64_t xch = (p.xI[k] * R + 31) / 32;
    const int64_t bb = b - p.xblk_off[k];
    const int vx = (int)(bb / xch);
    const int64_t ex = (bb - (int64_t)vx * xch) * 32 + lane;
    const int64_t noutx = p.xI[k] * R;
    const bool inx = ex < noutx;
    const int64_t ix = inx ? ex / R : 0;
    const int rx = inx ? (int)(ex - ix * R) : 0;
    const int64_t idxx = ix * p.col_stride + p.col_off[vx] + rx;
    redf[w][lane] = inx ? strided_sum(p.xpp[k] + idxx, w, p.xcount[k], 8, p.xI[k] * p.col_stride) : 0.f;
    __syncthreads();
    if (w == 0 && inx) {
      float t = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += redf[q][lane];
      p.xout[k][(int64_t)vx * noutx + ex] = (double)t;
    }
  } else {
    const int v = (int)(blockIdx.x / p.chunks);
    const int64_t e = (blockIdx.x - (int64_t)v * p.chunks) * 32 + lane;
    const int64_t nout = p.I * R;
    const bool in = e < nout;
    const int64_t i = in ? e / R : 0;
    const int r = in ? (int)(e - i * R) : 0;
    const int64_t nel = p.I * p.col_stride;
    const int64_t idx = i * p.col_stride + p.col_off[v] + r;
    // M_v[i][r]: warp w adds partials c = w, w + 8, ...; warp 0 the warp sums
    if (p.f32) {
      redf[w][lane] = in ? strided_sum((const float*)p.pp[v] + idx, w, p.count[v], 8, nel) : 0.f;
    } else {
      redd[w][lane] = in ? strided_sum((const double*)p.pp[v] + idx, w, p.count[v], 8, nel) : 0.0;
    }
    __syncthreads();
    if (w == 0) {
      double m = 0.0;
      if (p.f32) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += redf[q][lane];
        m = (double)t;
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) m += redd[q][lane];
      }
      if (p.mv_out && in) p.mv_out[(int64_t)v * nout + e] = m;
      double a = in ? m * p.Alast[e] : 0.0;
      double b = in ? m * p.Dlast[e] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        p.blk[blockIdx.x] = a;
        p.blk[gridDim.x + blockIdx.x] = b;
      }
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(p.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // <M_v, A_last> and <M_v, D_last>: one warp per sum, lanes stride the chunks
  for (int k = w; k < 2 * p.nvar; k += 8) {
    const int vv = k >> 1, which = k & 1;
    const double* src = p.blk + (which ? gridDim.x : 0) + (int64_t)vv * p.chunks;
    double s = 0.0;
    for (int64_t c = lane; c < p.chunks; c += 32) s += __ldcg(&src[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sums[k] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double poly[kMaxDeg + 1];
  for (int q = 0; q <= 2 * N; ++q) poly[q] = 0.5 * __ldcg(&p.epoly[q]);
  // C(beta): variant v (bit m: mode m uses D) with the last mode's A adds to
  // beta^popc(v), with its D to beta^(popc(v) + 1)
  for (int vv = 0; vv < p.nvar; ++vv) {
    const int k = __popc(vv);
    poly[k] -= sums[2 * vv];
    poly[k + 1] -= sums[2 * vv + 1];
  }
  poly[0] += 0.5 * p.norm2;
  for (int q = 0; q <= 2 * N; ++q) p.poly[q] = poly[q];
  // More-Thuente on phi, phi' by Horner's rule
  MTState s;
  mtdev::mt_init(s, poly[0], poly[1], p.o);
  while (!s.done) {
    const double b = s.stp;
    double f = poly[2 * N], g = 2 * N * poly[2 * N];
    for (int q = 2 * N - 1; q >= 1; --q) {
      f = fma(f, b, poly[q]);
      g = fma(g, b, q * poly[q]);
    }
    f = fma(f, b, poly[0]);
    mtdev::mt_advance(&s, &f, &g);
  }
  *p.st = s;
  const bool accept = s.nfev > 0 && (s.info == 1 || s.f <= s.f0 + s.ftol * s.stp_eval * s.g0);
  if (p.ctl) {
    SolveCtl* c = p.ctl;
    c->ls_evals += s.nfev;
    if (s.info != 1) c->ls_failures += 1;
    if (accept) {
      c->accepts += 1;
      c->fg_evals += 1;
    }
  }
  if (p.use_h) cudaGraphSetConditional(p.h, accept ? 1u : 0u);
  *p.counter = 0u;
}

// Mixed iterates w_v (v < nvar): factor m < N-1 is d's when bit m of v is
// set, else a's; the last factor is a's.
__global__ void mix_kernel(Layout L, const double* __restrict__ a, const double* __restrict__ d, int nvar,
                           double* __restrict__ w) {
  CP_PDL_ENTRY();
  const int64_t P = L.off[L.N];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
    int n = 0;
    while (n + 1 < L.N && e >= L.off[n + 1]) ++n;
    const double av = a[e], dv = d[e];
    for (int v = 0; v < nvar; ++v) w[(int64_t)v * P + e] = (n < L.N - 1 && ((v >> n) & 1)) ? dv : av;
  }
}

}  // namespace

cp_status ls_poly(cp_ctx* ctx, const cp_tensor* t_in, const Layout& L, const double* base, const double* d,
                  cp_precision prec, const cp_ls_opts& o, MTState* st, double* poly, SolveCtl* ctl,
                  cudaGraphConditionalHandle h, int use_h, double* mv_out, bool* all_modes, double* grams_out,
                  const float* base32, const float* d32_in) {
  cp_tensor* t = const_cast<cp_tensor*>(t_in);
  const int N = L.N, R = L.R, RR = R * R;
  const int last = N - 1;
  const int nvar = 1 << (N - 1);
  if (N > CP_MAX_N) return CP_ERR_ARG;
  const bool tc = t->kind == 0 && prec == CP_MIXED_BF16X3;
  const bool tc_var = tc && tc_variants_supported(L);
  int64_t acc32 = 0;
  const F32Off o32 = f32_layout(L, &acc32);
  // every mode's variants in the same launch when they are kept and the
  // Khatri-Rao tiles stay narrow (at most 64 variant columns per contraction
  // element: wider ones make the tile builders, not the stream of T, the
  // bound, and the variants of the other modes would cost more than the
  // plain passes they replace)
  const bool all = tc_var && mv_out && nvar * o32.rs <= 64;
  if (all_modes) *all_modes = all;
  const int64_t P = L.P();
  const unsigned eblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((P + 255) / 256, 4 * ctx->num_sms));
  // Grams on the aux stream, overlapped with the MTTKRP
  double* work = nullptr;
  const size_t eblocks_n = (size_t)((RR + 255) / 256);
  CP_TRY(ws_alloc(ctx, (void**)&work,
                  sizeof(double) * (3 * (size_t)N * RR + (eblocks_n + 1) * (kMaxDeg + 1))));
  double* grams = grams_out ? grams_out : work;
  double* eblk = work + 3 * (size_t)N * RR;
  double* epoly = eblk + eblocks_n * (kMaxDeg + 1);
  CP_CUDA(cudaEventRecord(ctx->ev_fork, ctx->stream));
  CP_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
  {
    GramJob jobs[kMaxGramJobs];
    int nj = 0;
    for (int n = 0; n < N; ++n) {
      const double* A = base + L.off[n];
      const double* D = d + L.off[n];
      jobs[nj++] = GramJob{A, A, L.dims[n], grams + (size_t)(0 * N + n) * RR, 1};
      jobs[nj++] = GramJob{A, D, L.dims[n], grams + (size_t)(1 * N + n) * RR, 0};
      jobs[nj++] = GramJob{D, D, L.dims[n], grams + (size_t)(2 * N + n) * RR, 1};
    }
    CP_TRY(grams_jobs(ctx, ctx->aux, ctx->d_counter + 1, R, jobs, nj));
    const unsigned eb = (unsigned)((RR + 255) / 256);
    (void)launch_pdl(ls_epoly_kernel, dim3(eb), dim3(256), 0, ctx->aux, grams, N, R, eblk, epoly, ctx->d_counter + 1);
    CP_LAUNCH_CHECK();
  }
  CP_CUDA(cudaEventRecord(ctx->ev_join, ctx->aux));
  // the variant MTTKRPs of the last mode
  CoefParams cp{};
  Parts parts[kMaxVar];
  Parts pts[CP_MAX_N];
  int nm = 0;
  float *a32 = nullptr, *d32 = nullptr, *w32 = nullptr;
  bool own_a32 = false, own_d32 = false;
  double* wv = nullptr;
  if (tc_var) {
    own_a32 = !base32;
    own_d32 = !d32_in;
    a32 = const_cast<float*>(base32);
    d32 = const_cast<float*>(d32_in);
    if (own_a32) {
      CP_TRY(ws_alloc(ctx, (void**)&a32, sizeof(float) * (size_t)acc32 + 64));
      CP_TRY(f32_copy(ctx, L, base, o32, acc32, a32));
    }
    if (own_d32) {
      CP_TRY(ws_alloc(ctx, (void**)&d32, sizeof(float) * (size_t)acc32 + 64));
      CP_TRY(f32_copy(ctx, L, d, o32, acc32, d32));
    }
    // the last mode first, then (all) the others
    int modes[CP_MAX_N];
    modes[nm++] = last;
    if (all)
      for (int n = 0; n < last; ++n) modes[nm++] = n;
    CP_TRY(mttkrp_tc_variants(ctx, t, L, a32, d32, o32, modes, nm, pts));
    // variant v occupies columns v rs .. v rs + R - 1 of the partial sums
    for (int v = 0; v < nvar; ++v) {
      parts[v] = pts[0];
      cp.col_off[v] = v * o32.rs;
    }
    cp.col_stride = nvar * o32.rs;
    cp.nx = nm - 1;
    cp.xblk_off[0] = 0;
    for (int k = 0; k + 1 < nm; ++k) {
      const int n = modes[k + 1];
      cp.xpp[k] = (const float*)pts[k + 1].p;
      cp.xcount[k] = pts[k + 1].count;
      cp.xI[k] = L.dims[n];
      cp.xout[k] = mv_out + (size_t)nvar * L.off[n];
      cp.xblk_off[k + 1] = cp.xblk_off[k] + (int64_t)nvar * ((L.dims[n] * R + 31) / 32);
    }
  } else {
    CP_TRY(ws_alloc(ctx, (void**)&wv, sizeof(double) * (size_t)nvar * P));
    if (tc) CP_TRY(ws_alloc(ctx, (void**)&w32, sizeof(float) * (size_t)nvar * acc32 + 64));
    (void)launch_pdl(mix_kernel, dim3(eblocks), dim3(256), 0, ctx->stream, L, base, d, nvar, wv);
    CP_LAUNCH_CHECK();
    if (w32)
      for (int v = 0; v < nvar; ++v) CP_TRY(f32_copy(ctx, L, wv + (size_t)v * P, o32, acc32, w32 + (size_t)v * acc32));
    for (int v = 0; v < nvar; ++v) {
      CP_TRY(mttkrp_parts(ctx, t, L, wv + (size_t)v * P, w32 ? w32 + (size_t)v * acc32 : nullptr, o32, last, prec,
                          &parts[v]));
      cp.col_off[v] = 0;
    }
    cp.col_stride = R;
  }
  for (int v = 0; v < nvar; ++v) {
    cp.pp[v] = parts[v].p;
    cp.count[v] = parts[v].count;
  }
  cp.f32 = parts[0].f32;
  cp.nvar = nvar;
  cp.I = L.dims[last];
  cp.chunks = (L.dims[last] * R + 31) / 32;
  cp.R = R;
  cp.N = N;
  cp.Alast = base + L.off[last];
  cp.Dlast = d + L.off[last];
  cp.epoly = epoly;
  cp.norm2 = t->norm2;
  cp.poly = poly;
  cp.mv_out = mv_out ? mv_out + (size_t)nvar * L.off[last] : nullptr;
  cp.st = st;
  cp.o = o;
  cp.ctl = ctl;
  cp.h = h;
  cp.use_h = use_h;
  cp.counter = ctx->d_counter;
  cp.status = ctx->d_status;
  const int64_t nblocks = (int64_t)nvar * cp.chunks + cp.xblk_off[cp.nx];
  CP_TRY(ws_alloc(ctx, (void**)&cp.blk, sizeof(double) * 2 * (size_t)nblocks + 16));
  CP_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  (void)launch_pdl(ls_coef_kernel, dim3((unsigned)nblocks), dim3(256), 0, ctx->stream, cp);
  CP_LAUNCH_CHECK();
  ws_free(ctx, cp.blk);
  if (tc_var) {
    for (int k = 0; k < nm; ++k) ws_free(ctx, const_cast<void*>(pts[k].p));
  } else {
    for (int v = 0; v < nvar; ++v) ws_free(ctx, const_cast<void*>(parts[v].p));
  }
  if (own_a32) ws_free(ctx, a32);
  if (own_d32) ws_free(ctx, d32);
  if (w32) ws_free(ctx, w32);
  if (wv) ws_free(ctx, wv);
  ws_free(ctx, work);
  return CP_OK;
}

}  // namespace cpg
