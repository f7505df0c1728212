// N-GMRES Step II (Section 2.1, Eq. accel, Eq. linearize, Eq. normal): from a
// window of m previous iterates u_j and gradients g(u_j), and the preliminary
// iterate ubar with gradient gbar,
//     p_j = gbar - g(u_j),  (P^T P + delta I) alpha = -P^T gbar,
//     delta = eps * max_j (P^T P)_jj,  uhat = ubar + sum_j alpha_j (ubar - u_j).
// One pass over the window computes every p_j . p_l and p_j . gbar (the p_j
// are formed per element, never stored); the last block of the reduction adds
// the per-CTA sums in a fixed order and solves the m x m system by
// Gauss-Jordan elimination (no pivoting: the matrix is SPD); a last pass
// forms uhat (and, for the normalisation that follows, the column sums of
// squares of its factors).
//
// The window is a ring of `cap` slots in device memory; its state
// win = {start, m} also lives in device memory (window row j, oldest first, is
// slot (start + j) % cap), so the whole step can be replayed from a CUDA graph
// while the window grows and rotates (window size w of Section 2.1).
#include <algorithm>

#include "cp_internal.cuh"
#include "newton.cuh"
#include "reduce.cuh"

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
  CP_PDL_ENTRY();
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

// Block b adds the per-CTA partial sums of outputs 32b .. 32b+31 (warp w
// takes CTAs w, w + 8, ...; fixed order).  The last block assembles
// H = P^T P + delta I and the right-hand side -P^T gbar and solves by
// Gauss-Jordan elimination on [H | rhs] (no pivoting: H is SPD, and a
// non-positive pivot reports CP_ERR_NOT_SPD with alpha = 0).
__global__ void __launch_bounds__(256) ngmres_reduce_solve_kernel(const double* __restrict__ part, int nparts,
                                                                  int nout_max, const int* __restrict__ win,
                                                                  double eps, double* __restrict__ sums,
                                                                  double* __restrict__ alpha, unsigned* counter,
                                                                  int* status) {
  CP_PDL_ENTRY();
  __shared__ double red[8][33];
  __shared__ double Ab[CP_MAX_W * (CP_MAX_W + 1)];
  __shared__ double dmax;
  __shared__ int flag;
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m = win[1];
  const int npairs = m * (m + 1) / 2;
  const int nout = npairs + m;
  const int o = blockIdx.x * 32 + lane;
  red[w][lane] = o < nout ? strided_sum(part + o, w, nparts, 8, (int64_t)nout_max) : 0.0;
  __syncthreads();
  if (w == 0 && o < nout) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q][lane];
    sums[o] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const int W = m + 1;   // row stride of [H | rhs]
  for (int q = threadIdx.x; q < nout; q += blockDim.x) {
    const double v = __ldcg(&sums[q]);
    if (q < npairs) {
      int j, l;
      pair_of(q, m, &j, &l);
      Ab[j * W + l] = v;
      Ab[l * W + j] = v;
    } else {
      Ab[(q - npairs) * W + m] = -v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int j = 0; j < m; ++j) d = fmax(d, Ab[j * W + j]);
    dmax = d;
    flag = 0;
    if (d > 0.0)
      for (int j = 0; j < m; ++j) Ab[j * W + j] += eps * d;
  }
  __syncthreads();
  if (!(dmax > 0.0)) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) alpha[j] = 0.0;
    if (threadIdx.x == 0) *counter = 0u;
    return;
  }
  // Elimination of column k from every other row touches columns > k only
  // and never row k, so it runs in place with one barrier per pivot; the
  // thread that updates the next diagonal entry forms its reciprocal at once
  // (look-ahead).  Each thread keeps the same entries (i, j) of the m x W
  // array at every pivot, stepped without divisions.
  __shared__ double piv2[2];
  if (threadIdx.x == 0) {
    const double d = Ab[0];
    if (!(d > 0.0) || !isfinite(d)) flag = 1;
    else piv2[0] = recip_nr(d);
  }
  __syncthreads();
  const int i0 = (int)threadIdx.x / W, j0 = (int)threadIdx.x - ((int)threadIdx.x / W) * W;
  const int qi = (int)blockDim.x / W, qj = (int)blockDim.x - ((int)blockDim.x / W) * W;
  for (int k = 0; k < m; ++k) {
    if (flag) break;                             // uniform: read after a barrier
    const double pinv = piv2[k & 1];
    int i = i0, j = j0;
    for (int e = threadIdx.x; e < m * W; e += blockDim.x, i += qi, j += qj) {
      if (j >= W) {
        j -= W;
        ++i;
      }
      if (i == k || j <= k) continue;
      const double v = fma(-Ab[i * W + k] * pinv, Ab[k * W + j], Ab[i * W + j]);
      Ab[i * W + j] = v;
      if (i == k + 1 && j == k + 1) {
        if (!(v > 0.0) || !isfinite(v)) flag = 1;
        else piv2[(k + 1) & 1] = recip_nr(v);
      }
    }
    __syncthreads();
  }
  if (flag) {
    if (threadIdx.x == 0) record_status(status, CP_ERR_NOT_SPD);
    for (int j = threadIdx.x; j < m; j += blockDim.x) alpha[j] = 0.0;
  } else {
    // the system is now diagonal: alpha_j = rhs_j / H_jj
    for (int j = threadIdx.x; j < m; j += blockDim.x) alpha[j] = Ab[j * W + m] * recip_nr(Ab[j * W + j]);
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// uhat = ubar + sum_j alpha_j (ubar - u_j) over contiguous chunks of `chunk`
// entries (a multiple of R).  With colsq, the block size is a multiple of R so
// every thread stays on one rank r, and the block's column sums of squares of
// uhat per (mode, r) go to colsq[block][n][r] (fixed order).
__global__ void ngmres_combine_kernel(const double* __restrict__ U, const int* __restrict__ win, int cap,
                                      int64_t P, const double* __restrict__ ubar,
                                      const double* __restrict__ alpha, double* __restrict__ uhat, Layout L,
                                      int64_t chunk, double* __restrict__ colsq) {
  CP_PDL_ENTRY();
  __shared__ double a[CP_MAX_W];
  __shared__ int slot[CP_MAX_W];
  __shared__ double red[CP_MAX_N * 256];     // [N][blockDim] per-thread sums
  const int start = win[0];
  const int m = win[1];
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    a[j] = alpha[j];
    slot[j] = (start + j) % cap;
  }
  __syncthreads();
  const int R = L.R;
  const int64_t kb = (int64_t)blockIdx.x * chunk;
  const int64_t ke = min(P, kb + chunk);
  int n = 0;
  while (n + 1 < L.N && kb + (int64_t)threadIdx.x >= L.off[n + 1]) ++n;
  double acc = 0.0;
  int curn = n;
  // per-thread sums of squares, flushed into shared memory when the mode changes
  double* mine = red;
  const bool want = colsq != nullptr;
  if (want)
    for (int q = threadIdx.x; q < L.N * (int)blockDim.x; q += blockDim.x) red[q] = 0.0;
  __syncthreads();
  for (int64_t k = kb + threadIdx.x; k < ke; k += blockDim.x) {
    const double ub = ubar[k];
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
    int j = 0;
    for (; j + 3 < m; j += 4) {
      c0 = fma(a[j], ub - U[(int64_t)slot[j] * P + k], c0);
      c1 = fma(a[j + 1], ub - U[(int64_t)slot[j + 1] * P + k], c1);
      c2 = fma(a[j + 2], ub - U[(int64_t)slot[j + 2] * P + k], c2);
      c3 = fma(a[j + 3], ub - U[(int64_t)slot[j + 3] * P + k], c3);
    }
    for (; j < m; ++j) c0 = fma(a[j], ub - U[(int64_t)slot[j] * P + k], c0);
    const double v = ub + ((c0 + c1) + (c2 + c3));
    uhat[k] = v;
    if (want) {
      while (n + 1 < L.N && k >= L.off[n + 1]) ++n;
      if (n != curn) {
        mine[curn * blockDim.x + threadIdx.x] = acc;
        acc = 0.0;
        curn = n;
      }
      acc = fma(v, v, acc);
    }
  }
  if (!want) return;
  mine[curn * blockDim.x + threadIdx.x] = acc;
  __syncthreads();
  // thread t holds rank t % R; add the threads of each (mode, rank) in order
  for (int q = threadIdx.x; q < L.N * R; q += blockDim.x) {
    const int nn = q / R, r = q - (q / R) * R;
    double s = 0.0;
    for (int t = r; t < (int)blockDim.x; t += R) s += mine[nn * blockDim.x + t];
    colsq[((int64_t)nn * gridDim.x + blockIdx.x) * R + r] = s;
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
                      const double* ubar, const double* gbar, double eps, double* uhat, double* alpha,
                      const Layout* L, double* colsq, int* S_out) {
  if (cap < 1 || cap > CP_MAX_W) {
    set_error("ngmres: window capacity %d outside [1, %d]", cap, CP_MAX_W);
    return CP_ERR_ARG;
  }
  const int nout_max = cap * (cap + 1) / 2 + cap;
  // one CTA per SM (at most): the P (m(m+1)/2 + m) FP64 FMAs of the dots
  // spread over the whole chip
  int64_t nb = std::min<int64_t>((P + kTile - 1) / kTile, (int64_t)ctx->num_sms);
  nb = std::max<int64_t>(nb, 1);
  const int64_t chunk = (P + nb - 1) / nb;
  nb = std::max<int64_t>((P + chunk - 1) / chunk, 1);
  double* part = nullptr;
  double* a = alpha;
  CP_TRY(ws_alloc(ctx, (void**)&part, sizeof(double) * ((size_t)nb * nout_max + nout_max + CP_MAX_W)));
  double* sums = part + (size_t)nb * nout_max;
  if (!a) a = sums + nout_max;
  (void)launch_pdl(ngmres_dots_kernel, dim3((unsigned)nb), dim3(256), 0, ctx->stream, G, win, cap, P, gbar, chunk, nout_max, part);
  CP_LAUNCH_CHECK();
  (void)launch_pdl(ngmres_reduce_solve_kernel, dim3((unsigned)((nout_max + 31) / 32)), dim3(256), 0, ctx->stream, 
      part, (int)nb, nout_max, win, eps, sums, a, ctx->d_counter, ctx->d_status);
  CP_LAUNCH_CHECK();
  if (L && colsq) {
    // block size a multiple of R, chunks a multiple of the block size: every
    // thread keeps one rank, and the chunks tile the modes' R-aligned rows
    const int threads = std::max(L->R, (256 / L->R) * L->R);
    const int64_t per = std::max<int64_t>(1, (P + 2 * (int64_t)ctx->num_sms - 1) / (2 * (int64_t)ctx->num_sms));
    const int64_t chunk = (per + threads - 1) / threads * threads;
    const int64_t cb = (P + chunk - 1) / chunk;
    *S_out = (int)cb;
    (void)launch_pdl(ngmres_combine_kernel, dim3((unsigned)cb), dim3(threads), 0, ctx->stream, U, win, cap, P, ubar, a, uhat, *L, chunk,
                                                                     colsq);
  } else {
    Layout L1;
    L1.N = 1;
    L1.R = 1;
    L1.off[0] = 0;
    L1.off[1] = P;
    int64_t cb = std::min<int64_t>((P + 255) / 256, 8 * (int64_t)ctx->num_sms);
    cb = std::max<int64_t>(cb, 1);
    const int64_t chunk = (P + cb - 1) / cb;
    (void)launch_pdl(ngmres_combine_kernel, dim3((unsigned)cb), dim3(256), 0, ctx->stream, U, win, cap, P, ubar, a, uhat, L1, chunk, nullptr);
  }
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
