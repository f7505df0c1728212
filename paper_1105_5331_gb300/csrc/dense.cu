// Dense tensors: per-mode matricised copies, ||T||^2, and the FP64 MTTKRP.
//
// Layout decision: the handle keeps one row-major copy of T_(n) for every mode
// n (I_n x Kbar_n, Kbar_n = prod_{m != n} I_m, column index over the other
// modes in natural order with the last one fastest).  Every mode's MTTKRP
// M^(n) = T_(n) Phibar^(n) (Section 2.3, Eq. Gn) is then the same row-major,
// contiguous-in-the-contraction product, whatever n is.  The extra memory
// (N copies) is small next to the GPU's HBM.
#include "cp_internal.cuh"
#include "reduce.cuh"

#include <mutex>

namespace cpg {

namespace {

// T_(n)[i, l*Q + q] = T[l, i, q] where L = prod_{m<n} I_m, Q = prod_{m>n} I_m.
template <typename TT>
__global__ void matricize_kernel(const TT* __restrict__ src, TT* __restrict__ dst, int64_t L,
                                 int64_t I, int64_t Q) {
  const int64_t Kbar = L * Q;
  const int64_t total = I * Kbar;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = o / Kbar;
    const int64_t kb = o - i * Kbar;
    const int64_t l = kb / Q;
    const int64_t q = kb - l * Q;
    dst[o] = src[(l * I + i) * Q + q];
  }
}

// Deterministic sum of squares: per-block tree partials.
template <typename TT>
__global__ void sumsq_partial_kernel(const TT* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[k];
    acc = fma(v, v, acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
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

// Factors of the modes other than n, in natural order (last one fastest in k).
struct KRDesc {
  const double* A[CP_MAX_N - 1];
  int64_t I[CP_MAX_N - 1];
  int cnt;
};

constexpr int kF64BK = 32;     // contraction elements per tile
constexpr int kF64RSUB = 16;   // ranks per thread

// FP64 MTTKRP, one CTA per contiguous range of the contraction index kbar.
// Each CTA builds the Khatri-Rao tile KR[kbar, r] = prod_{m != n} A_m[i_m, r]
// for kF64BK columns in shared memory (FP64), then every thread owns one row
// i of T_(n) and up to kF64RSUB ranks and accumulates T[i, kbar] * KR[kbar, r].
// The CTA writes its partial I x R sum; a second kernel adds the partials in
// a fixed order, so results do not depend on scheduling.
template <typename TT>
__global__ void __launch_bounds__(256) mttkrp_f64_kernel(const TT* __restrict__ Tn, int64_t I,
                                                          int64_t Kbar, KRDesc kr, int R,
                                                          int64_t tiles_per_cta,
                                                          double* __restrict__ partial) {
  extern __shared__ double kr_tile[];  // [kF64BK][R]
  const int nsplit = (R + kF64RSUB - 1) / kF64RSUB;
  const int64_t k_begin = (int64_t)blockIdx.x * tiles_per_cta * kF64BK;
  const int64_t k_end = min(Kbar, k_begin + tiles_per_cta * kF64BK);
  const int rows_per_pass = blockDim.x / nsplit;
  const int my_row = threadIdx.x / nsplit;
  const int r0 = (threadIdx.x % nsplit) * kF64RSUB;
  const int rcount = min(kF64RSUB, R - r0);
  double* out = partial + (int64_t)blockIdx.x * I * R;

  for (int64_t row_base = 0; row_base < I; row_base += rows_per_pass) {
    const int64_t row = row_base + my_row;
    const bool active = my_row < rows_per_pass && row < I;
    double acc[kF64RSUB];
#pragma unroll
    for (int j = 0; j < kF64RSUB; ++j) acc[j] = 0.0;
    for (int64_t k0 = k_begin; k0 < k_end; k0 += kF64BK) {
      const int kt = (int)min((int64_t)kF64BK, k_end - k0);
      __syncthreads();
      for (int e = threadIdx.x; e < kt * R; e += blockDim.x) {
        const int kk = e / R;
        const int r = e - kk * R;
        int64_t rem = k0 + kk;
        double v = 1.0;
        for (int j = kr.cnt - 1; j >= 0; --j) {
          const int64_t q = rem / kr.I[j];
          const int64_t idx = rem - q * kr.I[j];
          rem = q;
          v *= kr.A[j][idx * R + r];
        }
        kr_tile[kk * R + r] = v;
      }
      __syncthreads();
      if (active) {
        const TT* trow = Tn + row * Kbar + k0;
        for (int kk = 0; kk < kt; ++kk) {
          const double x = (double)trow[kk];
          const double* krow = kr_tile + kk * R + r0;
#pragma unroll
          for (int j = 0; j < kF64RSUB; ++j)
            if (j < rcount) acc[j] = fma(x, krow[j], acc[j]);
        }
      }
    }
    if (active)
      for (int j = 0; j < rcount; ++j) out[row * R + r0 + j] = acc[j];
  }
}

}  // namespace

cp_status reduce_partials(cp_ctx* ctx, const double* partial, int nparts, int64_t n, double* out) {
  return reduce_parts<double>(ctx, partial, nparts, n, out);
}

cp_status sumsq(cp_ctx* ctx, const void* x, cp_dtype dt, int64_t n, double* d_out) {
  const int threads = 256;
  int nb = (int)std::min<int64_t>((n + threads - 1) / threads, 2 * ctx->num_sms);
  if (nb < 1) nb = 1;
  double* part = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&part, sizeof(double) * nb));
  if (dt == CP_DTYPE_F64)
    sumsq_partial_kernel<double><<<nb, threads, 0, ctx->stream>>>((const double*)x, n, part);
  else
    sumsq_partial_kernel<float><<<nb, threads, 0, ctx->stream>>>((const float*)x, n, part);
  CP_LAUNCH_CHECK();
  sum_partials_kernel<<<1, 256, 0, ctx->stream>>>(part, nb, d_out);
  CP_LAUNCH_CHECK();
  ws_free(ctx, part);
  return CP_OK;
}

cp_status dense_build(cp_ctx* ctx, cp_tensor* t, const void* d_data) {
  const size_t esz = t->dtype == CP_DTYPE_F64 ? 8 : 4;
  for (int n = 0; n < t->N; ++n) {
    CP_CUDA(cudaMallocAsync(&t->Tn[n], esz * (size_t)t->K, ctx->stream));
    int64_t L = 1, Q = 1;
    for (int m = 0; m < n; ++m) L *= t->dims[m];
    for (int m = n + 1; m < t->N; ++m) Q *= t->dims[m];
    int64_t blocks = (t->K + 255) / 256;
    if (blocks > 16 * ctx->num_sms) blocks = 16 * ctx->num_sms;
    if (n == 0) {
      CP_CUDA(cudaMemcpyAsync(t->Tn[0], d_data, esz * (size_t)t->K, cudaMemcpyDeviceToDevice,
                              ctx->stream));
    } else if (t->dtype == CP_DTYPE_F64) {
      matricize_kernel<double><<<(unsigned)blocks, 256, 0, ctx->stream>>>(
          (const double*)d_data, (double*)t->Tn[n], L, t->dims[n], Q);
    } else {
      matricize_kernel<float><<<(unsigned)blocks, 256, 0, ctx->stream>>>(
          (const float*)d_data, (float*)t->Tn[n], L, t->dims[n], Q);
    }
    CP_LAUNCH_CHECK();
  }
  double* d_norm = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&d_norm, sizeof(double)));
  CP_TRY(sumsq(ctx, d_data, t->dtype, t->K, d_norm));
  CP_CUDA(cudaMemcpyAsync(ctx->h_pinned, d_norm, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  t->norm2 = ctx->h_pinned[0];
  ws_free(ctx, d_norm);
  return CP_OK;
}

static cp_status mttkrp_f64_impl(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u,
                                 int mode, double* out, Parts* parts_out);

cp_status mttkrp_dense_f64(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u,
                           int mode, double* out) {
  return mttkrp_f64_impl(ctx, t, L, u, mode, out, nullptr);
}

// Split-K partial sums only (grid x I x R doubles), for a fused consumer.
cp_status mttkrp_f64_parts(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, int mode,
                           Parts* out) {
  return mttkrp_f64_impl(ctx, t, L, u, mode, nullptr, out);
}

static cp_status mttkrp_f64_impl(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u,
                                 int mode, double* out, Parts* parts_out) {
  const int R = L.R;
  const int64_t I = t->dims[mode];
  const int64_t Kb = kbar(t, mode);
  KRDesc kr;
  kr.cnt = 0;
  for (int m = 0; m < t->N; ++m) {
    if (m == mode) continue;
    kr.A[kr.cnt] = u + L.off[m];
    kr.I[kr.cnt] = t->dims[m];
    ++kr.cnt;
  }
  const int nsplit = (R + kF64RSUB - 1) / kF64RSUB;
  int64_t want = ((I * nsplit + 31) / 32) * 32;
  const int threads = (int)std::max<int64_t>(32, std::min<int64_t>(256, want));
  const int64_t ntiles = (Kb + kF64BK - 1) / kF64BK;
  const int64_t target = 2 * (int64_t)ctx->num_sms;
  const int64_t tiles_per_cta = (ntiles + target - 1) / target;
  const int grid = (int)((ntiles + tiles_per_cta - 1) / tiles_per_cta);
  double* partial = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&partial, sizeof(double) * (size_t)grid * I * R));
  const size_t smem = sizeof(double) * kF64BK * R;
  {
    TimerScope ts(ctx, 1);
    if (t->dtype == CP_DTYPE_F64)
      mttkrp_f64_kernel<double><<<grid, threads, smem, ctx->stream>>>(
          (const double*)t->Tn[mode], I, Kb, kr, R, tiles_per_cta, partial);
    else
      mttkrp_f64_kernel<float><<<grid, threads, smem, ctx->stream>>>(
          (const float*)t->Tn[mode], I, Kb, kr, R, tiles_per_cta, partial);
  }
  CP_LAUNCH_CHECK();
  if (parts_out) {
    *parts_out = Parts{partial, grid, 0};
    return CP_OK;
  }
  CP_TRY(reduce_partials(ctx, partial, grid, I * R, out));
  ws_free(ctx, partial);
  return CP_OK;
}

// ---------------------------------------------------------------------------
// FP64 dense MTTKRP that allocates nothing (cp_mttkrp_noalloc).
//
// Callers that cannot allocate device memory while they run -- code that
// enqueues work inside someone else's stream capture, real-time or serving
// loops with a fixed memory budget in which cudaMalloc may stall or fail,
// or host programs whose device memory is owned by another allocator -- can
// still run the MTTKRP: its split-K partial sums go to this file-scope device
// array instead of workspace memory.  The array is part of the library image:
// every GPU that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;   // 8 MiB
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current); the host-side symbol is not a device address.
constexpr int kMaxDevices = 64;
void* g_noalloc_addr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

cp_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("cp_mttkrp_noalloc: device %d out of range", device);
    return CP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    CP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[device] = p;
  }
  *out = g_noalloc_addr[device];
  return CP_OK;
}

}  // namespace

}  // namespace cpg

extern "C" cp_status cp_mttkrp_noalloc(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, int mode,
                                       double* out) {
  using namespace cpg;
  if (!ctx || !t || !u || !out) {
    set_error("cp_mttkrp_noalloc: null argument");
    return CP_ERR_ARG;
  }
  if (t->kind != 0) {
    set_error("cp_mttkrp_noalloc: dense tensors only");
    return CP_ERR_UNSUPPORTED;
  }
  if (t->device != ctx->device) {
    set_error("cp_mttkrp_noalloc: tensor on device %d, context on device %d", t->device, ctx->device);
    return CP_ERR_ARG;
  }
  if (R < 1 || R > CP_MAX_R || mode < 0 || mode >= t->N) {
    set_error("cp_mttkrp_noalloc: R = %d or mode = %d out of range", R, mode);
    return CP_ERR_ARG;
  }
  const int64_t I = t->dims[mode];
  const size_t per_cta = sizeof(double) * (size_t)I * R;
  if (per_cta > kNoAllocScratchBytes) {
    set_error("cp_mttkrp_noalloc: I_mode x R x 8 bytes = %zu exceeds the %zu-byte scratch", per_cta,
              kNoAllocScratchBytes);
    return CP_ERR_SHAPE;
  }
  int cur = -1;
  CP_CUDA(cudaGetDevice(&cur));
  if (cur != ctx->device) CP_CUDA(cudaSetDevice(ctx->device));
  void* scratch = nullptr;
  CP_TRY(noalloc_scratch(ctx->device, &scratch));
  Layout L;
  L.set(t->N, t->dims, R);
  const int64_t Kb = kbar(t, mode);
  KRDesc kr;
  kr.cnt = 0;
  for (int m = 0; m < t->N; ++m) {
    if (m == mode) continue;
    kr.A[kr.cnt] = u + L.off[m];
    kr.I[kr.cnt] = t->dims[m];
    ++kr.cnt;
  }
  const int nsplit = (R + kF64RSUB - 1) / kF64RSUB;
  const int64_t want = ((I * nsplit + 31) / 32) * 32;
  const int threads = (int)std::max<int64_t>(32, std::min<int64_t>(256, want));
  const int64_t ntiles = (Kb + kF64BK - 1) / kF64BK;
  const int64_t fit = (int64_t)(kNoAllocScratchBytes / per_cta);   // partial blocks that fit
  const int64_t target = std::max<int64_t>(1, std::min<int64_t>(2 * (int64_t)ctx->num_sms, fit));
  const int64_t tiles_per_cta = (ntiles + target - 1) / target;
  const int grid = (int)((ntiles + tiles_per_cta - 1) / tiles_per_cta);
  double* partial = (double*)scratch;
  const size_t smem = sizeof(double) * kF64BK * R;
  if (t->dtype == CP_DTYPE_F64)
    mttkrp_f64_kernel<double><<<grid, threads, smem, ctx->stream>>>((const double*)t->Tn[mode], I, Kb, kr, R,
                                                                     tiles_per_cta, partial);
  else
    mttkrp_f64_kernel<float><<<grid, threads, smem, ctx->stream>>>((const float*)t->Tn[mode], I, Kb, kr, R,
                                                                    tiles_per_cta, partial);
  CP_LAUNCH_CHECK();
  return reduce_parts<double>(ctx, partial, grid, I * R, out);
}
