// Deterministic reduction of per-CTA partial sums (split-K epilogues).
#pragma once

#include "cp_internal.cuh"

namespace cpg {

// out[e] = sum_c partial[c * n + e] in FP64.  Each block owns 32 consecutive
// outputs; warp w adds the partials c = w, w + 8, ... (coalesced rows), then
// one warp adds the eight warp sums in order.  The order depends only on
// (nparts, n), so results are reproducible run to run.
template <typename TP>
__global__ void reduce_parts_kernel(const TP* __restrict__ partial, int nparts, int64_t n,
                                    double* __restrict__ out) {
  __shared__ double sh[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t e0 = (int64_t)blockIdx.x * 32; e0 < n; e0 += (int64_t)gridDim.x * 32) {
    const int64_t e = e0 + lane;
    double s = 0.0;
    if (e < n)
#pragma unroll 4
      for (int c = w; c < nparts; c += 8) s += (double)partial[(int64_t)c * n + e];
    sh[w][lane] = s;
    __syncthreads();
    if (w == 0 && e < n) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += sh[q][lane];
      out[e] = t;
    }
    __syncthreads();
  }
}

template <typename TP>
inline cp_status reduce_parts(cp_ctx* ctx, const TP* partial, int nparts, int64_t n, double* out) {
  int64_t blocks = (n + 31) / 32;
  blocks = blocks < 8 * (int64_t)ctx->num_sms ? blocks : 8 * (int64_t)ctx->num_sms;
  if (blocks < 1) blocks = 1;
  reduce_parts_kernel<TP><<<(unsigned)blocks, 256, 0, ctx->stream>>>(partial, nparts, n, out);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

}  // namespace cpg

namespace cpg {

// sum over c = c0, c0 + step, ... < count of q[c * stride], with four
// independent accumulators so that up to 16 loads are in flight (the loads
// are L2 hits; a single running sum would wait for each before issuing the
// next).  Fixed order: ((a0 + a1) + (a2 + a3)).
template <typename T>
__device__ __forceinline__ T strided_sum(const T* __restrict__ q, int c0, int count, int step, int64_t stride) {
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int c = c0;
#pragma unroll 4
  for (; c + 3 * step < count; c += 4 * step) {
    a0 += __ldcg(&q[(int64_t)c * stride]);
    a1 += __ldcg(&q[(int64_t)(c + step) * stride]);
    a2 += __ldcg(&q[(int64_t)(c + 2 * step) * stride]);
    a3 += __ldcg(&q[(int64_t)(c + 3 * step) * stride]);
  }
  for (; c < count; c += step) a0 += __ldcg(&q[(int64_t)c * stride]);
  return (a0 + a1) + (a2 + a3);
}

}  // namespace cpg
