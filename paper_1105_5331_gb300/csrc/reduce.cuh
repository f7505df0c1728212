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
