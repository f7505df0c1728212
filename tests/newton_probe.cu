// Test probe: applies the library's Newton-refined FP64 helpers (recip_nr,
// rsqrt_nr, div_nr, sqrt_nr from csrc/newton.cuh) to arrays of inputs, so
// that a test can compare them with correctly rounded results.  Built by
// tests/test_gpu_newton.py; not part of the library.
#include <cuda_runtime.h>

#include "newton.cuh"

__global__ void newton_probe_kernel(const double* x, const double* y, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[4 * i + 0] = cpg::recip_nr(x[i]);
  out[4 * i + 1] = x[i] > 0.0 ? cpg::rsqrt_nr(x[i]) : 0.0;
  out[4 * i + 2] = cpg::div_nr(y[i], x[i]);
  out[4 * i + 3] = x[i] > 0.0 ? cpg::sqrt_nr(x[i]) : 0.0;
}

// x, y: n host doubles; out: 4 n host doubles.  Returns a cudaError_t value.
extern "C" int newton_probe(const double* x, const double* y, int n, double* out) {
  double *dx = nullptr, *dy = nullptr, *dout = nullptr;
  cudaError_t e = cudaMalloc(&dx, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * 4 * n);
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dy, y, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    newton_probe_kernel<<<(n + 255) / 256, 256>>>(dx, dy, n, dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dy);
  cudaFree(dout);
  return (int)e;
}
