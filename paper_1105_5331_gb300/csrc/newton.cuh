// FP64 reciprocal, reciprocal square root, quotient and square root from FP32
// hardware seeds refined by Newton-Raphson steps.  On this GPU an FP64
// divide or sqrt is a serial chain of about 650 cycles (a dependent FMA 64);
// two Newton steps from the 23-bit FP32 seed (each doubles the correct bits)
// cost 4-6 FMAs.  Results are within a few ulps of the IEEE operations.
// Outside the FP32 exponent range the IEEE operation is used.
#pragma once

namespace cpg {

// 1/d:  r <- r + r (1 - d r)
__device__ __forceinline__ double recip_nr(double d) {
  const double ad = fabs(d);
  if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
  double r = (double)__frcp_rn((float)d);
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

// 1/sqrt(s) for s > 0:  y <- y (3/2 - s y^2 / 2)
__device__ __forceinline__ double rsqrt_nr(double s) {
  if (!(s > 1e-30 && s < 1e30)) return 1.0 / sqrt(s);
  double y = (double)rsqrtf((float)s);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double h = 0.5 * s * y;
    y = y * fma(-h, y, 1.5);
  }
  return y;
}

__device__ __forceinline__ double div_nr(double x, double y) { return x * recip_nr(y); }

__device__ __forceinline__ double sqrt_nr(double s) {
  if (!(s > 1e-30 && s < 1e30)) return sqrt(s);
  return s * rsqrt_nr(s);
}

}  // namespace cpg
