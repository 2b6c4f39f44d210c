// FP64 reciprocal, quotient and square root by Newton-Raphson refinement of
// the FP32 hardware approximations.
#pragma once

namespace rq {

// Reciprocal and square root for the scalar steps of the QR sweeps.  On this
// GPU every FP64 instruction occupies an SM sub-partition's FP64 pipe for 64
// cycles and a square root plus a divide measured ~1,350 cycles, so both
// start from the FP32 hardware approximation and apply Newton-Raphson steps in
// FP64 (quadratic convergence: two steps from 24 bits exceed 53 bits), plus
// one residual correction.  Outside the FP32 exponent range they fall back to
// the FP64 operators.
__device__ __forceinline__ bool f32_range(double x) {
  double a = fabs(x);
  return a > 1e-30 && a < 1e30;
}
__device__ __forceinline__ double rcp_nr(double x) {
  if (!f32_range(x)) return 1.0 / x;
  double r = (double)(1.0f / (float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ double div_nr(double a, double b) {
  double r = rcp_nr(b);
  double q = a * r;
  return fma(r, fma(-b, q, a), q);   // one residual correction
}
__device__ __forceinline__ double sqrt_nr(double x) {
  if (!(x > 1e-30 && x < 1e30)) return sqrt(x);
  double y = (double)rsqrtf((float)x);         // ~ 1/sqrt(x)
  y = y * fma(-0.5 * x * y, y, 1.5);           // y <- y (3 - x y^2) / 2
  y = y * fma(-0.5 * x * y, y, 1.5);
  double s = x * y;                            // sqrt(x), then one residual correction
  return fma(0.5 * y, fma(-s, s, x), s);
}

}  // namespace rq
