// FP64 reciprocal, quotient and square root by Newton-Raphson refinement of
// the FP32 hardware approximations.
#pragma once

namespace rq {

// Reciprocal and square root for the scalar steps of the QR sweeps.  On this
// GPU every FP64 instruction occupies an SM sub-partition's FP64 pipe for 64
// cycles and a square root plus a divide measured ~1,350 cycles, so both
// start from the FP32 hardware approximation and apply Newton-Raphson steps in
// FP64 (quadratic convergence): two steps for the reciprocal, one step plus a
// residual correction for the square root.  Outside the FP32 exponent range
// they fall back to the FP64 operators.

// |x| in [2^-99, 2^100): an integer test on the exponent field of the high
// word (no FP64 instruction), so that the FP32 seeds below stay normal.
__device__ __forceinline__ bool f32_range(double x) {
  const int e = (__double2hiint(x) >> 20) & 0x7ff;
  return e > 1023 - 100 && e < 1023 + 100;
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
// One Newton step on the FP32 reciprocal square root (relative error about
// 1.5 e0^2 < 2^-41 from e0 < 2^-21), then sqrt(x) = x y with one residual
// correction s + (y/2)(x - s^2), which squares the error again.
__device__ __forceinline__ double sqrt_nr(double x) {
  if (!(x > 0.0) || !f32_range(x)) return sqrt(x);
  double y = (double)rsqrtf((float)x);         // ~ 1/sqrt(x)
  y = y * fma(-0.5 * x * y, y, 1.5);           // y <- y (3 - x y^2) / 2
  double s = x * y;
  return fma(0.5 * y, fma(-s, s, x), s);
}

}  // namespace rq
