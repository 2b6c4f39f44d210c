// FP64 reciprocal, quotient and square root by Newton-Raphson refinement of
// the FP32 hardware approximations.
#pragma once

namespace rq {

// Reciprocal and square root for the scalar steps of the QR sweeps.  On this
// GPU every FP64 instruction occupies an SM sub-partition's FP64 pipe for 64
// cycles and a square root plus a divide measured ~1,350 cycles, so both
// start from the FP32 hardware approximation (relative error eps < 2^-21)
// and refine it in a few FP64 instructions:
//   reciprocal: with e = 1 - x r, r (1 + e + e^2) is the truncated geometric
//     series of r / (1 - e) = 1/x, so x r' = 1 - e^3 (three instructions);
//   square root: s = x y with y ~ 1/sqrt(x), then twice s += (x - s^2) y/2
//     (Newton's step for s^2 = x with the derivative 2s replaced by the fixed
//     2/y); each step multiplies the relative error by about eps, so the
//     second leaves ~1.5 eps^3 (six instructions).
// Outside the FP32 exponent range (and for x <= 0 in the square root) they
// fall back to the FP64 operators.  The range and sign tests are integer
// operations on the bits, not FP64 compares, and so are the conversions of
// the argument to FP32 and of the seed back to FP64 (with the conversion
// instructions the Ritz step took 0.39 ms longer per eigensolve).

// |x| in [2^-99, 2^100): an integer test on the exponent field of the high
// word (no FP64 instruction), so that the FP32 seeds below stay normal.
__device__ __forceinline__ bool f32_range(double x) {
  const int e = (__double2hiint(x) >> 20) & 0x7ff;
  return e > 1023 - 100 && e < 1023 + 100;
}
// The FP32 value of x with its significand truncated to 24 bits, and the
// exact FP64 value of a normal FP32 number: the exponent field is re-biased
// (1023 against 127) and the significand shifted by 29 bits, in integer
// operations on the two words (the conversion instructions would take FP64
// issue slots on the reflector's critical chain).  For |x| in the f32_range.
__device__ __forceinline__ float f32_of(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = ((hi >> 20) & 0x7ffu) - (1023u - 127u);
  return __uint_as_float((hi & 0x80000000u) | (e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
__device__ __forceinline__ double f64_of(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = ((b >> 23) & 0xffu) + (1023u - 127u);
  return __hiloint2double((int)((b & 0x80000000u) | (e << 20) | ((b & 0x7fffffu) >> 3)),
                          (int)(b << 29));
}
__device__ __forceinline__ double rcp_nr(double x) {
  if (!f32_range(x)) return 1.0 / x;
  const double r = f64_of(__fdividef(1.0f, f32_of(x)));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double div_nr(double a, double b) {
  double r = rcp_nr(b);
  double q = a * r;
  return fma(r, fma(-b, q, a), q);   // one residual correction
}
__device__ __forceinline__ double sqrt_nr(double x) {
  if (__double2hiint(x) < 0 || !f32_range(x)) return sqrt(x);
  const double y = f64_of(rsqrtf(f32_of(x)));
  const double h = 0.5 * y;
  double s = x * y;
  s = fma(fma(-s, s, x), h, s);
  return fma(fma(-s, s, x), h, s);
}

}  // namespace rq
