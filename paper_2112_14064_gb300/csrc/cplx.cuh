// Complex FP64 scalar of the complex-shift factorisation (Q(s) = K + s C +
// s^2 M with s in C is complex symmetric): the multifrontal kernels are
// templates on the scalar type and are instantiated for float, double and
// this type.  Helpers give each scalar type its pivot test, its parts and
// the real type of the operator outputs.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace rq {

struct __align__(16) zd {
  double re, im;
  zd() = default;
  __host__ __device__ constexpr zd(double r, double i = 0.0) : re(r), im(i) {}
};

__host__ __device__ inline zd operator+(zd a, zd b) { return zd(a.re + b.re, a.im + b.im); }
__host__ __device__ inline zd operator-(zd a, zd b) { return zd(a.re - b.re, a.im - b.im); }
__host__ __device__ inline zd operator-(zd a) { return zd(-a.re, -a.im); }
__host__ __device__ inline zd operator*(zd a, zd b) {
  return zd(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__host__ __device__ inline zd operator*(zd a, double b) { return zd(a.re * b, a.im * b); }
__host__ __device__ inline zd operator*(double a, zd b) { return zd(a * b.re, a * b.im); }
// a / b by Smith's scaling (no overflow of |b|^2)
__host__ __device__ inline zd operator/(zd a, zd b) {
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return zd((a.re + a.im * r) / d, (a.im - a.re * r) / d);
  }
  const double r = b.re / b.im, d = b.im + b.re * r;
  return zd((a.re * r + a.im) / d, (a.im * r - a.re) / d);
}
__host__ __device__ inline zd& operator+=(zd& a, zd b) { a = a + b; return a; }
__host__ __device__ inline zd& operator-=(zd& a, zd b) { a = a - b; return a; }
__host__ __device__ inline zd& operator*=(zd& a, zd b) { a = a * b; return a; }
__host__ __device__ inline bool operator==(zd a, zd b) { return a.re == b.re && a.im == b.im; }
__host__ __device__ inline bool operator!=(zd a, zd b) { return !(a == b); }

#ifdef __CUDACC__
// the overloads below join CUDA's own (kept visible inside this namespace)
using ::__ldcg;
using ::__shfl_sync;
__device__ __forceinline__ zd __ldcg(const zd* p) {
  const double2 v = ::__ldcg(reinterpret_cast<const double2*>(p));
  return zd(v.x, v.y);
}
__device__ __forceinline__ zd __shfl_sync(unsigned mask, zd v, int src) {
  return zd(::__shfl_sync(mask, v.re, src), ::__shfl_sync(mask, v.im, src));
}
#endif

// real type of a scalar type (the operator's vectors stay real)
template <class T>
struct RealOf {
  using type = T;
};
template <>
struct RealOf<zd> {
  using type = double;
};

// pivot test: SPD (d > 0), indefinite (d != 0, finite), complex (|d| > 0, finite)
template <class T>
__host__ __device__ inline bool pivot_bad(T d, int indef) {
  return indef ? !(d != T(0) && isfinite((double)d)) : !(d > T(0));
}
template <>
__host__ __device__ inline bool pivot_bad<zd>(zd d, int) {
  return !(isfinite(d.re) && isfinite(d.im) && (d.re != 0.0 || d.im != 0.0));
}
template <class T>
__host__ __device__ inline bool pivot_negative(T d) { return d < T(0); }
template <>
__host__ __device__ inline bool pivot_negative<zd>(zd) { return false; }

// the scalar re + i im (the imaginary part dropped for real types)
template <class T>
__host__ __device__ inline T from_parts(double re, double) { return T(re); }
template <>
__host__ __device__ inline zd from_parts<zd>(double re, double im) { return zd(re, im); }

}  // namespace rq
