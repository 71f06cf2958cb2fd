// common.cuh -- complex arithmetic and small utilities shared by the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace psfd {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };
template <typename R> using cplx = typename CT<R>::T;

template <typename C> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }
template <typename C> __host__ __device__ __forceinline__ C cneg(C a) { return mk(-a.x, -a.y); }
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
// multiply by i / -i
template <typename C> __host__ __device__ __forceinline__ C cmul_i(C a) { return mk(-a.y, a.x); }
template <typename C> __host__ __device__ __forceinline__ C cmul_mi(C a) { return mk(a.y, -a.x); }
template <typename C> __host__ __device__ __forceinline__ auto cabs2(C a) { return a.x * a.x + a.y * a.y; }

// Division by Smith's method (robust against overflow of |b|^2).
template <typename C> __host__ __device__ __forceinline__ C cdiv(C a, C b) {
  using R = typename RealOf<C>::T;
  if (fabs(b.x) >= fabs(b.y)) {
    R r = b.y / b.x;
    R d = b.x + b.y * r;
    return mk((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    R r = b.x / b.y;
    R d = b.x * r + b.y;
    return mk((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}

__host__ __device__ __forceinline__ float2 to_c32(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 to_c64(float2 a) { return make_double2(a.x, a.y); }
template <typename C> __host__ __device__ __forceinline__ C from_c64(double2 a);
template <> __host__ __device__ __forceinline__ float2 from_c64<float2>(double2 a) { return to_c32(a); }
template <> __host__ __device__ __forceinline__ double2 from_c64<double2>(double2 a) { return a; }
__host__ __device__ __forceinline__ double2 as_c64(float2 a) { return to_c64(a); }
__host__ __device__ __forceinline__ double2 as_c64(double2 a) { return a; }

// exp(z) for complex z (exp of the real part times cos/sin of the imaginary part).
__device__ __forceinline__ double2 cexp_d(double2 z) {
  double s, c;
  sincos(z.y, &s, &c);
  double e = exp(z.x);
  return make_double2(e * c, e * s);
}

// Square root on the branch Im >= 0 (outgoing / decaying wave), from
// sqrt(a + ib) = t + i b/(2t), t = sqrt((|z| + a)/2), and its mirror for a < 0.
__device__ __forceinline__ double2 csqrt_upper_d(double2 z) {
  double r = hypot(z.x, z.y);
  double2 s;
  if (r == 0.0) return make_double2(0.0, 0.0);
  if (z.x >= 0.0) {
    double t = sqrt(0.5 * (r + z.x));
    s = make_double2(t, z.y / (2.0 * t));
  } else {
    double t = sqrt(0.5 * (r - z.x));
    s = make_double2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
  }
  if (s.y < 0.0 || (s.y == 0.0 && s.x < 0.0)) s = make_double2(-s.x, -s.y);
  return s;
}

// Signed frequency of FFT bin i of an n-point transform (Nyquist bin negative).
__host__ __device__ __forceinline__ int fft_freq(int i, int n) { return (i < (n + 1) / 2) ? i : i - n; }

}  // namespace psfd
