// dfloat.cuh -- double-float arithmetic: a real number as an unevaluated sum hi + lo of two
// FP32 values (|lo| <= ulp(hi)/2), about 48 significant bits.
//
// B300 runs FP32 about sixty times faster than FP64, so the FP64 residual of the refined
// solve (Sec. 3's operator applied to the FP64 iterate) is cheaper with its z transforms and
// dyadic products in double-float than on the FP64 pipe, at 10-20 FP32 operations per FP64
// one. The algorithms are the classical error-free transformations: Knuth's TwoSum,
// Dekker's FastTwoSum, and the FMA form of TwoProduct; addition is the "sloppy" variant
// (TwoSum of the high parts, the low parts added once), whose error is bounded by a few
// 2^-48 (|a| + |b|): normwise accuracy, which is what a transform needs.
//
// The complex type dfc has members x, y and an mk() overload, so the generic complex helpers
// and the register FFT instantiate with it unchanged.
#pragma once

#include "common.cuh"

namespace psfd {

struct dfr {
  float hi, lo;
  dfr() = default;
  // nearest double-float of a double: exact for literals folded at compile time
  __host__ __device__ constexpr dfr(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr dfr(float h, float l) : hi(h), lo(l) {}
};

struct __align__(16) dfc {
  dfr x, y;
};

template <> struct RealOf<dfc> { using T = dfr; };

__host__ __device__ __forceinline__ dfc mk(dfr a, dfr b) {
  dfc c;
  c.x = a;
  c.y = b;
  return c;
}

// Rounded FP32 operations that the compiler may not fuse into an FMA: the error-free
// transformations below need every sum and product rounded exactly once. (On the host the
// plain operators serve, compiled without floating-point contraction.)
__host__ __device__ __forceinline__ float df_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float df_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float df_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

// s + e = a + b exactly (no magnitude condition)
__host__ __device__ __forceinline__ dfr df_two_sum(float a, float b) {
  const float s = df_add(a, b);
  const float bb = df_sub(s, a);
  const float e = df_add(df_sub(a, df_sub(s, bb)), df_sub(b, bb));
  return dfr(s, e);
}
// s + e = a + b exactly, given |a| >= |b| or a = 0
__host__ __device__ __forceinline__ dfr df_fast_two_sum(float a, float b) {
  const float s = df_add(a, b);
  return dfr(s, df_sub(b, df_sub(s, a)));
}

__host__ __device__ __forceinline__ dfr operator+(dfr a, dfr b) {
  const dfr s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, df_add(s.lo, df_add(a.lo, b.lo)));
}
__host__ __device__ __forceinline__ dfr operator-(dfr a) { return dfr(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dfr operator-(dfr a, dfr b) { return a + (-b); }
// TwoProduct by FMA: p + e = a.hi b.hi exactly, then the cross terms (a.lo b.lo is below
// the format's precision)
__host__ __device__ __forceinline__ dfr operator*(dfr a, dfr b) {
  const float p = df_mul(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// conversions from and to FP64 (one FP64 subtraction or addition per real)
__host__ __device__ __forceinline__ dfr to_dfr(double d) {
  const float h = (float)d;
  return dfr(h, (float)(d - (double)h));
}
__host__ __device__ __forceinline__ dfc to_dfc(double2 v) { return mk(to_dfr(v.x), to_dfr(v.y)); }
__host__ __device__ __forceinline__ double to_d(dfr a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ double2 to_d2(dfc a) { return make_double2(to_d(a.x), to_d(a.y)); }

}  // namespace psfd
