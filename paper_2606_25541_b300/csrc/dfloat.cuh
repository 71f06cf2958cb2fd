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

#include <cstring>

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

// Conversions from and to FP64. On B300 the FP64 pipe, which also runs the FP64 <-> FP32
// conversion instructions, issues about two operations per SM and clock, so a conversion
// done with conversion instructions (three of them and one FP64 subtraction per real) can cost
// more than the transform it feeds. The integer forms below do the exponent rebias and the
// round-to-nearest-even of the significand with integer operations and keep one exact FP64
// addition or subtraction per real; they give bitwise the values of the plain conversions
// (every zero or FP32-normal operand; anything else takes the plain route).
__host__ __device__ __forceinline__ unsigned long long df_dbits(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long b;
  std::memcpy(&b, &d, sizeof(b));
  return b;
#endif
}
__host__ __device__ __forceinline__ double df_bdouble(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  std::memcpy(&d, &b, sizeof(d));
  return d;
#endif
}
__host__ __device__ __forceinline__ unsigned df_fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  std::memcpy(&u, &f, sizeof(u));
  return u;
#endif
}
__host__ __device__ __forceinline__ float df_bfloat(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof(f));
  return f;
#endif
}

// FP32 round-to-nearest-even of d by integer operations, when d is zero or rounds to a normal
// FP32 number from the normal FP32 exponent range; false otherwise.
__host__ __device__ __forceinline__ bool df_f32_rn(double d, float& out) {
  const unsigned long long b = df_dbits(d);
  const unsigned s = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long mag = b & 0x7fffffffffffffffull;
  if (mag == 0) {
    out = df_bfloat(s);
    return true;
  }
  const int e = (int)(mag >> 52);
  if (e < 897 || e > 1150) return false;  // FP32 exponent field 1 .. 254 (bias 127 against 1023)
  const unsigned long long t = mag - (896ull << 52);
  unsigned q = (unsigned)(t >> 29);  // exponent field and the top 23 significand bits
  const unsigned rem = (unsigned)t & 0x1fffffffu;
  if (rem > 0x10000000u || (rem == 0x10000000u && (q & 1u))) ++q;  // a carry moves into the exponent
  if (q >= 0x7f800000u) return false;                                // rounded to infinity
  out = df_bfloat(q | s);
  return true;
}
// The FP64 value of a zero or normal FP32 number (exact) by integer operations; false for
// subnormal, infinite or NaN operands.
__host__ __device__ __forceinline__ bool df_f64_of(float f, double& out) {
  const unsigned u = df_fbits(f);
  const unsigned em = u & 0x7fffffffu;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  if (em == 0) {
    out = df_bdouble(s);
    return true;
  }
  if (em < 0x00800000u || em >= 0x7f800000u) return false;
  out = df_bdouble(s | (((unsigned long long)em << 29) + (896ull << 52)));
  return true;
}

// hi = RN(d), lo = RN(d - hi) (d - hi is exact in FP64)
__host__ __device__ __forceinline__ dfr to_dfr_plain(double d) {
  const float h = (float)d;
  return dfr(h, (float)(d - (double)h));
}
__host__ __device__ __forceinline__ dfr to_dfr_int(double d) {
  float h, l;
  double hd;
  if (df_f32_rn(d, h) && df_f64_of(h, hd)) {
    const double r = d - hd;
    if (df_f32_rn(r, l)) return dfr(h, l);
    return dfr(h, (float)r);
  }
  return to_dfr_plain(d);
}
__host__ __device__ __forceinline__ double to_d_plain(dfr a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ double to_d_int(dfr a) {
  double h, l;
  if (df_f64_of(a.hi, h) && df_f64_of(a.lo, l)) return h + l;
  return to_d_plain(a);
}

__host__ __device__ __forceinline__ dfr to_dfr(double d) {
#ifdef __CUDA_ARCH__
  return to_dfr_int(d);
#else
  return to_dfr_plain(d);
#endif
}
__host__ __device__ __forceinline__ dfc to_dfc(double2 v) { return mk(to_dfr(v.x), to_dfr(v.y)); }
__host__ __device__ __forceinline__ double to_d(dfr a) {
#ifdef __CUDA_ARCH__
  return to_d_int(a);
#else
  return to_d_plain(a);
#endif
}
__host__ __device__ __forceinline__ double2 to_d2(dfc a) { return make_double2(to_d(a.x), to_d(a.y)); }

// Pairs stored as float4 (re.hi, re.lo, im.hi, im.lo) / float2 (hi, lo) in device tables.
__host__ __device__ __forceinline__ dfc dfc_of(float4 v) { return mk(dfr(v.x, v.y), dfr(v.z, v.w)); }
__host__ __device__ __forceinline__ dfr dfr_of(float2 v) { return dfr(v.x, v.y); }

}  // namespace psfd
