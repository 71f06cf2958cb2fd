// Host check that the integer-path conversions of csrc/dfloat.cuh (to_dfr_int, to_d_int) give
// bitwise the values of the plain conversions (to_dfr_plain, to_d_plain) on seeded doubles
// over the whole FP32 range and beyond it, on round-to-nearest-even halfway cases, on values
// at the edges of the FP32 normal range, on signed zeros and on FP64 subnormals. Compiled by
// tests/test_dfloat_host.py with floating-point contraction off. Prints "name value" lines.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "dfloat.cuh"

using psfd::dfr;

static uint64_t b64(double d) {
  uint64_t b;
  std::memcpy(&b, &d, 8);
  return b;
}
static uint32_t b32(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return b;
}

int main() {
  std::mt19937_64 rng(11);
  double to_dfr_mismatch = 0, to_d_mismatch = 0, checked = 0, int_path = 0;
  auto check = [&](double x) {
    const dfr a = psfd::to_dfr_int(x), b = psfd::to_dfr_plain(x);
    checked += 1;
    if (b32(a.hi) != b32(b.hi) || b32(a.lo) != b32(b.lo)) to_dfr_mismatch += 1;
    float h;
    if (psfd::df_f32_rn(x, h)) int_path += 1;
    const double c = psfd::to_d_int(b), d = psfd::to_d_plain(b);
    if (b64(c) != b64(d) && !(std::isnan(c) && std::isnan(d))) to_d_mismatch += 1;
  };
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-160, 140);
  for (int i = 0; i < 2000000; ++i) check(u(rng) * std::ldexp(1.0, ex(rng)));
  // raw bit patterns: every exponent, random significands
  for (int i = 0; i < 1000000; ++i) {
    uint64_t bits = rng();
    double x;
    std::memcpy(&x, &bits, 8);
    if (std::isnan(x)) continue;
    check(x);
  }
  // halfway and near-halfway cases of the FP32 rounding, both parities, many exponents
  for (int e = -130; e <= 130; ++e)
    for (int k = 0; k < 64; ++k) {
      const double f = std::ldexp((double)(0x800000 + (rng() & 0x7fffff)), e - 23);
      const double half = std::ldexp(1.0, e - 24);
      for (double x : {f + half, f - half, f + half * (1 + 1e-15), f + half * (1 - 1e-15)}) {
        check(x);
        check(-x);
      }
    }
  // FP32 range edges, zeros, FP64 subnormals, the largest finite values
  for (double x : {0.0, -0.0, 1e-310, -1e-310, 4.9e-324, 1.1754943508222875e-38, 1.1754942e-38, 1.17549435e-38,
                   1.401298464324817e-45, 7.006492321624085e-46, 3.4028234663852886e+38, 3.4028235677973366e+38,
                   3.402823669209385e+38, 1e300, -1e300, 1.7976931348623157e308, (double)INFINITY, -(double)INFINITY})
    check(x);
  std::printf("to_dfr_mismatch %.0f\nto_d_mismatch %.0f\nchecked %.0f\nint_path %.0f\n", to_dfr_mismatch,
              to_d_mismatch, checked, int_path);
  return 0;
}
