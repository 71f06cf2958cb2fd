// Host check of the double-float primitives of the CUDA path (paper_2606_25541_b300/csrc/
// dfloat.cuh), compiled by tests/test_dfloat_host.py with floating-point contraction off.
// Reference arithmetic: long double (64-bit significand), exact for the sums and products of
// two FP32 numbers that the error-free transformations claim to represent.
// Prints "name value" lines; the test compares them with the bounds it states.
#include <cmath>
#include <cstdio>
#include <random>

#include "dfloat.cuh"

using psfd::dfr;
typedef long double Q;

static Q q(dfr a) { return (Q)a.hi + (Q)a.lo; }

int main() {
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  double conv = 0, add = 0, mul = 0, unnormalised = 0, two_sum_inexact = 0, two_prod_inexact = 0;
  for (int i = 0; i < 1000000; ++i) {
    const double x = u(rng) * std::ldexp(1.0, (int)(u(rng) * 30));
    double y = u(rng) * std::ldexp(1.0, (int)(u(rng) * 30));
    if (i % 4 == 0) y = -x * (1.0 + u(rng) * 1e-6);  // near cancellation
    const dfr a = psfd::to_dfr(x), b = psfd::to_dfr(y);
    conv = std::fmax(conv, (double)(fabsl(q(a) - (Q)x) / fabsl((Q)x)));
    const dfr s = a + b, p = a * b;
    add = std::fmax(add, (double)(fabsl(q(s) - (q(a) + q(b))) / (fabsl(q(a)) + fabsl(q(b)))));
    mul = std::fmax(mul, (double)(fabsl(q(p) - q(a) * q(b)) / fabsl(q(a) * q(b))));
    if (std::fabs(s.lo) > std::ldexp(std::fabs(s.hi), -24) || std::fabs(p.lo) > std::ldexp(std::fabs(p.hi), -24))
      unnormalised += 1;
    // the error-free transformations themselves: exact in long double
    const float fa = (float)x, fb = (float)y;
    const dfr ts = psfd::df_two_sum(fa, fb);
    if ((Q)ts.hi + (Q)ts.lo != (Q)fa + (Q)fb) two_sum_inexact += 1;
    const float pp = fa * fb;
    const float pe = std::fmaf(fa, fb, -pp);
    if ((Q)pp + (Q)pe != (Q)fa * (Q)fb) two_prod_inexact += 1;
  }
  constexpr dfr h(0.70710678118654752440);
  const double cst = (double)fabsl(q(h) - 0.70710678118654752440L) / 0.70710678118654752440;
  std::printf("conv %.6e\nadd %.6e\nmul %.6e\nunnormalised %.0f\ntwo_sum_inexact %.0f\ntwo_prod_inexact %.0f\n"
              "constant %.6e\n",
              conv, add, mul, unnormalised, two_sum_inexact, two_prod_inexact, cst);
  return 0;
}
