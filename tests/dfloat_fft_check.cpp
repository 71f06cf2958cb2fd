// Host run of the register four-step transform of the CUDA path (paper_2606_25541_b300/csrc/
// fft.cuh: reg_fft_step1 / reg_fft_step2, 16 x nf/16) in double-float and in FP64, compiled by
// tests/test_dfloat_host.py. The nf/16 lanes of a group run one after the other (step 1 of every
// lane, then step 2), which is the order the warp's __syncwarp enforces on the device; the
// device-only names the header uses are given host stand-ins below. Reference: the DFT summed in
// long double. Prints "name value" lines (normwise relative errors).
#define _GNU_SOURCE 1
#include <cmath>
#include <math.h>
using std::copysign;
using std::exp;
using std::fabs;
using std::hypot;
using std::sqrt;
struct HostDim {
  unsigned x, y, z;
};
static HostDim threadIdx{0, 0, 0}, blockDim{1, 1, 1};
#define __syncwarp(...) ((void)0)
#include "fft.cuh"
#include "dfloat.cuh"

#include <complex>
#include <cstdio>
#include <random>
#include <vector>

using namespace psfd;
typedef long double Q;
typedef std::complex<Q> CQ;

static CQ toq(dfc a) { return CQ((Q)a.x.hi + (Q)a.x.lo, (Q)a.y.hi + (Q)a.y.lo); }
static CQ toq(double2 a) { return CQ(a.x, a.y); }
template <typename C> C fromd(double re, double im);
template <> dfc fromd<dfc>(double re, double im) { return to_dfc(make_double2(re, im)); }
template <> double2 fromd<double2>(double re, double im) { return make_double2(re, im); }

// one length-NF transform of x (half: x[n] = 0 for n >= NF/2) through the two register steps
template <typename C, int NF, bool INV, bool HALF>
static double run(const std::vector<std::complex<double>>& x) {
  constexpr int N2 = NF / 16, R1 = 16 / N2, EP = N2 + 1;
  std::vector<C> tw(NF), ex(16 * EP);
  for (int t = 0; t < NF; ++t) {
    const Q a = -2.0L * 3.14159265358979323846264338327950288L * t / NF;
    tw[t] = fromd<C>((double)cosl(a), (double)sinl(a));
  }
  for (int j = 0; j < N2; ++j) {
    C v[16];
    for (int k = 0; k < 16; ++k) {
      const int n = j + N2 * k;
      v[k] = (HALF && k >= 8) ? fromd<C>(0.0, 0.0) : fromd<C>(x[n].real(), x[n].imag());
    }
    reg_fft_step1<C, NF, INV, HALF>(v, j, tw.data());
    for (int k1 = 0; k1 < 16; ++k1) ex[k1 * EP + j] = v[k1];
  }
  std::vector<CQ> got(NF);
  for (int j = 0; j < N2; ++j) {
    C o[16];
    reg_fft_step2<C, NF, INV, EP>(ex.data(), j, o);
    for (int r = 0; r < R1; ++r)
      for (int k2 = 0; k2 < N2; ++k2) got[j + N2 * r + 16 * k2] = toq(o[r * N2 + k2]);
  }
  Q num = 0, den = 0;
  const Q sgn = INV ? 1.0L : -1.0L;
  for (int k = 0; k < NF; ++k) {
    CQ ref = 0;
    for (int n = 0; n < NF; ++n) {
      if (HALF && n >= NF / 2) continue;
      const Q a = sgn * 2.0L * 3.14159265358979323846264338327950288L * (Q)((long)k * n % NF) / NF;
      ref += CQ(x[n].real(), x[n].imag()) * CQ(cosl(a), sinl(a));
    }
    num += std::norm(got[k] - ref);
    den += std::norm(ref);
  }
  return (double)sqrtl(num / den);
}

int main() {
  std::mt19937_64 rng(3);
  std::normal_distribution<double> g(0.0, 1.0);
  std::vector<std::complex<double>> x(128);
  double worst_df = 0, worst_f64 = 0;
  for (int trial = 0; trial < 20; ++trial) {
    const double scale = std::ldexp(1.0, (int)(g(rng) * 10));
    for (auto& v : x) v = std::complex<double>(g(rng), g(rng)) * scale;
    worst_df = std::fmax(worst_df, run<dfc, 128, false, true>(x));
    worst_df = std::fmax(worst_df, run<dfc, 128, true, false>(x));
    worst_df = std::fmax(worst_df, run<dfc, 64, false, true>(x));
    worst_df = std::fmax(worst_df, run<dfc, 64, true, false>(x));
    worst_f64 = std::fmax(worst_f64, run<double2, 128, false, true>(x));
    worst_f64 = std::fmax(worst_f64, run<double2, 128, true, false>(x));
    worst_f64 = std::fmax(worst_f64, run<double2, 64, true, false>(x));
  }
  std::printf("fft_dfloat %.6e\nfft_fp64 %.6e\n", worst_df, worst_f64);
  return 0;
}
