// Host run of the shared-memory Stockham transform of the CUDA path (paper_2606_25541_b300/csrc/
// fft.cuh: fft_stages, the stages of cta_fft) for every supported length, compiled by
// tests/test_stockham_host.py. One lane does every butterfly of a stage (group size 1), so each
// stage loads all its inputs into registers before it stores any output, which is the order the
// group barrier enforces on the device. Each length runs in FP32 (element padding every 16, as
// the FP32 plane passes) and in FP64 with the plain twiddle table and, where it fits, with the
// per-stage table of build_stw; and in double-float pairs (padding every 8, as the FP64
// residual's row and column passes) with the plain table. Reference: the DFT of the same
// (rounded) input summed in long double. Prints "name value" lines.
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
#include <cstring>
#include <random>
#include <vector>

using namespace psfd;
typedef long double Q;
typedef std::complex<Q> CQ;
static const Q kPi = 3.14159265358979323846264338327950288L;

static CQ toq(double2 a) { return CQ(a.x, a.y); }
static CQ toq(float2 a) { return CQ(a.x, a.y); }
static CQ toq(dfc a) { return CQ((Q)a.x.hi + (Q)a.x.lo, (Q)a.y.hi + (Q)a.y.lo); }
template <typename C> C fromd(double re, double im);
template <> double2 fromd<double2>(double re, double im) { return make_double2(re, im); }
template <> float2 fromd<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> dfc fromd<dfc>(double re, double im) { return to_dfc(make_double2(re, im)); }

struct Outcome {
  double err;     // normwise relative error against the long-double DFT
  std::vector<unsigned char> bytes;  // the outputs, natural order, for the bitwise comparison
};

// one length-N transform of x (forward: exp(-2 pi i n k / N); INV: the conjugate kernel)
template <typename C, int N, bool INV, int RUN, bool STW>
static Outcome run(const std::vector<std::complex<double>>& x, const std::vector<double2>& t64,
                   const std::vector<float2>& t32) {
  std::vector<C> a(fft_physr<RUN>(N)), tw(N);
  for (int n = 0; n < N; ++n) a[fpadr<RUN>(n)] = fromd<C>(x[n].real(), x[n].imag());
  // the plain table's entry k in the run's format: FP32 and FP64 copies, or FP64 rounded to pairs
  auto get = [&](int k) -> C {
    if constexpr (sizeof(C) == sizeof(float2)) return t32[k];
    else return fromd<C>(t64[k].x, t64[k].y);
  };
  if constexpr (STW) {
    build_stw<C, N>(tw.data(), t64.data(), t32.data(), 1, 0, 1);
  } else {
    for (int k = 0; k < N; ++k) tw[k] = get(k);
  }
  fft_stages<C, N, 1, INV, 0, 1, 1, false, RUN, STW>(a.data(), 0, tw.data(), true, 0);
  Outcome o;
  o.bytes.resize(N * sizeof(C));
  std::vector<CQ> root(N), xin(N);
  for (int m = 0; m < N; ++m) root[m] = CQ(cosl(2 * kPi * m / N), (INV ? 1 : -1) * sinl(2 * kPi * m / N));
  for (int n = 0; n < N; ++n) xin[n] = toq(fromd<C>(x[n].real(), x[n].imag()));
  Q num = 0, den = 0;
  for (int k = 0; k < N; ++k) {
    CQ ref = 0;
    for (int n = 0; n < N; ++n) ref += xin[n] * root[(long)k * n % N];
    const C got = a[fpadr<RUN>(k)];
    std::memcpy(o.bytes.data() + k * sizeof(C), &got, sizeof(C));
    num += std::norm(toq(got) - ref);
    den += std::norm(ref);
  }
  o.err = (double)sqrtl(num / den);
  return o;
}

struct Tally {
  double worst32 = 0, worst64 = 0, worstdf = 0;
  long stw_mismatch = 0, stw_checked = 0, lengths = 0, pow2_not_fitting = 0;
};

template <int N>
static void check_length(Tally& t, std::mt19937_64& rng) {
  std::normal_distribution<double> g(0.0, 1.0);
  std::vector<double2> t64(N);
  std::vector<float2> t32(N);
  for (int k = 0; k < N; ++k) {
    const Q ang = -2 * kPi * k / N;
    t64[k] = make_double2((double)cosl(ang), (double)sinl(ang));
    t32[k] = make_float2((float)t64[k].x, (float)t64[k].y);
  }
  static_assert(stw_size(N) >= 0, "");
  if ((N & (N - 1)) == 0 && !stw_fits(N)) ++t.pow2_not_fitting;
  ++t.lengths;
  for (int trial = 0; trial < 3; ++trial) {
    std::vector<std::complex<double>> x(N);
    for (auto& v : x) v = std::complex<double>(g(rng), g(rng));
    const Outcome f32 = run<float2, N, false, 16, false>(x, t64, t32);
    const Outcome i32 = run<float2, N, true, 16, false>(x, t64, t32);
    const Outcome f64 = run<double2, N, false, 8, false>(x, t64, t32);
    const Outcome i64 = run<double2, N, true, 8, false>(x, t64, t32);
    t.worst32 = std::fmax(t.worst32, std::fmax(f32.err, i32.err));
    t.worst64 = std::fmax(t.worst64, std::fmax(f64.err, i64.err));
    const Outcome fdf = run<dfc, N, false, 8, false>(x, t64, t32);
    const Outcome idf = run<dfc, N, true, 8, false>(x, t64, t32);
    t.worstdf = std::fmax(t.worstdf, std::fmax(fdf.err, idf.err));
    if constexpr (stw_fits(N)) {
      const Outcome s[4] = {run<float2, N, false, 16, true>(x, t64, t32), run<float2, N, true, 16, true>(x, t64, t32),
                            run<double2, N, false, 8, true>(x, t64, t32), run<double2, N, true, 8, true>(x, t64, t32)};
      const Outcome* p[4] = {&f32, &i32, &f64, &i64};
      for (int i = 0; i < 4; ++i) {
        ++t.stw_checked;
        if (s[i].bytes != p[i]->bytes) ++t.stw_mismatch;
      }
    }
  }
}

int main() {
  std::mt19937_64 rng(5);
  Tally t;
  check_length<4>(t, rng);
  check_length<8>(t, rng);
  check_length<16>(t, rng);
  check_length<32>(t, rng);
  check_length<64>(t, rng);
  check_length<96>(t, rng);
  check_length<128>(t, rng);
  check_length<160>(t, rng);
  check_length<192>(t, rng);
  check_length<256>(t, rng);
  check_length<320>(t, rng);
  check_length<384>(t, rng);
  check_length<512>(t, rng);
  check_length<640>(t, rng);
  check_length<768>(t, rng);
  check_length<1024>(t, rng);
  std::printf("lengths %ld\nstockham_fp32 %.6e\nstockham_fp64 %.6e\nstockham_dfloat %.6e\nstw_checked %ld\n"
              "stw_mismatch %ld\npow2_not_fitting %ld\n",
              t.lengths, t.worst32, t.worst64, t.worstdf, t.stw_checked, t.stw_mismatch, t.pow2_not_fitting);
  return 0;
}
