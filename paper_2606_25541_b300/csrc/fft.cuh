// fft.cuh -- mixed-radix Stockham FFT on shared memory, executed by groups of lanes
// inside one warp.
//
// Sec. 3 of the paper evaluates every derivative / convolution with FFTs (Eqs. (6),
// (18)); this is the project's own transform. A length-N transform is carried out by a
// group of G lanes of one warp (G divides 32) on data that already sits in shared
// memory with element stride `es`. Each stage of radix R loads R elements per
// butterfly into registers, applies the twiddles, does the radix-R DFT in registers,
// and writes the results in self-sorting (Stockham) order, so that the output is in
// natural order without a bit-reversal pass. Stages are separated by __syncwarp only:
// warps progress independently. Radices: 8 first, then 4, 2, 3, 5.
//
// Twiddles come from a table tw[t] = exp(-2 pi i t / N), t < N, prepared in FP64 on
// the host and placed in shared memory by the caller. Forward transforms use
// exp(-i ...); inverse transforms are unnormalised.
#pragma once

#include "common.cuh"

namespace psfd {

__host__ __device__ constexpr int fft_plan_radix(int n, int stage) {
  int s = 0;
  while (n % 8 == 0 && n >= 8) { if (s == stage) return 8; n /= 8; ++s; }
  while (n % 4 == 0) { if (s == stage) return 4; n /= 4; ++s; }
  while (n % 2 == 0) { if (s == stage) return 2; n /= 2; ++s; }
  while (n % 3 == 0) { if (s == stage) return 3; n /= 3; ++s; }
  while (n % 5 == 0) { if (s == stage) return 5; n /= 5; ++s; }
  return 0;
}

__host__ __device__ constexpr int fft_plan_stages(int n) {
  int s = 0;
  while (fft_plan_radix(n, s) != 0) ++s;
  return s;
}

// Per-stage twiddle table of the plan of length n. A Stockham stage of radix R after stages
// whose radices multiply to NS > 1 multiplies input r of butterfly b by w_n^{r j TWS},
// j = b mod NS, TWS = n / (NS R). In the plain table those reads are strided by r j TWS, and
// the lanes of a stage meet bank conflicts; here row j of the stage holds its R - 1 twiddles
// contiguously, rows of odd length (R - 1) | 1, so that lanes reading consecutive rows hit
// distinct banks. Same values as the plain table; every offset is a compile-time constant
// (offsets computed in the stage loop at run time cost more than the conflicts they remove).
__host__ __device__ constexpr int stw_stride(int n, int stage) {
  int ns = 1;
  for (int s = 0; s < stage; ++s) ns *= fft_plan_radix(n, s);
  return ns;
}
__host__ __device__ constexpr int stw_count(int n, int stage) {
  return stw_stride(n, stage) > 1 ? stw_stride(n, stage) * ((fft_plan_radix(n, stage) - 1) | 1) : 0;
}
__host__ __device__ constexpr int stw_offset(int n, int stage) {
  int o = 0;
  for (int s = 0; s < stage; ++s) o += stw_count(n, s);
  return o;
}
__host__ __device__ constexpr int stw_size(int n) { return stw_offset(n, fft_plan_stages(n)); }
// Whether the staged table fits where the plain one (n entries) sits: every power-of-two plan.
__host__ __device__ constexpr bool stw_fits(int n) { return stw_size(n) <= n; }

// Shared-memory layout of a transform: element i sits at fpad(i) = i + i/8 (times the
// element stride), one spare slot after every eight elements. Without it the first
// radix-8 stage stores with a stride of eight elements and eight lanes of a half-warp
// hit the same bank pair; with it every stage's loads and stores are (nearly)
// conflict free. A transform of length n occupies fft_phys(n) slots.
__host__ __device__ constexpr int fft_phys(int n) { return n + (n >> 3); }
__host__ __device__ __forceinline__ int fpad(int i) { return i + (i >> 3); }
// The same with one spare slot after every RUN elements (RUN = 8 is the layout above). With
// RUN = 16 a 16-lane memory phase reading 16 consecutive elements stays inside one run and
// hits 16 different banks, while stores with a stride of eight elements still spread.
template <int RUN> __host__ __device__ constexpr int fft_physr(int n) { return n + n / RUN; }
template <int RUN> __host__ __device__ __forceinline__ int fpadr(int i) { return i + i / RUN; }

// Lanes per transform: N/8 rounded down to a power of two, clamped to [1, 32] up to
// N = 512. Longer transforms span several warps (64 lanes, or 128 in FP64) so that a lane
// holds at most 16 complex values per stage; such groups synchronise with a named barrier.
template <typename C>
__host__ __device__ constexpr int fft_group_lanes(int n) {
  const int cap = sizeof(C) == 16 ? (n <= 512 ? 32 : 128) : (n <= 256 ? 32 : 128);
  int g = 1;
  while (g * 2 <= n / 8 && g * 2 <= cap) g *= 2;
  return g;
}

// Barrier between the load and store phases of a stage: the warp, or the G threads of a
// multi-warp group (named barrier `bar`, 1..15).
template <int G>
__device__ __forceinline__ void group_sync(int bar) {
  if constexpr (G <= 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(G) : "memory");
  }
}

// ---------------------------------------------------------------------------
// radix-R DFTs in registers (forward: exp(-2 pi i r k / R); INV: conjugate kernel)
// ---------------------------------------------------------------------------
template <typename C, bool INV>
__device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  C t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = csub(v1, v3);
  t3 = INV ? cmul_i(t3) : cmul_mi(t3);
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

template <typename C, int R, bool INV> struct Dft;

template <typename C, bool INV> struct Dft<C, 2, INV> {
  __device__ __forceinline__ static void run(C* v) { dft2<C, INV>(v[0], v[1]); }
};

template <typename C, bool INV> struct Dft<C, 4, INV> {
  __device__ __forceinline__ static void run(C* v) { dft4<C, INV>(v[0], v[1], v[2], v[3]); }
};

template <typename C, bool INV> struct Dft<C, 8, INV> {
  __device__ __forceinline__ static void run(C* v) {
    using R = typename RealOf<C>::T;
    const R h = (R)0.70710678118654752440;  // 1/sqrt(2)
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<C, INV>(e0, e1, e2, e3);
    dft4<C, INV>(o0, o1, o2, o3);
    // o_k *= exp(-+ i pi k / 4)
    if (INV) {
      o1 = mk((o1.x - o1.y) * h, (o1.x + o1.y) * h);
      o2 = cmul_i(o2);
      o3 = mk(-(o3.x + o3.y) * h, (o3.x - o3.y) * h);
    } else {
      o1 = mk((o1.x + o1.y) * h, (o1.y - o1.x) * h);
      o2 = cmul_mi(o2);
      o3 = mk((o3.y - o3.x) * h, -(o3.x + o3.y) * h);
    }
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
  }
};

template <typename C, bool INV> struct Dft<C, 3, INV> {
  __device__ __forceinline__ static void run(C* v) {
    using R = typename RealOf<C>::T;
    const R c = (R)-0.5;
    const R s = (R)0.86602540378443864676;  // sin(2 pi / 3)
    C t = cadd(v[1], v[2]);
    C u = csub(v[1], v[2]);
    C m = mk(v[0].x + c * t.x, v[0].y + c * t.y);
    C su = cscale(u, s);
    C isu = INV ? cmul_i(su) : cmul_mi(su);  // -+ i s u
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, isu);
    v[2] = csub(m, isu);
  }
};

template <typename C, bool INV> struct Dft<C, 5, INV> {
  __device__ __forceinline__ static void run(C* v) {
    using R = typename RealOf<C>::T;
    const R c1 = (R)0.30901699437494742410;   // cos(2 pi / 5)
    const R c2 = (R)-0.80901699437494742410;  // cos(4 pi / 5)
    const R s1 = (R)0.95105651629515357212;   // sin(2 pi / 5)
    const R s2 = (R)0.58778525229247312917;   // sin(4 pi / 5)
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C u1 = csub(v[1], v[4]), u2 = csub(v[2], v[3]);
    C a1 = mk(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    C a2 = mk(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    C b1 = mk(s1 * u1.x + s2 * u2.x, s1 * u1.y + s2 * u2.y);
    C b2 = mk(s2 * u1.x - s1 * u2.x, s2 * u1.y - s1 * u2.y);
    C ib1 = INV ? cmul_i(b1) : cmul_mi(b1);  // -+ i b1
    C ib2 = INV ? cmul_i(b2) : cmul_mi(b2);
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, ib1);
    v[4] = csub(a1, ib1);
    v[2] = cadd(a2, ib2);
    v[3] = csub(a2, ib2);
  }
};

// 10-point DFT as two 5-point DFTs of the even and odd inputs combined with w_10^k.
template <typename C, bool INV> struct Dft<C, 10, INV> {
  __device__ __forceinline__ static void run(C* v) {
    using R = typename RealOf<C>::T;
    C e[5] = {v[0], v[2], v[4], v[6], v[8]};
    C o[5] = {v[1], v[3], v[5], v[7], v[9]};
    Dft<C, 5, INV>::run(e);
    Dft<C, 5, INV>::run(o);
    const R c36 = (R)0.80901699437494742410, s36 = (R)0.58778525229247312917;
    const R c72 = (R)0.30901699437494742410, s72 = (R)0.95105651629515357212;
    const R sg = INV ? (R)1 : (R)-1;  // w_10^k = exp(-+ 2 pi i k / 10)
    const C w[5] = {mk((R)1, (R)0), mk(c36, sg * s36), mk(c72, sg * s72), mk(-c72, sg * s72), mk(-c36, sg * s36)};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const C t = k ? cmul(o[k], w[k]) : o[k];
      v[k] = cadd(e[k], t);
      v[k + 5] = csub(e[k], t);
    }
  }
};

// Radix-R DFT of inputs whose upper half is zero (v[r] = 0 for r >= R/2; only v[0..R/2)
// are read), as the first stage of a transform whose input is zero on [N/2, N).
template <typename C, int R, bool INV> struct DftHalf;

template <typename C, bool INV> struct DftHalf<C, 2, INV> {
  __device__ __forceinline__ static void run(C* v) { v[1] = v[0]; }
};

template <typename C, bool INV> struct DftHalf<C, 4, INV> {
  __device__ __forceinline__ static void run(C* v) {
    const C a = v[0], b = v[1];
    const C jb = INV ? cmul_i(b) : cmul_mi(b);  // exp(-+ i pi / 2) b
    v[0] = cadd(a, b);
    v[1] = cadd(a, jb);
    v[2] = csub(a, b);
    v[3] = csub(a, jb);
  }
};

// X[2j] = DFT4(v)[j], X[2j+1] = DFT4(v_n w8^n)[j] for the four nonzero inputs.
template <typename C, bool INV> struct DftHalf<C, 8, INV> {
  __device__ __forceinline__ static void run(C* v) {
    using R = typename RealOf<C>::T;
    const R h = (R)0.70710678118654752440;  // 1/sqrt(2)
    C e0 = v[0], e1 = v[1], e2 = v[2], e3 = v[3];
    C o0 = v[0], o1, o2, o3;
    if (INV) {
      o1 = mk((v[1].x - v[1].y) * h, (v[1].x + v[1].y) * h);
      o2 = cmul_i(v[2]);
      o3 = mk(-(v[3].x + v[3].y) * h, (v[3].x - v[3].y) * h);
    } else {
      o1 = mk((v[1].x + v[1].y) * h, (v[1].y - v[1].x) * h);
      o2 = cmul_mi(v[2]);
      o3 = mk((v[3].y - v[3].x) * h, -(v[3].x + v[3].y) * h);
    }
    dft4<C, INV>(e0, e1, e2, e3);
    dft4<C, INV>(o0, o1, o2, o3);
    v[0] = e0; v[2] = e1; v[4] = e2; v[6] = e3;
    v[1] = o0; v[3] = o1; v[5] = o2; v[7] = o3;
  }
};

// v * exp(-+ 2 pi i e / 16) for a compile-time e (after unrolling), INV: conjugate.
template <typename C, bool INV>
__device__ __forceinline__ C mulw16(C v, int e) {
  using R = typename RealOf<C>::T;
  e &= 15;
  if (e == 0) return v;
  if (e == 4) return INV ? cmul_i(v) : cmul_mi(v);
  if (e == 8) return cneg(v);
  if (e == 12) return INV ? cmul_mi(v) : cmul_i(v);
  // cos and sin of 2 pi e / 16 from c(r) = cos(r pi / 8), r = 1, 2, 3 (e is not a multiple of 4)
  auto c = [](int r) -> R {
    return r == 1 ? (R)0.92387953251128675613 : (r == 2 ? (R)0.70710678118654752440 : (R)0.38268343236508977173);
  };
  const int q = e >> 2, r = e & 3;
  R cs = q == 0 ? c(r) : (q == 1 ? -c(4 - r) : (q == 2 ? -c(r) : c(4 - r)));
  R sn = q == 0 ? c(4 - r) : (q == 1 ? c(r) : (q == 2 ? -c(4 - r) : -c(r)));
  if (!INV) sn = -sn;
  return cmul(v, mk(cs, sn));
}

// 16-point DFT in registers as 4 x 4: v[n2 + 4 n1] -> v[k1 + 4 k2].
template <typename C, bool INV> struct Dft<C, 16, INV> {
  __device__ __forceinline__ static void run(C* v) {
    C a[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      C x0 = v[n2], x1 = v[n2 + 4], x2 = v[n2 + 8], x3 = v[n2 + 12];
      dft4<C, INV>(x0, x1, x2, x3);
      a[4 * n2 + 0] = x0;
      a[4 * n2 + 1] = mulw16<C, INV>(x1, n2);
      a[4 * n2 + 2] = mulw16<C, INV>(x2, 2 * n2);
      a[4 * n2 + 3] = mulw16<C, INV>(x3, 3 * n2);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C y0 = a[k1], y1 = a[4 + k1], y2 = a[8 + k1], y3 = a[12 + k1];
      dft4<C, INV>(y0, y1, y2, y3);
      v[k1] = y0;
      v[k1 + 4] = y1;
      v[k1 + 8] = y2;
      v[k1 + 12] = y3;
    }
  }
};

// 16-point DFT of inputs v[0..7] (v[8..15] = 0): X[2m] = DFT8(v)[m],
// X[2m+1] = DFT8(v_n w16^n)[m].
template <typename C, bool INV> struct DftHalf<C, 16, INV> {
  __device__ __forceinline__ static void run(C* v) {
    C e[8], o[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      e[n] = v[n];
      o[n] = mulw16<C, INV>(v[n], n);
    }
    Dft<C, 8, INV>::run(e);
    Dft<C, 8, INV>::run(o);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      v[2 * m] = e[m];
      v[2 * m + 1] = o[m];
    }
  }
};

// ---------------------------------------------------------------------------
// Register-resident transform of length N = 16 N2 (N2 = 4, 8, 16) by a group of N2 lanes,
// as two DFT steps (the "four-step" factorisation N = 16 x N2): lane j holds the 16
// elements j + N2 k, transforms them over k (16 points), multiplies by w_N^{j k1},
// exchanges through shared memory so that lane j' holds rows k1 = j' (16/N2) + r, and
// transforms over j (N2 points): output k1 + 16 k2. `ex` is the group's exchange scratch
// (16 rows of pitch EP); the caller synchronises the group around its use.
// ---------------------------------------------------------------------------
template <int N>
__host__ __device__ constexpr int reg_fft_n2() { return N / 16; }

// step 1 on v (in place): 16-point DFT over k, then twiddles w_N^{+- j k1}; HALF: v[8..15] = 0
template <typename C, int N, bool INV, bool HALF>
__device__ __forceinline__ void reg_fft_step1(C (&v)[16], int j, const C* tw) {
  if constexpr (HALF) {
    DftHalf<C, 16, INV>::run(v);
  } else {
    Dft<C, 16, INV>::run(v);
  }
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) {
    C w = tw[j * k1];
    if (INV) w = cconj(w);
    v[k1] = cmul(v[k1], w);
  }
}

// step 2: rows k1 of the exchange (written as ex[k1 * EP + j] by step 1's lanes) to outputs:
// out[r][k2] = X[(j + N2 r) + 16 k2] (lane j takes rows j, j + N2, ...: at a common r the
// lanes of a group read rows EP apart, which spreads them over the banks).
template <typename C, int N, bool INV, int EP>
__device__ __forceinline__ void reg_fft_step2(const C* ex, int j, C (&out)[16]) {
  constexpr int N2 = reg_fft_n2<N>(), R1 = 16 / N2;
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    C row[N2];
#pragma unroll
    for (int i = 0; i < N2; ++i) row[i] = ex[(j + N2 * r) * EP + i];
    Dft<C, N2, INV>::run(row);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) out[r * N2 + k2] = row[k2];
  }
}

// ---------------------------------------------------------------------------
// Stockham stages. Butterfly b of a radix-R stage (after stages whose radices multiply
// to NS) reads elements b + r N/R, twiddles them by exp(-2 pi i r (b mod NS)/(NS R)),
// and writes element r of its DFT to (b / NS) NS R + (b mod NS) + r NS.
// Element i sits at fpadr<RUN>(i) * ES. Whenever the R elements of a butterfly stay inside
// one run (or are spaced by a multiple of the run) their padded offsets differ by
// compile-time constants, so only the first address of a butterfly is computed.
// HALF_IN: the input is zero on [N/2, N) and only its lower half is read.
// ---------------------------------------------------------------------------
// Fills the staged table of length N from the plain table (FP64 and FP32 copies; entry mul * k
// is w_N^k), one stage after another with compile-time offsets and divisors; the calling
// threads share the entries and the caller synchronises.
template <typename C, int N, int S = 0>
__device__ __forceinline__ void build_stw(C* ts, const double2* src64, const float2* src32, int mul, int tid,
                                          int nthreads) {
  if constexpr (S < fft_plan_stages(N)) {
    constexpr int CNT = stw_count(N, S);
    if constexpr (CNT > 0) {
      constexpr int OFF = stw_offset(N, S), R = fft_plan_radix(N, S), RS = (R - 1) | 1;
      constexpr int TWS = N / (stw_stride(N, S) * R);
      for (int i = tid; i < CNT; i += nthreads) {
        const int j = i / RS, r = i - j * RS + 1;
        const int k = r < R ? r * j * TWS : 0;
        if constexpr (sizeof(C) == sizeof(float2)) ts[OFF + i] = src32[mul * k];
        else ts[OFF + i] = src64[mul * k];
      }
    }
    build_stw<C, N, S + 1>(ts, src64, src32, mul, tid, nthreads);
  }
}

template <typename C, int N, int G, bool INV, int S, int NS, int ES, bool HALF_IN, int RUN = 8, bool STW = false>
__device__ __forceinline__ void fft_stages(C* a, int g, const C* tw, bool valid, int bar) {
  if constexpr (S < fft_plan_stages(N)) {
    constexpr int R = fft_plan_radix(N, S);
    constexpr int NB = N / R;
    constexpr int K = (NB + G - 1) / G;
    constexpr int TWS = N / (NS * R);
    constexpr bool HIN = HALF_IN && S == 0 && (R == 2 || R == 4 || R == 8);
    constexpr int RL = HIN ? R / 2 : R;  // inputs read per butterfly
    C v[K][R];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int b = g + k * G;
      if (valid && (NB % G == 0 || b < NB)) {
        if constexpr (NB % RUN == 0) {
          const C* src = a + fpadr<RUN>(b) * ES;
#pragma unroll
          for (int r = 0; r < RL; ++r) v[k][r] = src[r * fft_physr<RUN>(NB) * ES];
        } else {
#pragma unroll
          for (int r = 0; r < RL; ++r) v[k][r] = a[fpadr<RUN>(b + r * NB) * ES];
        }
        if constexpr (NS > 1) {
          if constexpr (STW) {
            constexpr int OFF = stw_offset(N, S), RS = (R - 1) | 1;
            const C* tr = tw + (OFF - 1) + (b % NS) * RS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
              C w = tr[r];
              if (INV) w = cconj(w);
              v[k][r] = cmul(v[k][r], w);
            }
          } else {
            const int jt = (b % NS) * TWS;
#pragma unroll
            for (int r = 1; r < R; ++r) {
              C w = tw[r * jt];
              if (INV) w = cconj(w);
              v[k][r] = cmul(v[k][r], w);
            }
          }
        }
        if constexpr (HIN) {
          DftHalf<C, R, INV>::run(v[k]);
        } else {
          Dft<C, R, INV>::run(v[k]);
        }
      }
    }
    group_sync<G>(bar);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int b = g + k * G;
      if (valid && (NB % G == 0 || b < NB)) {
        const int jj = b % NS;
        const int base = (b / NS) * NS * R + jj;
        if constexpr (NS % RUN == 0) {
          C* dst = a + fpadr<RUN>(base) * ES;
#pragma unroll
          for (int r = 0; r < R; ++r) dst[r * fft_physr<RUN>(NS) * ES] = v[k][r];
        } else if constexpr (NS == 1 && RUN % R == 0) {
          C* dst = a + fpadr<RUN>(base) * ES;
#pragma unroll
          for (int r = 0; r < R; ++r) dst[r * ES] = v[k][r];
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) a[fpadr<RUN>(base + r * NS) * ES] = v[k][r];
        }
      }
    }
    group_sync<G>(bar);
    fft_stages<C, N, G, INV, S + 1, NS * R, ES, HALF_IN, RUN, STW>(a, g, tw, valid, bar);
  }
}

// One length-N transform per group of G lanes. Every lane of the warp must call this
// (lanes of groups without work pass valid = false) because stages end in __syncwarp.
template <typename C, int N, bool INV, int ES = 1, bool HALF_IN = false, int RUN = 8, bool STW = false>
__device__ __forceinline__ void group_fft(C* a, int g, const C* tw, bool valid, int bar = 0) {
  constexpr int G = fft_group_lanes<C>(N);
  fft_stages<C, N, G, INV, 0, 1, ES, HALF_IN, RUN, STW>(a, g, tw, valid, bar);
}

// Batched transforms by a whole CTA: `count` transforms, transform f starting at
// a + f' * fs with f' = fpadr<FRUN>(f) if PADF (transforms along the second axis of a padded
// 2-D tile) else f, element i at fpadr<RUN>(i) * ES. Groups of G <= 32 lanes share a warp
// (32/G transforms per warp at a time); larger groups are G consecutive threads with
// named barrier 1 + (thread / G), so the CTA size must be a multiple of G and below 16 G.
// STW: tw is the staged table of build_stw (stw_fits(N)), else the plain table.
template <typename C, int N, bool INV, bool PADF = false, int ES = 1, bool HALF_IN = false, int RUN = 8,
          int FRUN = 8, bool STW = false>
__device__ __forceinline__ void cta_fft(C* a, int count, int fs, const C* tw) {
  constexpr int G = fft_group_lanes<C>(N);
  int gid, ngroups, bar = 0;
  if constexpr (G <= 32) {
    gid = (threadIdx.x >> 5) * (32 / G) + (threadIdx.x & 31) / G;
    ngroups = (blockDim.x >> 5) * (32 / G);
  } else {
    gid = threadIdx.x / G;
    ngroups = blockDim.x / G;
    bar = 1 + gid;
  }
  const int g = threadIdx.x % G;
  const int rounds = (count + ngroups - 1) / ngroups;
  for (int it = 0; it < rounds; ++it) {
    const int f = gid + it * ngroups;
    const bool valid = f < count;
    const int fo = valid ? (PADF ? fpadr<FRUN>(f) : f) : 0;
    group_fft<C, N, INV, ES, HALF_IN, RUN, STW>(a + fo * fs, g, tw, valid, bar);
  }
}

}  // namespace psfd
