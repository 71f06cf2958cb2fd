// op_kernels.cuh -- the Lippmann-Schwinger operator application, templated on the
// complex type (float2 for the FP32 bulk path, double2 for the FP64 path).
//
// One application A u = u - (I + R) G*(V u) (Sec. 3, Eq. (18) with the reflection
// operator of Eq. (9) folded in) runs as three passes over HBM:
//   K1  per (rhs, component, absorber plane): J = V * u, forward 2-D FFT over (y, x);
//   K2  per (rhs, transverse mode): the nslab planes of all three components are zero
//       padded to nf, transformed along z, multiplied by the windowed dyadic Green's
//       function (a symmetric 3x3 per wavevector, evaluated on the fly), transformed
//       back, and the stack reflection T_R E(plane 0) exp(i beta (p-1) dz) is added;
//   K3  per (rhs, component, plane): inverse 2-D FFT and the epilogue out = u - w
//       (or the FP64 residual b - (u - w)), fused with the Krylov dot products.
// Planes that fit in shared memory are transformed in one CTA (K1/K3 "plane"
// kernels); larger planes use a row pass and a column pass.
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace psfd {

template <typename T, typename P>
__device__ __forceinline__ T* align16(P* p) {
  return reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
}

template <typename C> struct Prec;
template <> struct Prec<float2> { static constexpr int PHI_TERMS = 10; };
template <> struct Prec<double2> { static constexpr int PHI_TERMS = 17; };

__device__ __forceinline__ void split_hi_lo(double2 v, float2& hi, float2& lo) {
  hi = to_c32(v);
  lo = make_float2((float)(v.x - (double)hi.x), (float)(v.y - (double)hi.y));
}
__device__ __forceinline__ void split_hi_lo(double2 v, double2& hi, double2& lo) {
  hi = v;
  lo = make_double2(0.0, 0.0);
}
__device__ __forceinline__ void split_hi_lo_r(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}
__device__ __forceinline__ void split_hi_lo_r(double v, double& hi, double& lo) {
  hi = v;
  lo = 0.0;
}

// Twiddle entry in the working precision. The FP32 kernels read the tables rounded to FP32
// once per context (the values a conversion of the FP64 entry gives), so no FP64 conversion
// runs per CTA: the FP64 pipe of this GPU issues them far slower than the FP32 pipes.
template <typename C>
__device__ __forceinline__ C twid(const double2* t64, const float2* t32, int i) {
  if constexpr (sizeof(C) == sizeof(float2)) return t32[i];
  else return t64[i];
}

// FP32 transforms of the plane passes read their twiddles from the per-stage table.
template <typename C, int N> __host__ __device__ constexpr bool plane_stw() {
  return sizeof(C) == sizeof(float2) && stw_fits(N);
}

// Copies the twiddles of a length-N transform into shared memory: entry mul * i of the
// global table is w_N^i. Plain table, or the per-stage table when plane_stw<C, N>().
template <typename C, int N, int NT>
__device__ __forceinline__ void stage_twiddles(C* dst, const double2* t64, const float2* t32, int mul) {
  if constexpr (plane_stw<C, N>()) build_stw<C, N>(dst, t64, t32, mul, threadIdx.x, NT);
  else
    for (int i = threadIdx.x; i < N; i += NT) dst[i] = twid<C>(t64, t32, mul * i);
}

// a / b through one reciprocal of |b|^2; here |b| stays far from under- and overflow
// (|kappa + beta| >= |beta| and |delta| >= 1/(2L) on this branch).
__device__ __forceinline__ float2 cdiv_fast(float2 a, float2 b) {
  return cscale(cmulc(b, a), __frcp_rn(b.x * b.x + b.y * b.y));
}
__device__ __forceinline__ double2 cdiv_fast(double2 a, double2 b) {
  return cscale(cmulc(b, a), 1.0 / (b.x * b.x + b.y * b.y));
}


// ---------------------------------------------------------------------------
// input stage (K1) and epilogue (K3) element operations
// ---------------------------------------------------------------------------
template <typename C> struct InScal { C a, b; };

template <typename C, int IN>
__device__ __forceinline__ InScal<C> load_in_scalars(const OpCall<C>& a, int g) {
  InScal<C> s;
  s.a = mk((typename RealOf<C>::T)0, (typename RealOf<C>::T)0);
  s.b = s.a;
  if constexpr (sizeof(C) == sizeof(float2) && IN != IN_PLAIN) {
    // one lane per warp converts the FP64 scalars and the warp shares them: the FP64 pipe of
    // this GPU issues conversions far slower than the FP32 pipes (the whole CTA calls this)
    if ((threadIdx.x & 31) == 0) {
      if constexpr (IN == IN_PUPDATE) {
        s.a = from_c64<C>(a.sc[g].beta);
        s.b = from_c64<C>(a.sc[g].omega);
      } else {
        s.a = from_c64<C>(a.sc[g].alpha);
      }
    }
    s.a.x = __shfl_sync(0xffffffffu, s.a.x, 0);
    s.a.y = __shfl_sync(0xffffffffu, s.a.y, 0);
    s.b.x = __shfl_sync(0xffffffffu, s.b.x, 0);
    s.b.y = __shfl_sync(0xffffffffu, s.b.y, 0);
  } else if constexpr (IN == IN_PUPDATE) {
    s.a = from_c64<C>(a.sc[g].beta);
    s.b = from_c64<C>(a.sc[g].omega);
  } else if constexpr (IN == IN_SUPDATE) {
    s.a = from_c64<C>(a.sc[g].alpha);
  }
  return s;
}

template <typename C> struct Acc;
template <> struct Acc<float2> { using T = float2; };
template <> struct Acc<double2> { using T = double2; };

template <typename C>
struct Dots {
  typename Acc<C>::T d[NDOT];
};

// Split forms of the two element operations: all operands of a few elements are loaded
// first (so that their loads are in flight together), then combined and stored.
template <typename C, int IN> struct InVals { C p, r, v; };

template <typename C, int IN>
__device__ __forceinline__ InVals<C, IN> load_in(const OpCall<C>& a, size_t idx) {
  InVals<C, IN> o;
  if constexpr (IN == IN_PLAIN) {
    o.p = a.u[idx];
  } else if constexpr (IN == IN_PUPDATE) {
    o.p = a.u[idx];
    o.r = a.r[idx];
    o.v = a.v[idx];
  } else {
    o.r = a.r[idx];
    o.v = a.v[idx];
  }
  return o;
}

// p = r + beta (p - omega v), s = r - alpha v, or the plain input
template <typename C, int IN>
__device__ __forceinline__ C combine_in(const InVals<C, IN>& o, const InScal<C>& s) {
  if constexpr (IN == IN_PLAIN) return o.p;
  else if constexpr (IN == IN_PUPDATE) return cadd(o.r, cmul(s.a, csub(o.p, cmul(s.b, o.v))));
  else return csub(o.r, cmul(s.a, o.v));
}

template <typename C> struct EpiVals { C u, b, r0; };

template <typename C, int EPI>
__device__ __forceinline__ EpiVals<C> load_epi(const OpCall<C>& a, const C* uin, size_t idx) {
  EpiVals<C> e;
  e.u = uin[idx];
  e.b = e.r0 = mk((typename RealOf<C>::T)0, (typename RealOf<C>::T)0);
  if constexpr (EPI == EPI_RESID) e.b = a.b[idx];
  if (a.dot_mask & DOT_R0_OUT) e.r0 = a.r0[idx];
  return e;
}

template <typename C, int EPI>
__device__ __forceinline__ void store_epi(const OpCall<C>& a, size_t idx, const EpiVals<C>& e, C w, Dots<C>& dt) {
  C out = csub(e.u, w);
  if constexpr (EPI == EPI_RESID) out = csub(e.b, out);
  a.out[idx] = out;
  if (a.dot_mask & DOT_R0_OUT) dt.d[0] = cadd(dt.d[0], cmulc(e.r0, out));
  if (a.dot_mask & DOT_OUT_U) dt.d[1] = cadd(dt.d[1], cmulc(out, e.u));
  if (a.dot_mask & DOT_OUT_OUT) dt.d[2].x += out.x * out.x + out.y * out.y;
}

// Elements whose loads a thread keeps in flight together (input stage / epilogue).
template <typename C> struct Batch {
  static constexpr int IN = sizeof(C) == 8 ? 4 : 1;  // FP32: 4 (2 measured 1-2 % slower on 512^2-1024^2)
  static constexpr int OUT = sizeof(C) == 8 ? 8 : 2;
};

// Input stage of n consecutive elements starting at base: tile[slot(i)] = V[i] * input(i),
// updating p or s in place on the way.
template <typename C, int IN, int NT, typename Slot>
__device__ __forceinline__ void stage_in(const OpCall<C>& a, const InScal<C>& s, size_t base, const C* Vp, int n,
                                         C* tile, Slot slot) {
  constexpr int BT = Batch<C>::IN;
  for (int i0 = threadIdx.x; i0 < n; i0 += BT * NT) {
    InVals<C, IN> in[BT];
    C vv[BT];
#pragma unroll
    for (int j = 0; j < BT; ++j) {
      const int i = i0 + j * NT;
      if (i < n) {
        vv[j] = Vp[i];
        in[j] = load_in<C, IN>(a, base + i);
      }
    }
#pragma unroll
    for (int j = 0; j < BT; ++j) {
      const int i = i0 + j * NT;
      if (i < n) {
        const C u = combine_in<C, IN>(in[j], s);
        if constexpr (IN != IN_PLAIN) a.ustore[base + i] = u;
        tile[slot(i)] = cmul(vv[j], u);
      }
    }
  }
}

// Epilogue of n consecutive elements starting at base, w(i) = tile[slot(i)].
template <typename C, int EPI, int NT, typename Slot>
__device__ __forceinline__ void stage_out(const OpCall<C>& a, const C* uin, size_t base, int n, const C* tile,
                                          Slot slot, Dots<C>& dt) {
  constexpr int BT = Batch<C>::OUT;
  for (int i0 = threadIdx.x; i0 < n; i0 += BT * NT) {
    EpiVals<C> e[BT];
#pragma unroll
    for (int j = 0; j < BT; ++j)
      if (i0 + j * NT < n) e[j] = load_epi<C, EPI>(a, uin, base + i0 + j * NT);
#pragma unroll
    for (int j = 0; j < BT; ++j) {
      const int i = i0 + j * NT;
      if (i < n) store_epi<C, EPI>(a, base + i, e[j], tile[slot(i)], dt);
    }
  }
}

__device__ __forceinline__ double2 shfl_down_d2(double2 v, int o) {
  return make_double2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
}

// Sum of v over the warp as an unevaluated pair hi + lo of FP32 numbers (lane 0 holds it):
// Knuth's TwoSum of the high parts at each level of the tree, the low parts and the rounding
// error added, then Dekker's FastTwoSum renormalises. About 48 bits: the block's FP64
// reduction receives the warp's sum without FP64 arithmetic in every warp.
__device__ __forceinline__ float2 warp_sum_pair(float v) {
  float hi = v, lo = 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
    const float s = __fadd_rn(hi, h2);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(h2, bp));
    const float t = __fadd_rn(__fadd_rn(lo, l2), e);
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
  }
  return make_float2(hi, lo);
}

// Deterministic block reduction of the (up to three) dot products; thread 0 writes
// dst[k * stride] for every requested k. Needs 3 * 32 double2 of shared scratch.
template <typename C>
__device__ __forceinline__ void block_write_dots(const Dots<C>& dt, int mask, double2* dst, int stride,
                                                 double2* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NDOT; ++k) {
    if (!(mask & (1 << k))) continue;
    if constexpr (sizeof(C) == sizeof(float2)) {
      // FP32 partial sums: the warp adds them as FP32 pairs (about 48 bits) and one lane
      // converts the pair, so that no warp runs an FP64 reduction tree on the slow FP64 pipe
      const float2 re = warp_sum_pair(dt.d[k].x), im = warp_sum_pair(dt.d[k].y);
      if (lane == 0)
        scratch[k * 32 + warp] = make_double2((double)re.x + (double)re.y, (double)im.x + (double)im.y);
    } else {
      double2 v = as_c64(dt.d[k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = cadd(v, shfl_down_d2(v, o));
      if (lane == 0) scratch[k * 32 + warp] = v;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NDOT; ++k) {
      if (!(mask & (1 << k))) continue;
      double2 v = lane < nw ? scratch[k * 32 + lane] : make_double2(0.0, 0.0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = cadd(v, shfl_down_d2(v, o));
      if (lane == 0) dst[k * stride] = v;
    }
  }
}

template <typename C>
__device__ __forceinline__ void zero_dots(Dots<C>& dt) {
#pragma unroll
  for (int k = 0; k < NDOT; ++k) dt.d[k] = mk((typename RealOf<C>::T)0, (typename RealOf<C>::T)0);
}

// ---------------------------------------------------------------------------
// K1 / K3 for planes that fit in shared memory
// ---------------------------------------------------------------------------
// Shared tile of a whole plane: row y at fpad(y) * PITCH, element x of a row at fpad(x);
// PITCH is odd so that column transforms (element stride PITCH) spread over the banks.
template <int NX> __host__ __device__ constexpr int plane_pitch() { return fft_phys(NX) | 1; }
template <int NX, int NY> __host__ __device__ constexpr int plane_tile_elems() {
  return fft_phys(NY) * plane_pitch<NX>();
}
template <int NX>
__device__ __forceinline__ int plane_slot(int i) {
  return fpad(i / NX) * plane_pitch<NX>() + fpad(i % NX);
}

template <typename C, int NX, int NY, int IN, int NT>
__global__ void __launch_bounds__(NT) k_plane_fwd(OpCall<C> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PITCH = plane_pitch<NX>();
  C* tile = reinterpret_cast<C*>(smem);
  C* twx = tile + plane_tile_elems<NX, NY>();
  C* twy = twx + NX;
  const int p = blockIdx.x, c = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  for (int i = threadIdx.x; i < NX; i += NT) twx[i] = twid<C>(a.twx, a.twx32, i);
  for (int i = threadIdx.x; i < NY; i += NT) twy[i] = twid<C>(a.twy, a.twy32, i);
  const InScal<C> s = load_in_scalars<C, IN>(a, g);
  const size_t plane = (((size_t)lr * 3 + c) * a.nslab + p) * (size_t)(NX * NY);
  const C* Vp = a.V + ((size_t)a.rhsp[g].clip * a.nslab + p) * (NX * NY);
  stage_in<C, IN, NT>(a, s, plane, Vp, NX * NY, tile, [](int i) { return plane_slot<NX>(i); });
  __syncthreads();
  cta_fft<C, NX, false, true, 1>(tile, NY, PITCH, twx);
  __syncthreads();
  cta_fft<C, NY, false, true, PITCH>(tile, NX, 1, twy);
  __syncthreads();
  for (int i = threadIdx.x; i < NX * NY; i += NT) a.work[plane + i] = tile[plane_slot<NX>(i)];
}

template <typename C, int NX, int NY, int EPI, int NT>
__global__ void __launch_bounds__(NT) k_plane_inv(OpCall<C> a, const C* uin) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PITCH = plane_pitch<NX>();
  C* tile = reinterpret_cast<C*>(smem);
  C* twx = tile + plane_tile_elems<NX, NY>();
  C* twy = twx + NX;
  double2* scratch = align16<double2>(twy + NY);
  const int p = blockIdx.x, c = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  for (int i = threadIdx.x; i < NX; i += NT) twx[i] = twid<C>(a.twx, a.twx32, i);
  for (int i = threadIdx.x; i < NY; i += NT) twy[i] = twid<C>(a.twy, a.twy32, i);
  const size_t plane = (((size_t)lr * 3 + c) * a.nslab + p) * (size_t)(NX * NY);
  for (int i = threadIdx.x; i < NX * NY; i += NT) tile[plane_slot<NX>(i)] = a.work[plane + i];
  __syncthreads();
  cta_fft<C, NY, true, true, PITCH>(tile, NX, 1, twy);
  __syncthreads();
  cta_fft<C, NX, true, true, 1>(tile, NY, PITCH, twx);
  __syncthreads();
  Dots<C> dt;
  zero_dots(dt);
  stage_out<C, EPI, NT>(a, uin, plane, NX * NY, tile, [](int i) { return plane_slot<NX>(i); }, dt);
  if (a.dot_mask) {
    const int blk = c * a.nslab + p;
    block_write_dots(dt, a.dot_mask, a.partials + ((size_t)g * NDOT) * a.maxblk + blk, a.maxblk, scratch);
  }
}

// ---------------------------------------------------------------------------
// K1 / K3 on half planes: two CTAs per plane, each holding NY/2 rows, so that two
// planes' worth of CTAs share one SM and one CTA's loads overlap the other's FFTs.
// The y transform is split by one radix-2 decimation-in-frequency step done while
// loading: with H = NY/2 and w = exp(-2 pi i / NY),
//   Y[2m + h] = sum_{r<H} [(x_r + (-1)^h x_{r+H}) w^{r h}] exp(-2 pi i r m / H),
// so CTA h reads the whole plane (the second read of each element hits L2), forms the
// H combined rows, and transforms them along x (length NX) and along y (length H),
// giving the spectral rows of parity h. The inverse uses the conjugate identity
//   y[2m + h] = sum_{k<H} [(Y_k + (-1)^h Y_{k+H}) w^{-k h}] exp(+2 pi i k m / H)
// and applies the epilogue to the output rows of parity h.
// ---------------------------------------------------------------------------
// Row pitch of a half-plane tile. The y transforms (length NY/2, element stride PITCH) run in
// groups of G lanes, 16/G of them side by side in a 16-lane memory phase at consecutive
// columns; for 8-byte elements PITCH = 16/G (mod 16) interleaves their elements over the
// banks (an odd pitch would put two columns' elements on neighbouring banks).
// Half-plane tiles pad every 16 elements along x (the x transforms read 16 consecutive
// elements per 16-lane phase) and every 8 along y.
constexpr int kHalfXRun = 16;

template <typename C, int NX, int NY> __host__ __device__ constexpr int half_pitch() {
  constexpr int G = fft_group_lanes<C>(NY / 2), base = fft_physr<kHalfXRun>(NX);
  if constexpr (sizeof(C) == 8 && G < 16) {
    constexpr int m = 16 / G;
    return base + ((m - base % 16) % 16 + 16) % 16;
  } else {
    return base | 1;
  }
}
static_assert(half_pitch<float2, 128, 128>() == 146, "half-plane pitch");
template <typename C, int NX, int NY> __host__ __device__ constexpr int half_tile_elems() {
  return fft_phys(NY / 2) * half_pitch<C, NX, NY>();
}

// L2 prefetch of a contiguous range by the bulk-copy unit (no registers, no wait).
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Half-plane K1 and K3 are latency-bound: a CTA's global loads come in one phase and its
// transforms in another. Thread 0 of each CTA therefore asks the bulk-copy unit to bring into
// L2 the planes that the CTA a.pf launches later (in linear block order) will read, so that
// its loads hit L2. Only the even CTA of a plane pair prefetches (both read the whole plane).
template <typename C, int NX, int NY, int IN, bool INV>
__device__ __forceinline__ void half_prefetch(const OpCall<C>& a, const C* uin) {
  const unsigned nbx = gridDim.x, nby = gridDim.y;
  const unsigned lin = blockIdx.x + nbx * (blockIdx.y + nby * blockIdx.z) + (unsigned)a.pf;
  if (lin >= nbx * nby * gridDim.z) return;
  const unsigned bx = lin % nbx, yz = lin / nbx;
  if (bx & 1u) return;
  const int p = (int)(bx >> 1), c = (int)(yz % nby), lr = (int)(yz / nby), g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  constexpr unsigned bytes = NX * NY * sizeof(C);
  const size_t plane = (((size_t)lr * 3 + c) * a.nslab + p) * (size_t)(NX * NY);
  if constexpr (INV) {
    l2_prefetch(a.work + plane, bytes);
    l2_prefetch(uin + plane, bytes);
    if (a.dot_mask & DOT_R0_OUT) l2_prefetch(a.r0 + plane, bytes);
  } else {
    l2_prefetch(a.V + ((size_t)a.rhsp[g].clip * a.nslab + p) * (NX * NY), bytes);
    l2_prefetch(a.u + plane, bytes);
  }
}

template <typename C, int NX, int NY, int IN, int NT>
__global__ void __launch_bounds__(NT, 2) k_half_fwd(OpCall<C> a) {
  constexpr int H = NY / 2, PITCH = half_pitch<C, NX, NY>();
  extern __shared__ __align__(16) unsigned char smem[];
  C* tile = reinterpret_cast<C*>(smem);
  C* twx = tile + half_tile_elems<C, NX, NY>();
  C* twy = twx + NX;  // exp(-2 pi i r / NY), r < H
  C* twh = twy + H;   // exp(-2 pi i t / H), t < H
  const int p = blockIdx.x >> 1, h = blockIdx.x & 1, c = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  // the update stages (p, s) read three vectors and V per plane: prefetching all of them ahead
  // measured slower inside the solve, so only the plain input stage prefetches
  if constexpr (IN == IN_PLAIN)
    if (a.pf && threadIdx.x == 0) half_prefetch<C, NX, NY, IN, false>(a, nullptr);
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  stage_twiddles<C, NX, NT>(twx, a.twx, a.twx32, 1);
  stage_twiddles<C, H, NT>(twh, a.twy, a.twy32, 2);
  for (int i = threadIdx.x; i < H; i += NT) twy[i] = twid<C>(a.twy, a.twy32, i);
  __syncthreads();
  const InScal<C> s = load_in_scalars<C, IN>(a, g);
  const size_t plane = (((size_t)lr * 3 + c) * a.nslab + p) * (size_t)(NX * NY);
  const C* Vp = a.V + ((size_t)a.rhsp[g].clip * a.nslab + p) * (NX * NY);
  constexpr int TOT = H * NX;
  // elements per thread whose loads overlap: four for the plain and s-update stages (two and
  // three operands per element), two for the p update, whose four operands would spill
  constexpr int BT = (IN != IN_PUPDATE && TOT % (4 * NT) == 0) ? 4 : (TOT % (2 * NT) == 0 ? 2 : 1);
  static_assert(TOT % NT == 0, "half plane must be a multiple of the CTA size");
  for (int i0 = threadIdx.x; i0 < TOT; i0 += BT * NT) {
    InVals<C, IN> in0[BT], in1[BT];
    C va[BT], vb[BT];
#pragma unroll
    for (int j = 0; j < BT; ++j) {
      const int i = i0 + j * NT;
      va[j] = Vp[i];
      vb[j] = Vp[i + TOT];
      in0[j] = load_in<C, IN>(a, plane + i);
      in1[j] = load_in<C, IN>(a, plane + i + TOT);
    }
#pragma unroll
    for (int j = 0; j < BT; ++j) {
      const int i = i0 + j * NT, r = i / NX;
      const C u0 = combine_in<C, IN>(in0[j], s), u1 = combine_in<C, IN>(in1[j], s);
      if constexpr (IN != IN_PLAIN) a.ustore[plane + i + (h ? TOT : 0)] = h ? u1 : u0;  // owner's half
      const C v0 = cmul(va[j], u0), v1 = cmul(vb[j], u1);
      tile[fpad(r) * PITCH + fpadr<kHalfXRun>(i % NX)] = h ? cmul(csub(v0, v1), twy[r]) : cadd(v0, v1);
    }
  }
  __syncthreads();
  cta_fft<C, NX, false, true, 1, false, kHalfXRun, 8, plane_stw<C, NX>()>(tile, H, PITCH, twx);
  __syncthreads();
  cta_fft<C, H, false, true, PITCH, false, 8, kHalfXRun, plane_stw<C, H>()>(tile, NX, 1, twh);
  __syncthreads();
  for (int i = threadIdx.x; i < H * NX; i += NT) {
    const int m = i / NX, x = i % NX;
    a.work[plane + (size_t)(2 * m + h) * NX + x] = tile[fpad(m) * PITCH + fpadr<kHalfXRun>(x)];
  }
}

template <typename C, int NX, int NY, int EPI, int NT>
__global__ void __launch_bounds__(NT, 2) k_half_inv(OpCall<C> a, const C* uin) {
  constexpr int H = NY / 2, PITCH = half_pitch<C, NX, NY>();
  extern __shared__ __align__(16) unsigned char smem[];
  C* tile = reinterpret_cast<C*>(smem);
  C* twx = tile + half_tile_elems<C, NX, NY>();
  C* twy = twx + NX;
  C* twh = twy + H;
  double2* scratch = align16<double2>(twh + H);
  const int p = blockIdx.x >> 1, h = blockIdx.x & 1, c = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  if (a.pf && threadIdx.x == 0) half_prefetch<C, NX, NY, IN_PLAIN, true>(a, uin);
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  stage_twiddles<C, NX, NT>(twx, a.twx, a.twx32, 1);
  stage_twiddles<C, H, NT>(twh, a.twy, a.twy32, 2);
  for (int i = threadIdx.x; i < H; i += NT) twy[i] = twid<C>(a.twy, a.twy32, i);
  __syncthreads();
  const size_t plane = (((size_t)lr * 3 + c) * a.nslab + p) * (size_t)(NX * NY);
  constexpr int BL = (H * NX) % (4 * NT) == 0 ? 4 : 1;  // elements per thread whose loads overlap
  for (int i0 = threadIdx.x; i0 < H * NX; i0 += BL * NT) {
    C y0[BL], y1[BL];
#pragma unroll
    for (int j = 0; j < BL; ++j) {
      y0[j] = a.work[plane + i0 + j * NT];
      y1[j] = a.work[plane + i0 + j * NT + H * NX];
    }
#pragma unroll
    for (int j = 0; j < BL; ++j) {
      const int i = i0 + j * NT, k = i / NX;
      tile[fpad(k) * PITCH + fpadr<kHalfXRun>(i % NX)] = h ? cmul(csub(y0[j], y1[j]), cconj(twy[k])) : cadd(y0[j], y1[j]);
    }
  }
  __syncthreads();
  cta_fft<C, H, true, true, PITCH, false, 8, kHalfXRun, plane_stw<C, H>()>(tile, NX, 1, twh);
  __syncthreads();
  cta_fft<C, NX, true, true, 1, false, kHalfXRun, 8, plane_stw<C, NX>()>(tile, H, PITCH, twx);
  __syncthreads();
  Dots<C> dt;
  zero_dots(dt);
  constexpr int TOT = H * NX;
  constexpr int BT = TOT % (4 * NT) == 0 ? 4 : 1;
  static_assert(TOT % NT == 0, "half plane must be a multiple of the CTA size");
  for (int i0 = threadIdx.x; i0 < TOT; i0 += BT * NT) {
    EpiVals<C> e[BT];
#pragma unroll
    for (int j = 0; j < BT; ++j) {
      const int i = i0 + j * NT;
      e[j] = load_epi<C, EPI>(a, uin, plane + (size_t)(2 * (i / NX) + h) * NX + i % NX);
    }
#pragma unroll
    for (int j = 0; j < BT; ++j) {
      const int i = i0 + j * NT, m = i / NX, x = i % NX;
      store_epi<C, EPI>(a, plane + (size_t)(2 * m + h) * NX + x, e[j], tile[fpad(m) * PITCH + fpadr<kHalfXRun>(x)], dt);
    }
  }
  if (a.dot_mask) {
    const int blk = (c * a.nslab + p) * 2 + h;
    block_write_dots(dt, a.dot_mask, a.partials + ((size_t)g * NDOT) * a.maxblk + blk, a.maxblk, scratch);
  }
}

// ---------------------------------------------------------------------------
// split path: row pass and column pass (planes larger than shared memory)
// ---------------------------------------------------------------------------
// CTAs per SM the split-plane kernels (rows, columns; planes above 128^2 in FP32, FP64
// planes above 64^2) are compiled for. In FP32 they are latency-bound: an 80-register cap
// makes three 256-thread CTAs resident instead of two. It spills a little at 512 and 1024
// points and still pays there (1024^2: K1 and K3 25-28 % faster). FP64 is FP64-pipe bound:
// up to 256 points a cap of 128 registers keeps two CTAs per SM without spills (an explicit
// minimum of one let the compiler take 130-136 registers, one CTA per SM and a 30 % slower
// FP64 residual); longer FP64 transforms would spill under that cap and keep one CTA.
// Padding run of the split passes' tiles: one spare slot after every 16 FP32 elements (a
// half-warp's run of 16 consecutive elements -- the loads and the later stores of a Stockham
// stage whose group spans whole warps -- stays inside one run), every 8 FP64 elements (eight
// 16-byte elements fill the banks).
template <typename C> __host__ __device__ constexpr int split_run() { return sizeof(C) == 8 ? 16 : 8; }

// Column pitch of the column pass's tile: a memory phase of its transposing copies holds tx
// columns x (16 / tx) rows (FP32: 16 lanes of 8 bytes) or tx x (8 / tx) (FP64: 8 lanes of 16
// bytes); a pitch of 16 / tx (8 / tx) modulo 16 (8) elements puts them on distinct banks (an
// odd pitch once tx fills the phase). The transforms run along one column per group of lanes,
// where the pitch plays no part.
template <typename C>
__host__ __device__ inline int cols_pitch(int ny, int tx) {
  constexpr int PH = sizeof(C) == 8 ? 16 : 8;
  const int base = fft_physr<split_run<C>()>(ny);
  const int pmod = tx >= PH ? 1 : PH / tx;
  return base + ((pmod - base % PH) % PH + PH) % PH;
}

template <typename C, int N> __host__ __device__ constexpr int split_min_blocks() {
  return sizeof(C) == 8 ? 3 : (N <= 256 ? 2 : 1);
}

// Each CTA transforms rb rows of length NX (k_rows_inv: blockIdx.x = plane * (ny / rb) + row
// block; k_rows_fwd orders its grid for V's reuse in L2, below).
template <typename C, int NX, int IN, int NT>
__global__ void __launch_bounds__(NT, split_min_blocks<C, NX>()) k_rows_fwd(OpCall<C> a, int rb) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int RUN = split_run<C>();
  constexpr int RP = fft_physr<RUN>(NX);  // row pitch of the tile
  C* tile = reinterpret_cast<C*>(smem);
  C* tw = tile + rb * RP;
  // blockIdx.x = rhs * 3 + component, blockIdx.y = row block, blockIdx.z = plane: the CTAs
  // that read the same rows of V run next to each other, so V (hundreds of MB on large
  // grids, beyond L2) comes from DRAM once per launch rather than once per rhs and component
  const int p = blockIdx.z, y0 = blockIdx.y * rb;
  const int c = blockIdx.x % 3, lr = blockIdx.x / 3, g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  stage_twiddles<C, NX, NT>(tw, a.twx, a.twx32, 1);
  const InScal<C> s = load_in_scalars<C, IN>(a, g);
  const size_t base = ((((size_t)lr * 3 + c) * a.nslab + p) * a.ny + y0) * (size_t)NX;
  const C* Vp = a.V + (((size_t)a.rhsp[g].clip * a.nslab + p) * a.ny + y0) * NX;
  stage_in<C, IN, NT>(a, s, base, Vp, rb * NX, tile, [](int i) { return (i / NX) * RP + fpadr<RUN>(i % NX); });
  __syncthreads();
  cta_fft<C, NX, false, false, 1, false, RUN, 8, plane_stw<C, NX>()>(tile, rb, RP, tw);
  __syncthreads();
  for (int i = threadIdx.x; i < rb * NX; i += NT) a.work[base + i] = tile[(i / NX) * RP + fpadr<RUN>(i % NX)];
}

template <typename C, int NX, int EPI, int NT>
__global__ void __launch_bounds__(NT, split_min_blocks<C, NX>()) k_rows_inv(OpCall<C> a, const C* uin, int rb) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int RUN = split_run<C>();
  constexpr int RP = fft_physr<RUN>(NX);
  C* tile = reinterpret_cast<C*>(smem);
  C* tw = tile + rb * RP;
  double2* scratch = align16<double2>(tw + NX);
  const int nrb = a.ny / rb;
  const int p = blockIdx.x / nrb, y0 = (blockIdx.x % nrb) * rb;
  const int c = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  stage_twiddles<C, NX, NT>(tw, a.twx, a.twx32, 1);
  const size_t base = ((((size_t)lr * 3 + c) * a.nslab + p) * a.ny + y0) * (size_t)NX;
  constexpr int LB = 4;  // elements per thread whose loads are in flight together
  for (int i0 = threadIdx.x; i0 < rb * NX; i0 += LB * NT) {
    C vv[LB];
#pragma unroll
    for (int j = 0; j < LB; ++j)
      if (i0 + j * NT < rb * NX) vv[j] = a.work[base + i0 + j * NT];
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      const int i = i0 + j * NT;
      if (i < rb * NX) tile[(i / NX) * RP + fpadr<RUN>(i % NX)] = vv[j];
    }
  }
  __syncthreads();
  cta_fft<C, NX, true, false, 1, false, RUN, 8, plane_stw<C, NX>()>(tile, rb, RP, tw);
  __syncthreads();
  Dots<C> dt;
  zero_dots(dt);
  stage_out<C, EPI, NT>(a, uin, base, rb * NX, tile, [](int i) { return (i / NX) * RP + fpadr<RUN>(i % NX); }, dt);
  if (a.dot_mask) {
    const int blk = (c * a.nslab + p) * nrb + (y0 / rb);
    block_write_dots(dt, a.dot_mask, a.partials + ((size_t)g * NDOT) * a.maxblk + blk, a.maxblk, scratch);
  }
}

// In-place transforms along y of tx consecutive columns of one plane.
// blockIdx.x = plane * (nx / tx) + column block.
template <typename C, int NY, bool INV, int NT>
__global__ void __launch_bounds__(NT, split_min_blocks<C, NY>()) k_cols(OpCall<C> a, int tx) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int RUN = split_run<C>();
  const int PITCH = cols_pitch<C>(NY, tx);
  C* tile = reinterpret_cast<C*>(smem);
  C* tw = tile + tx * PITCH;
  const int ncb = a.nx / tx;
  const int p = blockIdx.x / ncb, x0 = (blockIdx.x % ncb) * tx;
  const int c = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  stage_twiddles<C, NY, NT>(tw, a.twy, a.twy32, 1);
  const size_t base = (((size_t)lr * 3 + c) * a.nslab + p) * (size_t)NY * a.nx + x0;
  const int t0 = threadIdx.x % tx, y0 = threadIdx.x / tx, ystep = NT / tx;
  constexpr int CB = 8;  // column elements per thread whose loads are in flight together
  for (int y = y0; y < NY; y += CB * ystep) {
    C vv[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      const int yy = y + j * ystep;
      if (yy < NY) vv[j] = a.work[base + (size_t)yy * a.nx + t0];
    }
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      const int yy = y + j * ystep;
      if (yy < NY) tile[t0 * PITCH + fpadr<RUN>(yy)] = vv[j];
    }
  }
  __syncthreads();
  cta_fft<C, NY, INV, false, 1, false, RUN, 8, plane_stw<C, NY>()>(tile, tx, PITCH, tw);
  __syncthreads();
  for (int y = y0; y < NY; y += ystep) a.work[base + (size_t)y * a.nx + t0] = tile[t0 * PITCH + fpadr<RUN>(y)];
}

// ---------------------------------------------------------------------------
// K2: z columns -- zero padding, FFT_z, dyadic Green's function, IFFT_z, reflection
// ---------------------------------------------------------------------------
// Windowed periodic-transverse Green's function of one mode (q, beta) at kz_l:
//   F[G_L] = S (I - k k^T / kb^2) - (E / kb^2) z z^T,  k = (qx, qy, kz_l),
//   E = (-1)^l exp(i beta L),  S = (1 - E) / (kz^2 - beta^2),
// with L = nf dz / 2 so that kz_l L = pi l. Writing kappa = |kz_l| and
// delta = beta - kappa, E = exp(i delta L) and S = i L phi1(i delta L) / (kappa + beta),
// phi1(w) = (e^w - 1)/w. Near the removable singularity (|delta L| < 1/2) phi1 is summed
// as its Taylor series; elsewhere S = (E - 1)/(delta (kappa + beta)) with E from the FP64
// table exp(i beta L). delta is formed from hi/lo splits of beta and kappa so that it
// stays accurate in FP32 when beta ~ kappa. S and E depend on l only through kappa and
// the parity of l, so one evaluation serves l and nf - l.
template <typename C>
__device__ __forceinline__ bool green_scalars_far(typename RealOf<C>::T kh, typename RealOf<C>::T kl, C bh, C bl,
                                                  C E, typename RealOf<C>::T L, typename RealOf<C>::T cinv,
                                                  typename RealOf<C>::T scale, C& S, C& Es) {
  using R = typename RealOf<C>::T;
  const C d = mk((bh.x - kh) + (bl.x - kl), bh.y + bl.y);
  const C kpb = mk((kh + bh.x) + (kl + bl.x), bh.y + bl.y);
  const C w = mk(-d.y * L, d.x * L);
  if (w.x * w.x + w.y * w.y < (R)0.25) return false;  // near: green_scalars_near
  S = cscale(cdiv_fast(mk(E.x - (R)1, E.y), cmul(d, kpb)), scale);
  Es = cscale(E, cinv * scale);
  return true;
}
// The same scalars for |delta L| < 1/2, through phi1's Taylor series.
template <typename C>
__device__ __forceinline__ void green_scalars_near(typename RealOf<C>::T kh, typename RealOf<C>::T kl, C bh, C bl,
                                                   C E, typename RealOf<C>::T L, typename RealOf<C>::T cinv,
                                                   typename RealOf<C>::T scale, C& S, C& Es) {
  using R = typename RealOf<C>::T;
  const C d = mk((bh.x - kh) + (bl.x - kl), bh.y + bl.y);
  const C kpb = mk((kh + bh.x) + (kl + bl.x), bh.y + bl.y);
  const C w = mk(-d.y * L, d.x * L);
  // phi1(w) = 1 + w/2 (1 + w/3 (1 + ...)), Horner from the innermost term
  C phi = mk((R)1, (R)0);
#pragma unroll
  for (int k = Prec<C>::PHI_TERMS; k >= 2; --k) {
    const R ik = (R)1 / (R)k;
    const C t = cmul(w, phi);
    phi = mk((R)1 + t.x * ik, t.y * ik);
  }
  S = cscale(cdiv_fast(mk(-phi.y * L, phi.x * L), kpb), scale);  // i L phi1 / (kappa + beta)
  Es = cscale(E, cinv * scale);
}


// W = S (J - k (k.J) / kb^2) - (E / kb^2) z (z.J) for k = (qx, qy, kz), in place (registers).
template <typename C>
__device__ __forceinline__ void dyadic_reg(C& J0, C& J1, C& J2, typename RealOf<C>::T qx, typename RealOf<C>::T qy,
                                           typename RealOf<C>::T kz, C S, C Es, typename RealOf<C>::T cinv) {
  const C kJ = cadd(cadd(cscale(J0, qx), cscale(J1, qy)), cscale(J2, kz));
  const C ckJ = cscale(kJ, cinv);
  const C w0 = cmul(S, csub(J0, cscale(ckJ, qx)));
  const C w1 = cmul(S, csub(J1, cscale(ckJ, qy)));
  const C w2 = csub(cmul(S, csub(J2, cscale(ckJ, kz))), cmul(Es, J2));
  J0 = w0;
  J1 = w1;
  J2 = w2;
}
// The same product on three shared-memory elements.
template <typename C>
__device__ __forceinline__ void dyadic_apply(C* c0, C* c1, C* c2, typename RealOf<C>::T qx, typename RealOf<C>::T qy,
                                             typename RealOf<C>::T kz, C S, C Es, typename RealOf<C>::T cinv) {
  C J0 = *c0, J1 = *c1, J2 = *c2;
  dyadic_reg(J0, J1, J2, qx, qy, kz, S, Es, cinv);
  *c0 = J0;
  *c1 = J1;
  *c2 = J2;
}

// W = A J + (B/|k|^2) k (k.J) for k = (qx, qy, kz): the spherically windowed kernel of an
// isolated clip (Eqs. (15)-(17)), in place (registers).
template <typename C>
__device__ __forceinline__ void dyadic_sph_reg(C& J0, C& J1, C& J2, typename RealOf<C>::T qx,
                                               typename RealOf<C>::T qy, typename RealOf<C>::T kz, C A, C Bt) {
  const C t = cmul(Bt, cadd(cadd(cscale(J0, qx), cscale(J1, qy)), cscale(J2, kz)));
  const C w0 = cadd(cmul(A, J0), cscale(t, qx));
  const C w1 = cadd(cmul(A, J1), cscale(t, qy));
  const C w2 = cadd(cmul(A, J2), cscale(t, kz));
  J0 = w0;
  J1 = w1;
  J2 = w2;
}
// The same product on three shared-memory elements.
template <typename C>
__device__ __forceinline__ void dyadic_sph(C* c0, C* c1, C* c2, typename RealOf<C>::T qx, typename RealOf<C>::T qy,
                                           typename RealOf<C>::T kz, C A, C Bt) {
  C J0 = *c0, J1 = *c1, J2 = *c2;
  dyadic_sph_reg(J0, J1, J2, qx, qy, kz, A, Bt);
  *c0 = J0;
  *c1 = J1;
  *c2 = J2;
}

// Entries of the per-column reflection phase table exp(i beta dz j): j < 8 (fine
// steps) and 8 j' for j' < NF/16 (coarse steps); the phase of plane pl is the
// product of entries pl % 8 and 8 + pl / 8 (pl < nslab <= nf/2 - 1).
template <int NF> __host__ __device__ constexpr int phase_entries() { return 8 + (NF + 15) / 16; }
// Row pitch of the phase table: odd, so that the columns of a CTA read their rows from
// different banks.
template <int NF> __host__ __device__ constexpr int phase_pitch() { return phase_entries<NF>() | 1; }

// Column pitch of K2's shared tile (in elements). Odd in general, so that the columns of a
// CTA are read at a common z from different banks. For the FP32 register transform with
// groups of n2 = nf/16 < 16 lanes it is n2 modulo 16 instead: 16/n2 groups share a 16-lane
// memory phase there, and offsets of n2 elements between their columns keep the exchange
// stores and the contiguous loads and stores of the transforms free of bank conflicts.
__host__ __device__ constexpr int zcol_pitch(int nf, bool f32reg) {
  return (f32reg && nf / 16 < 16) ? fft_phys(nf) + ((nf / 16 - fft_phys(nf) % 16) % 16 + 16) % 16
                                  : (fft_phys(nf) | 1);
}
static_assert(zcol_pitch(128, true) == 152 && zcol_pitch(64, true) == 84 && zcol_pitch(256, true) == 289,
              "register-transform pitches");

// grid (nx / tx, ny, nrhs); dynamic shared memory: 3 tx (NF + 1) columns + tables.
// Columns of length 64, 128 and 256 use the register-resident transform in both precisions
// (groups of NF/16 lanes, one shared-memory exchange per transform, input read straight
// from HBM); the CTA then has 24 groups: 8 x-modes x 3 components. In FP64 the 16 x NF/16
// factorisation also needs fewer FP64 operations than the shared-memory radix 8-8-2 plan.
template <typename C, int NF> __host__ __device__ constexpr bool zcol_reg() {
  return NF == 64 || NF == 128 || NF == 256;
}
// FP32 columns of length 160 use a register transform as 16 x 10: a group of 16 lanes per
// column, lanes j < 10 doing 16-point DFTs of the elements j + 10k, then each lane one
// 10-point DFT of an exchange row; the spectrum and the output go through shared memory.
template <typename C, int NF> __host__ __device__ constexpr bool zcol_r10() { return sizeof(C) == 8 && NF == 160; }
// CTAs per SM the FP32 kernel is compiled for at the z lengths of the measured workloads
// (128: register transform with 192 threads, 160: the 16 x 10 transform with 384 threads); it
// is issue- or latency-bound, and more resident warps hide the shared-memory and barrier
// waits (neither cap spills). 1 = no register cap.
// Scaled with the CTA size NT (the 8-mode CTA has 192 and 384 threads), so that the register
// cap stays the same for the 4- and 16-mode CTAs the autotuner may pick.
template <typename C, int NF, int NT> __host__ __device__ constexpr int zcol_min_blocks() {
  return (sizeof(C) == 8 && NF == 128) ? (960 / NT > 1 ? 960 / NT : 1)
                                       : (zcol_r10<C, NF>() ? (1152 / NT > 1 ? 1152 / NT : 1) : 1);
}

template <typename C, int NF, int NT>
__global__ void __launch_bounds__(NT, zcol_min_blocks<C, NF, NT>()) k_zcol(OpCall<C> a, int tx) {
  using R = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr bool F32 = sizeof(C) == sizeof(float2);
  constexpr bool REG = zcol_reg<C, NF>();
  constexpr bool R10 = zcol_r10<C, NF>();
  constexpr int P = zcol_pitch(NF, F32 && REG);  // column pitch; spectral element z at spos(z)
  // The FP32 register transforms keep the spectrum unpadded: every access to it is a run of
  // consecutive elements (16 of them, 128 bytes, cover the 32 banks once at any alignment),
  // while padded runs straddle pad slots and conflict. The other paths keep fpad's layout.
  constexpr bool SPAD = !((REG || R10) && F32);
  auto spos = [](int z) { return SPAD ? fpad(z) : z; };
  C* col = reinterpret_cast<C*>(smem);
  C* tw = col + 3 * tx * P;
  R* kh = reinterpret_cast<R*>(tw + NF);
  R* kl = kh + NF;
  R* kzs = kl + NF;
  C* cb_h = reinterpret_cast<C*>(kzs + NF);  // per column: beta hi
  C* cb_l = cb_h + tx;                        // beta lo
  C* cebl = cb_l + tx;                        // exp(i beta L)
  C* ce1 = cebl + tx;                         // exp(i beta dz)
  C* ce8 = ce1 + tx;                          // exp(i beta 8 dz)
  C* R0 = ce8 + tx;                           // 3 tx: T_R E(plane 0)
  C* ptab = R0 + 3 * tx;                      // tx phase_entries<NF>(): exp(i beta dz j)
  C* crs = ptab + tx * phase_pitch<NF>();     // FP32: r_s, r_p and beta / kb per column
  C* crp = crs + tx;
  C* cbq = crp + tx;
  R* cqx = reinterpret_cast<R*>(cbq + tx);
  R* cqy = cqx + tx;
  R* chx = cqy + tx;                           // FP32: unit transverse direction and |q| / kb
  R* chy = chx + tx;
  R* cqn = chy + tx;
  int* near = reinterpret_cast<int*>(cqn + tx);  // per column: the l of phi1's series, or -1

  const int x0 = blockIdx.x * tx, y = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  const int slot = a.rhsp[g].slot;  // loaded together with the activity flag
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  const int nx = a.nx, ny = a.ny, ns = a.nslab;
  const size_t mbase = ((size_t)slot * ny + y) * nx + x0;
  const size_t pstride = (size_t)ny * nx;
  constexpr int N2 = NF / 16, R1 = N2 > 0 ? 16 / N2 : 1;
  const int rf = threadIdx.x / (N2 > 0 ? N2 : 1), rj = threadIdx.x % (N2 > 0 ? N2 : 1);
  const bool rvalid = REG && rf < 3 * tx;
  // Register transform: lane rj of the group of column rf holds planes rj + N2 k (k < 8, the
  // nonzero half: ns + 1 <= NF/2), read straight from HBM. In FP32 the loads are issued
  // before the tables below are set up, so that their latency overlaps that work.
  C v[16];
  auto load_column = [&]() {
    if (rvalid) {
      const int cc = rf / tx, t = rf % tx;
      const C* src = a.work + ((size_t)lr * 3 + cc) * ns * pstride + (size_t)y * nx + x0 + t;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int n = rj + N2 * k;
        v[k] = (n >= 1 && n <= ns) ? src[(size_t)(n - 1) * pstride] : mk((R)0, (R)0);
      }
#pragma unroll
      for (int k = 8; k < 16; ++k) v[k] = mk((R)0, (R)0);
    }
  };
  if constexpr (REG && F32) load_column();

  for (int i = threadIdx.x; i < NF; i += NT) {
    tw[i] = twid<C>(a.twz, a.twz32, i);
    if constexpr (F32) {
      kh[i] = a.ktab32[i];
      kl[i] = a.ktab32[NF + i];
      kzs[i] = a.ktab32[2 * NF + i];
    } else {
      const double k = a.ktab64[i];
      kh[i] = fabs(k);
      kl[i] = 0.0;
      kzs[i] = k;
    }
  }
  const double two_pi = 6.283185307179586476925286766559;
  for (int t = threadIdx.x; t < tx; t += NT) {
    if constexpr (F32) {
      const ModeF32 m = a.modes32[mbase + t];
      cb_h[t] = m.bh;
      cb_l[t] = m.bl;
      cebl[t] = m.ebL;
      ce1[t] = m.e1;
      ce8[t] = m.e8;
      cqx[t] = m.qx;
      cqy[t] = m.qy;
      crs[t] = m.rs;
      crp[t] = m.rp;
      cbq[t] = m.bq;
      chx[t] = m.hx;
      chy[t] = m.hy;
      cqn[t] = m.qnk;
    } else {
      const RhsParam& rp = a.rhsp[g];
      const double qx64 = rp.qix + two_pi * (double)fft_freq(x0 + t, nx) / ((double)nx * a.dx);
      const double qy64 = rp.qiy + two_pi * (double)fft_freq(y, ny) / ((double)ny * a.dy);
      const ModeEntry me = a.modes[mbase + t];
      split_hi_lo(me.beta, cb_h[t], cb_l[t]);
      cebl[t] = from_c64<C>(me.ebL);
      ce1[t] = from_c64<C>(cexp_d(make_double2(-me.beta.y * a.dz, me.beta.x * a.dz)));
      ce8[t] = from_c64<C>(cexp_d(make_double2(-8.0 * me.beta.y * a.dz, 8.0 * me.beta.x * a.dz)));
      cqx[t] = (R)qx64;
      cqy[t] = (R)qy64;
    }
    near[t] = -1;
  }
  constexpr int HF = NF / 2;
  // thread -> (column t0, planes p0, p0 + pstep, ...): no divisions inside the copy loops
  const int t0 = threadIdx.x % tx, p0 = threadIdx.x / tx, pstep = NT / tx;
  C* gcol = a.work + (size_t)lr * 3 * ns * pstride + (size_t)y * nx + x0 + t0;
  constexpr int EP = 16 * (N2 + 1) <= P ? N2 + 1 : N2;  // exchange row pitch
  C* rex = col + (rvalid ? rf : 0) * P;  // the group's column: exchange scratch, then spectrum
  if constexpr (REG) {
    if constexpr (!F32) load_column();
    __syncthreads();  // twiddles
    if (rvalid) {
      reg_fft_step1<C, NF, false, true>(v, rj, tw);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) rex[k1 * EP + rj] = v[k1];
    }
    __syncwarp();
    C o[16];
    if (rvalid) reg_fft_step2<C, NF, false, EP>(rex, rj, o);
    __syncwarp();
    if (rvalid) {
#pragma unroll
      for (int r = 0; r < R1; ++r)
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) rex[spos(rj + N2 * r + 16 * k2)] = o[r * N2 + k2];
    }
  } else if constexpr (R10) {
    __syncthreads();  // twiddles
    const int gf = threadIdx.x >> 4, gj = threadIdx.x & 15;
    const bool gok = gf < 3 * tx;
    C* gx = col + (gok ? gf : 0) * P;  // the group's column: exchange (16 rows of 11), then spectrum
    if (gok && gj < 10) {
      // planes j + 10 k (k < 8: the nonzero half, ns + 1 <= NF/2) straight from HBM
      const int cc = gf / tx, t = gf % tx;
      const C* src = a.work + (size_t)lr * 3 * ns * pstride + (size_t)cc * ns * pstride + (size_t)y * nx + x0 + t;
      C v[16];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int n = gj + 10 * k;
        v[k] = (n >= 1 && n <= ns) ? src[(size_t)(n - 1) * pstride] : mk((R)0, (R)0);
      }
#pragma unroll
      for (int k = 8; k < 16; ++k) v[k] = mk((R)0, (R)0);
      DftHalf<C, 16, false>::run(v);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) gx[k1 * 11 + gj] = k1 ? cmul(v[k1], tw[gj * k1]) : v[k1];
    }
    __syncwarp();
    C w10[10];
    if (gok) {  // lane j: row k1 = j, outputs k1 + 16 k2
#pragma unroll
      for (int i = 0; i < 10; ++i) w10[i] = gx[gj * 11 + i];
      Dft<C, 10, false>::run(w10);
    }
    __syncwarp();
    if (gok) {
#pragma unroll
      for (int k2 = 0; k2 < 10; ++k2) gx[spos(gj + 16 * k2)] = w10[k2];
    }
  } else {
    // The forward transform reads only planes 0 .. NF/2-1 (its input vanishes above, as
    // ns + 1 <= NF/2): zero plane 0 and planes ns+1 .. NF/2-1, copy planes 1 .. ns.
    const int nz = HF - ns;
    for (int i = threadIdx.x; i < 3 * tx * nz; i += NT) {
      const int cc = i / nz, zz = i % nz;
      col[cc * P + fpad(zz == 0 ? 0 : ns + zz)] = mk((R)0, (R)0);
    }
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
#pragma unroll 4
      for (int pl = p0; pl < ns; pl += pstep)
        col[(cc * tx + t0) * P + fpad(pl + 1)] = gcol[((size_t)cc * ns + pl) * pstride];
    }
    __syncthreads();
    cta_fft<C, NF, false, false, 1, true>(col, 3 * tx, P, tw);
  }
  __syncthreads();

  // constants in the working precision (no FP64 arithmetic in the FP32 kernel)
  R dzr, kbr;  // FP32: rounded on the host (no FP64 conversion in every thread)
  if constexpr (F32) {
    dzr = a.dz32;
    kbr = a.kb32;
  } else {
    dzr = a.dz;
    kbr = a.kb;
  }
  const R L = (R)0.5 * (R)NF * dzr;
  const R cinv = (R)1 / (kbr * kbr);
  const R scale = (R)1 / ((R)NF * (R)nx * (R)ny);
  const bool sph = F32 ? a.sph32 != nullptr : a.sph64 != nullptr;
  if (sph) {
    // isolated clip: tabulated A, B/|k|^2 of |k|, shared by l and nf - l
    for (int i = threadIdx.x; i < tx * (HF + 1); i += NT) {
      const int t = i / (HF + 1), l = i % (HF + 1);
      const size_t o = (((size_t)slot * (HF + 1) + l) * ny + y) * nx + x0 + t;
      C A, Bt;
      if constexpr (F32) {
        const float4 v = a.sph32[o];
        A = mk(v.x, v.y);
        Bt = mk(v.z, v.w);
      } else {
        A = from_c64<C>(a.sph64[2 * o]);
        Bt = from_c64<C>(a.sph64[2 * o + 1]);
      }
      C* c0 = col + (0 * tx + t) * P;
      C* c1 = col + (1 * tx + t) * P;
      C* c2 = col + (2 * tx + t) * P;
      dyadic_sph(c0 + spos(l), c1 + spos(l), c2 + spos(l), cqx[t], cqy[t], kzs[l], A, Bt);
      if (l > 0 && l < HF)
        dyadic_sph(c0 + spos(NF - l), c1 + spos(NF - l), c2 + spos(NF - l), cqx[t], cqy[t], kzs[NF - l], A, Bt);
    }
  }
  // Pairs (l, nf - l) share S and E; l = 0 and l = nf/2 stand alone. Of each column's
  // l = 0 .. nf/2 at most one lies near the removable singularity (|delta L| < 1/2 needs
  // |Re(beta) L - pi l| < 1/2, and consecutive l are pi apart): the loop leaves it to the
  // pass after it, so that its warps do not diverge on phi1's series.
  constexpr int HL = HF + 1;
  auto apply_l = [&](int t, int l, C S, C Es) {
    const R qx = cqx[t], qy = cqy[t];
    C* c0 = col + (0 * tx + t) * P;
    C* c1 = col + (1 * tx + t) * P;
    C* c2 = col + (2 * tx + t) * P;
    dyadic_apply(c0 + spos(l), c1 + spos(l), c2 + spos(l), qx, qy, kzs[l], S, Es, cinv);
    if (l > 0 && l < HF)
      dyadic_apply(c0 + spos(NF - l), c1 + spos(NF - l), c2 + spos(NF - l), qx, qy, kzs[NF - l], S, Es, cinv);
  };
  for (int i = threadIdx.x; i < (sph ? 0 : tx * HL); i += NT) {
    // items (t, l < nf/2) in order, then (t, nf/2): a half-warp's l stay in one column
    const bool tail = i >= tx * HF;
    const int t = tail ? i - tx * HF : i / HF, l = tail ? HF : i % HF;
    C E = cebl[t];
    if (l & 1) E = cneg(E);
    C S, Es;
    if (!green_scalars_far(kh[l], kl[l], cb_h[t], cb_l[t], E, L, cinv, scale, S, Es)) {
      near[t] = l;
      continue;
    }
    apply_l(t, l, S, Es);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < (sph ? 0 : tx); t += NT) {
    const int l = near[t];
    if (l < 0) continue;
    C E = cebl[t];
    if (l & 1) E = cneg(E);
    C S, Es;
    green_scalars_near(kh[l], kl[l], cb_h[t], cb_l[t], E, L, cinv, scale, S, Es);
    apply_l(t, l, S, Es);
  }
  __syncthreads();
  // FP32 register transform: the output leaves from the registers (below); in FP64 the
  // longer live range of o[] cost more than the shared-memory round trip saves
  constexpr bool REG_OUT = REG && F32;
  C o[16];  // register transform: this lane's inverse outputs, planes rj + N2 r + 16 k2
  if constexpr (REG) {
    C v[16];
    if (rvalid) {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = rex[spos(rj + N2 * k)];
    }
    __syncwarp();
    if (rvalid) {
      reg_fft_step1<C, NF, true, false>(v, rj, tw);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) rex[k1 * EP + rj] = v[k1];
    }
    __syncwarp();
    if (rvalid) reg_fft_step2<C, NF, true, EP>(rex, rj, o);
    __syncwarp();
    if (rvalid) {  // to shared memory: planes 0 and ns + 1 (R0, side spectra), or all used ones
#pragma unroll
      for (int r = 0; r < R1; ++r)
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const int n = rj + N2 * r + 16 * k2;
          if (REG_OUT ? (n == 0 || n == ns + 1) : n <= HF) rex[spos(n)] = o[r * N2 + k2];
        }
    }
  } else if constexpr (R10) {
    const int gf = threadIdx.x >> 4, gj = threadIdx.x & 15;
    const bool gok = gf < 3 * tx;
    C* gx = col + (gok ? gf : 0) * P;
    C v[16];
    if (gok && gj < 10) {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = gx[spos(gj + 10 * k)];
      Dft<C, 16, true>::run(v);
    }
    __syncwarp();
    if (gok && gj < 10) {
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) gx[k1 * 11 + gj] = k1 ? cmul(v[k1], cconj(tw[gj * k1])) : v[k1];
    }
    __syncwarp();
    C w10[10];
    if (gok) {
#pragma unroll
      for (int i = 0; i < 10; ++i) w10[i] = gx[gj * 11 + i];
      Dft<C, 10, true>::run(w10);
    }
    __syncwarp();
    if (gok) {  // planes 0 .. NF/2 are the ones used below
#pragma unroll
      for (int k2 = 0; k2 < 10; ++k2) {
        const int n = gj + 16 * k2;
        if (n <= HF) gx[spos(n)] = w10[k2];
      }
    }
  } else {
    cta_fft<C, NF, true>(col, 3 * tx, P, tw);
  }
  __syncthreads();

  // normalised spectra of G*(V u) on plane 0 and plane ns+1
  if (a.side) {
    for (int i = threadIdx.x; i < 3 * tx; i += NT) {
      const int cc = i / tx, t = i % tx;
      const size_t o = (((size_t)g * 2) * 3 + cc) * ny * nx + (size_t)y * nx + x0 + t;
      a.side[o] = col[(cc * tx + t) * P];
      a.side[o + (size_t)3 * ny * nx] = col[(cc * tx + t) * P + spos(ns + 1)];
    }
  }
  // stack reflection of the downgoing field on plane 0: R0 = T_R E0 (Eq. (9)),
  // T_R = r_s s s^T + r_p p+ p-^T with s = z x q/|q|, p+- = (-+beta qhat, |q|)/kb.
  for (int t = threadIdx.x; t < tx; t += NT) {
    if constexpr (F32) {  // the column's mode constants were staged in shared memory
      const float hx = chx[t], hy = chy[t], qnk = cqn[t];
      const float2 bq = cbq[t];
      const float2 e0 = col[(0 * tx + t) * P], e1 = col[(1 * tx + t) * P], e2 = col[(2 * tx + t) * P];
      const float2 sE = mk(-hy * e0.x + hx * e1.x, -hy * e0.y + hx * e1.y);
      const float2 tq = cadd(cscale(e0, hx), cscale(e1, hy));
      const float2 pmE = cadd(cmul(bq, tq), cscale(e2, qnk));
      const float2 as = cmul(crs[t], sE), ap = cmul(crp[t], pmE);
      const float2 apb = cmul(ap, bq);
      R0[0 * tx + t] = csub(cscale(as, -hy), cscale(apb, hx));
      R0[1 * tx + t] = csub(cscale(as, hx), cscale(apb, hy));
      R0[2 * tx + t] = cscale(ap, qnk);
      continue;
    }
    const int x = x0 + t;
    const RhsParam& rp = a.rhsp[g];
    const ModeEntry me = a.modes[mbase + t];
    const double qx64 = rp.qix + two_pi * (double)fft_freq(x, nx) / ((double)nx * a.dx);
    const double qy64 = rp.qiy + two_pi * (double)fft_freq(y, ny) / ((double)ny * a.dy);
    const double qn = sqrt(qx64 * qx64 + qy64 * qy64);
    const double hx = qn > 0.0 ? qx64 / qn : rp.cphi;
    const double hy = qn > 0.0 ? qy64 / qn : rp.sphi;
    const double2 e0 = as_c64(col[(0 * tx + t) * P]);
    const double2 e1 = as_c64(col[(1 * tx + t) * P]);
    const double2 e2 = as_c64(col[(2 * tx + t) * P]);
    const double ikb = 1.0 / a.kb;
    // s . E0 and p- . E0 (bilinear)
    const double2 sE = make_double2(-hy * e0.x + hx * e1.x, -hy * e0.y + hx * e1.y);
    const double2 bq = cscale(me.beta, ikb);  // beta / kb
    const double2 tq = cadd(cscale(e0, hx), cscale(e1, hy));
    const double2 pmE = cadd(cmul(bq, tq), cscale(e2, qn * ikb));  // (+beta qhat . E + |q| Ez)/kb
    const double2 as = cmul(me.rs, sE);
    const double2 ap = cmul(me.rp, pmE);
    // r_s s (s.E) + r_p p+ (p-.E), p+ = (-beta hx, -beta hy, |q|)/kb
    const double2 mbq = cneg(bq);
    const double2 Rx = cadd(cscale(as, -hy), cmul(ap, cscale(mbq, hx)));
    const double2 Ry = cadd(cscale(as, hx), cmul(ap, cscale(mbq, hy)));
    const double2 Rz = cscale(ap, qn * ikb);
    R0[0 * tx + t] = from_c64<C>(Rx);
    R0[1 * tx + t] = from_c64<C>(Ry);
    R0[2 * tx + t] = from_c64<C>(Rz);
  }
  // phase table: powers of exp(i beta dz) (fine, j < 8) and of exp(i beta 8 dz) (coarse),
  // both evaluated in FP64; every entry by binary powering in its own thread
  constexpr int PE = phase_entries<NF>(), PP = phase_pitch<NF>();
  for (int i = threadIdx.x; i < tx * PE; i += NT) {
    const int t = i / PE, j = i % PE;
    C w = j < 8 ? ce1[t] : ce8[t];
    int e = j < 8 ? j : j - 8;
    C r = mk((R)1, (R)0);
    while (e) {
      if (e & 1) r = cmul(r, w);
      e >>= 1;
      if (e) w = cmul(w, w);
    }
    ptab[t * PP + j] = r;
  }
  __syncthreads();
  const bool reflect = !a.no_reflect;  // the free-space operator adds no reflection
  if constexpr (REG_OUT) {
    // straight from the registers: plane pl = n - 1 gets R0 exp(i beta pl dz); a warp's four
    // columns are consecutive x-modes, so each plane is written as one 32- (64-) byte run.
    // The planes of one r share pl mod 16 = jm, so R0 exp(i beta jm dz) is formed once and
    // each plane multiplies it by exp(i beta 16 dz (pl >> 4)) (coarse entry 2 (pl >> 4)).
    if (rvalid) {
      const int cc = rf / tx, t = rf % tx;
      const C* pt = ptab + t * PP;
      C* dst = a.work + ((size_t)lr * 3 + cc) * ns * pstride + (size_t)y * nx + x0 + t;
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const int jm = (rj + N2 * r + 15) & 15;
        const C rb = reflect ? cmul(R0[cc * tx + t], cmul(pt[jm & 7], pt[8 + (jm >> 3)])) : mk((R)0, (R)0);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const int n = rj + N2 * r + 16 * k2;
          if (n >= 1 && n <= ns) {
            const int pl = n - 1;
            C val = o[r * N2 + k2];
            if (reflect) val = cadd(val, cmul(rb, pt[8 + 2 * (pl >> 4)]));
            dst[(size_t)pl * pstride] = val;
          }
        }
      }
    }
  } else {
    const int pl_end = reflect ? ns : 0;
    for (int pl = p0; pl < pl_end; pl += pstep) {
      const C ph = cmul(ptab[t0 * PP + (pl & 7)], ptab[t0 * PP + 8 + (pl >> 3)]);  // exp(i beta pl dz)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        C* e = col + (cc * tx + t0) * P + spos(pl + 1);
        *e = cadd(*e, cmul(R0[cc * tx + t0], ph));
      }
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
#pragma unroll 4
      for (int pl = p0; pl < ns; pl += pstep)
        gcol[((size_t)cc * ns + pl) * pstride] = col[(cc * tx + t0) * P + spos(pl + 1)];
    }
  }
}

}  // namespace psfd
