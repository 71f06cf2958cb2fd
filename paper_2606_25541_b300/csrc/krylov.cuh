// krylov.cuh -- BiCGStab building blocks: vector updates fused with their dot products,
// and per-RHS scalar kernels that reduce the partial sums in a fixed order.
//
// The paper solves its systems with GMRES (Sec. 3); the solver here is BiCGStab, a
// short-recurrence Krylov method whose memory and traffic do not grow with the
// iteration count. Every right-hand side carries its own scalars and convergence flag;
// partial sums are written per block and reduced in a fixed order, so the result of a
// right-hand side does not depend on which others share the batch.
#pragma once

#include "op_kernels.cuh"
#include "../../include/psfd.h"

namespace psfd {

constexpr int VEC_NT = 256;

__device__ __forceinline__ bool finite_c(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Deterministic block sum of partials[0 .. n) (stride 1) into every thread's return value.
__device__ __forceinline__ double2 block_sum_fixed(const double2* part, int n, double2* sh) {
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = cadd(acc, part[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sh[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0.0, 0.0);
    for (int w = 0; w < nw; ++w) s = cadd(s, sh[w]);
    sh[32] = s;
  }
  __syncthreads();
  double2 r = sh[32];
  __syncthreads();
  return r;
}

template <typename C>
__device__ __forceinline__ void vec_block_dots(typename Acc<C>::T d0, typename Acc<C>::T d2, int mask,
                                               double2* dst, int stride) {
  __shared__ double2 sh[NDOT * 32];
  Dots<C> dt;
  dt.d[0] = d0;
  dt.d[1] = mk((typename RealOf<C>::T)0, (typename RealOf<C>::T)0);
  dt.d[2] = d2;
  block_write_dots(dt, mask, dst, stride, sh);
}

// x = 0, r = r0 = b, p = v = 0; partial ||b||^2 into slot 2 (right-hand sides in mask only).
template <typename C>
__global__ void __launch_bounds__(VEC_NT) k_bicg_init(int n, int nblk, int rhs0, const int* mask, const C* b, C* x,
                                                       C* r, C* r0, C* p, C* v, double2* partials, int maxblk) {
  using R = typename RealOf<C>::T;
  const int blk = blockIdx.x, lr = blockIdx.y, g = rhs0 + lr;
  if (mask && !mask[g]) return;
  const size_t off = (size_t)lr * n;
  const int chunk = (n + nblk - 1) / nblk;
  const int lo = blk * chunk, hi = min(n, lo + chunk);
  const C z = mk((R)0, (R)0);
  typename Acc<C>::T bb = z;
  for (int i = lo + threadIdx.x; i < hi; i += VEC_NT) {
    const C bi = b[off + i];
    x[off + i] = z;
    r[off + i] = bi;
    r0[off + i] = bi;
    p[off + i] = z;
    v[off + i] = z;
    bb.x += bi.x * bi.x + bi.y * bi.y;
  }
  vec_block_dots<C>(z, bb, DOT_OUT_OUT, partials + ((size_t)g * NDOT) * maxblk + blk, maxblk);
}

// x += alpha p + omega s; r = s - omega t; partials <r0, r> (slot 0) and ||r||^2 (slot 2).
// The current p is read from pn; when pn is not p it is also copied into p.
template <typename C>
__global__ void __launch_bounds__(VEC_NT) k_bicg_xr(int n, int nblk, int rhs0, const int* act, const KScal* sc,
                                                     C* x, const C* pn, C* p, const C* s, const C* t, C* r,
                                                     const C* r0, double2* partials, int maxblk,
                                                     unsigned* ctac) {
  using R = typename RealOf<C>::T;
  const int blk = blockIdx.x, lr = blockIdx.y, g = rhs0 + lr;
  if (!act[g]) return;
  if (ctac && threadIdx.x == 0) atomicAdd(ctac, 1u);
  const size_t off = (size_t)lr * n;
  const C al = from_c64<C>(sc[g].alpha), om = from_c64<C>(sc[g].omega);
  typename Acc<C>::T d0 = mk((R)0, (R)0), d2 = d0;
  auto elem = [&](C si, C pk, C xk, C tk, C zk, C& xo, C& ro) {
    xo = cadd(xk, cadd(cmul(al, pk), cmul(om, si)));
    ro = csub(si, cmul(om, tk));
    d0 = cadd(d0, cmulc(zk, ro));
    d2.x += ro.x * ro.x + ro.y * ro.y;
  };
  if constexpr (sizeof(C) == 8) {
    // FP32: two elements per 16-byte access (n is even, so every chunk starts 16-byte aligned)
    const int chunk = (((n + nblk - 1) / nblk) + 1) & ~1;
    const int lo = blk * chunk, hi = min(n, lo + chunk);
    auto ld = [](const C* q) { return *reinterpret_cast<const float4*>(q); };
    auto lo2 = [](float4 v) { return make_float2(v.x, v.y); };
    auto hi2 = [](float4 v) { return make_float2(v.z, v.w); };
    for (int i = lo + 2 * (int)threadIdx.x; i < hi; i += 2 * VEC_NT) {
      const size_t k = off + i;
      const float4 S = ld(s + k), Pn = ld(pn + k), X = ld(x + k), T = ld(t + k), Z = ld(r0 + k);
      if (pn != p) *reinterpret_cast<float4*>(p + k) = Pn;
      C x0, x1, r0v, r1v;
      elem(lo2(S), lo2(Pn), lo2(X), lo2(T), lo2(Z), x0, r0v);
      elem(hi2(S), hi2(Pn), hi2(X), hi2(T), hi2(Z), x1, r1v);
      *reinterpret_cast<float4*>(x + k) = make_float4(x0.x, x0.y, x1.x, x1.y);
      *reinterpret_cast<float4*>(r + k) = make_float4(r0v.x, r0v.y, r1v.x, r1v.y);
    }
  } else {
    const int chunk = (n + nblk - 1) / nblk;
    const int lo = blk * chunk, hi = min(n, lo + chunk);
    for (int i = lo + threadIdx.x; i < hi; i += VEC_NT) {
      const size_t k = off + i;
      const C si = s[k], pk = pn[k];
      if (pn != p) p[k] = pk;
      C xo, ro;
      elem(si, pk, x[k], t[k], r0[k], xo, ro);
      x[k] = xo;
      r[k] = ro;
    }
  }
  vec_block_dots<C>(d0, d2, DOT_R0_OUT | DOT_OUT_OUT, partials + ((size_t)g * NDOT) * maxblk + blk, maxblk);
}

__device__ __forceinline__ const double2* slot_ptr(const double2* partials, int g, int slot, int maxblk) {
  return partials + ((size_t)g * NDOT + slot) * maxblk;
}

// ||b||^2 -> scalars and activity (b != 0) for the right-hand sides in mask (null = all);
// the others keep their state.
static __global__ void __launch_bounds__(VEC_NT) k_scal_init(int rhs0, int nblk, const double2* partials, int maxblk,
                                                       const int* mask, double tol, const double* tol_slot,
                                                       KScal* sc, int* act) {
  __shared__ double2 sh[33];
  const int g = rhs0 + blockIdx.x;
  if (mask && !mask[g]) return;
  const double2 bb = block_sum_fixed(slot_ptr(partials, g, 2, maxblk), nblk, sh);
  if (threadIdx.x == 0) {
    KScal s;
    s.bnorm2 = bb.x;
    s.rnorm2 = bb.x;
    s.rho = make_double2(bb.x, 0.0);
    s.alpha = make_double2(1.0, 0.0);
    s.omega = make_double2(1.0, 0.0);
    s.beta = make_double2(0.0, 0.0);
    s.scale = sc[g].scale;
    const double t = tol_slot ? tol_slot[g] : tol;
    s.tol2 = t * t;
    s.iters = 0;
    s.status = PSFD_OK;
    s.active = bb.x > 0.0;
    s.pad = 0;
    sc[g] = s;
    act[g] = s.active;
  }
}

// alpha = rho / <r0, v>
static __global__ void __launch_bounds__(VEC_NT) k_scal_alpha(int rhs0, int nblk, const double2* partials, int maxblk,
                                                        KScal* sc, int* act) {
  __shared__ double2 sh[33];
  const int g = rhs0 + blockIdx.x;
  if (!act[g]) return;
  const double2 sig = block_sum_fixed(slot_ptr(partials, g, 0, maxblk), nblk, sh);
  if (threadIdx.x == 0) {
    if (!(finite_c(sig)) || (sig.x == 0.0 && sig.y == 0.0)) {
      sc[g].status = PSFD_E_BREAKDOWN;
      sc[g].active = 0;
      act[g] = 0;
      sc[g].alpha = make_double2(0.0, 0.0);
    } else {
      sc[g].alpha = cdiv(sc[g].rho, sig);
    }
  }
}

// omega = <t, s> / <t, t>   (t = A s)
static __global__ void __launch_bounds__(VEC_NT) k_scal_omega(int rhs0, int nblk, const double2* partials, int maxblk,
                                                        KScal* sc, int* act) {
  __shared__ double2 sh[33];
  const int g = rhs0 + blockIdx.x;
  if (!act[g]) return;
  const double2 ts = block_sum_fixed(slot_ptr(partials, g, 1, maxblk), nblk, sh);
  const double2 tt = block_sum_fixed(slot_ptr(partials, g, 2, maxblk), nblk, sh);
  if (threadIdx.x == 0) {
    if (tt.x > 0.0 && isfinite(tt.x) && finite_c(ts))
      sc[g].omega = make_double2(ts.x / tt.x, ts.y / tt.x);
    else
      sc[g].omega = make_double2(0.0, 0.0);
  }
}

// rho_new = <r0, r>, convergence test on ||r||, beta = (rho_new / rho)(alpha / omega).
static __global__ void __launch_bounds__(VEC_NT) k_scal_rho(int rhs0, int nblk, const double2* partials, int maxblk,
                                                      int max_iter, KScal* sc, int* act) {
  __shared__ double2 sh[33];
  const int g = rhs0 + blockIdx.x;
  if (!act[g]) return;
  const double2 rn = block_sum_fixed(slot_ptr(partials, g, 0, maxblk), nblk, sh);
  const double2 rr = block_sum_fixed(slot_ptr(partials, g, 2, maxblk), nblk, sh);
  if (threadIdx.x == 0) {
    KScal s = sc[g];
    s.iters += 1;
    s.rnorm2 = rr.x;
    if (!isfinite(rr.x)) {
      s.status = PSFD_E_BREAKDOWN;
      s.active = 0;
    } else if (rr.x <= s.tol2 * s.bnorm2) {
      s.active = 0;
    } else if (s.iters >= max_iter) {
      s.status = PSFD_E_NOT_CONVERGED;
      s.active = 0;
    } else if (!finite_c(rn) || (rn.x == 0.0 && rn.y == 0.0) || (s.omega.x == 0.0 && s.omega.y == 0.0)) {
      s.status = PSFD_E_BREAKDOWN;
      s.active = 0;
    } else {
      s.beta = cmul(cdiv(rn, s.rho), cdiv(s.alpha, s.omega));
      s.rho = rn;
    }
    sc[g] = s;
    act[g] = s.active;
  }
}

}  // namespace psfd
