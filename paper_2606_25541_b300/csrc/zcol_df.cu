// zcol_df.cu -- the z-column pass (K2) of the FP64 residual with its transforms and dyadic
// products in double-float arithmetic.
//
// The refined solve certifies every illumination with r = b - A x in FP64 (defect
// correction around the FP32 Krylov sweeps). On B300 that residual is bound by the FP64
// pipe, and K2 -- six length-nf transforms and a 3x3 complex product per wavevector --
// carries most of its FP64 work. This kernel computes the same pass as the FP64 k_zcol
// (Sec. 3, Eq. (18): zero padding to nf, FFT_z, the windowed dyadic Green's function,
// IFFT_z, and the stack reflection of Eq. (9) folded in), reading and writing the FP64
// spectra, with
//   - the forward and inverse z transforms (the register four-step transform, 16 x nf/16)
//     and the dyadic products in double-float (dfloat.cuh: ~48 significant bits);
//   - the Green's scalars S_l, E_l in double-float too (the FP32 reciprocal refined by a
//     Newton step; the same closed forms and series as the FP64 kernel);
//   - the reflection T_R E(plane 0) and the per-column exponentials in FP64 (a few dozen
//     FP64 operations per column, not per element);
//   - the reflection phase table by binary powering in double-float.
// Columns of length 64 and 128 on the periodic (z-windowed) kernel; other lengths and the
// isolated clip's spherical kernel stay on the FP64 k_zcol.
#include "../../include/psfd.h"
#include "dfloat.cuh"
#include "dfloat_ops.h"
#include "op_kernels.cuh"

namespace psfd {
namespace {

constexpr int kDfTile = 8;  // x-modes per CTA

// dynamic shared memory: columns, twiddles, R0, phase table (16-byte entries), then the
// per-column FP64 and double-float constants and the kz tables (8-byte entries)
template <int NF>
__host__ __device__ constexpr int df_pitch() { return fft_phys(NF) | 1; }
template <int NF>
size_t df_smem_bytes(int tx) {
  const size_t c16 = (size_t)3 * tx * df_pitch<NF>() + NF + 3 * tx + (size_t)tx * phase_pitch<NF>();
  // beta, exp(i beta L) (FP64), exp(i beta dz), exp(i beta 8 dz), beta, exp(i beta L) (double-float), (qx, qy)
  const size_t c16col = 7 * (size_t)tx;
  const size_t c8 = 2 * (size_t)NF;               // kz (dfr) and kz (FP64)
  return (c16 + c16col) * 16 + c8 * 8 + 16;
}

// 1 / x in double-float: the FP32 reciprocal refined by one Newton step, r (1 + (1 - x r)),
// relative error about 2^-46.
__device__ __forceinline__ dfr df_recip(dfr x) {
  const dfr r(__frcp_rn(x.hi), 0.0f);
  const dfr e = dfr(1.0f, 0.0f) - x * r;
  return r + r * e;
}
// a / b = conj(b) a / |b|^2 in double-float
__device__ __forceinline__ dfc df_cdiv(dfc a, dfc b) {
  const dfr inv = df_recip(b.x * b.x + b.y * b.y);
  const dfc n = cmulc(b, a);
  return mk(n.x * inv, n.y * inv);
}
// 1/K as the nearest double-float (compile-time constants)
template <int K> struct DfInv {
  static constexpr float hi = (float)(1.0 / K);
  static constexpr float lo = (float)(1.0 / K - (double)(float)(1.0 / K));
};
// phi1(w) = 1 + w/2 (1 + w/3 (1 + ...)) by Horner from the K-th term down
template <int K>
__device__ __forceinline__ void df_phi1_horner(dfc w, dfc& phi) {
  const dfc t = cmul(w, phi);
  const dfr ik(DfInv<K>::hi, DfInv<K>::lo);
  phi = mk(dfr(1.0f, 0.0f) + t.x * ik, t.y * ik);
  if constexpr (K > 2) df_phi1_horner<K - 1>(w, phi);
}
// The windowed Green's scalars of one mode at |kz| = kap (the same closed forms as the FP64
// and FP32 kernels, Sec. 3's one-dimensional window): with delta = beta - kap and E =
// (-1)^l exp(i beta L), S = (E - 1) / (delta (kap + beta)), or i L phi1(i delta L) / (kap + beta)
// by its Taylor series where |delta L| < 1/2 (15 terms: below 1e-15 there); both scaled by the
// inverse-transform normalisation, Es = E / kb^2 likewise.
__device__ __forceinline__ void green_scalars_df(dfr kap, dfc beta, dfc E, dfr L, dfr cinv, dfr scale, dfc& S,
                                                 dfc& Es) {
  const dfc d = mk(beta.x - kap, beta.y);
  const dfc kpb = mk(kap + beta.x, beta.y);
  const dfc w = mk(-(d.y * L), d.x * L);
  if (w.x.hi * w.x.hi + w.y.hi * w.y.hi < 0.25f) {
    dfc phi = mk(dfr(1.0f, 0.0f), dfr(0.0f, 0.0f));
    df_phi1_horner<15>(w, phi);
    S = df_cdiv(mk(-(phi.y * L), phi.x * L), kpb);
  } else {
    S = df_cdiv(mk(E.x - dfr(1.0f, 0.0f), E.y), cmul(d, kpb));
  }
  S = mk(S.x * scale, S.y * scale);
  const dfr es = cinv * scale;
  Es = mk(E.x * es, E.y * es);
}

// CTAs per SM the kernel is compiled for: at nf = 128 three (96 registers, a few bytes of
// spill) measured faster than two at 168 registers (the pass is issue- and latency-bound,
// so resident warps count more than the spill); 1 = no register cap.
template <int NF> __host__ __device__ constexpr int df_min_blocks() { return NF == 128 ? 3 : 1; }

template <int NF, int NT, bool WDF>
__global__ void __launch_bounds__(NT, df_min_blocks<NF>()) k_zcol_df(OpCall<double2> a, int tx) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int P = df_pitch<NF>();
  constexpr int PE = phase_entries<NF>(), PP = phase_pitch<NF>();
  constexpr int HF = NF / 2;
  constexpr int N2 = NF / 16, R1 = 16 / N2;
  constexpr int EP = 16 * (N2 + 1) <= P ? N2 + 1 : N2;  // exchange row pitch
  dfc* col = reinterpret_cast<dfc*>(smem);
  dfc* tw = col + 3 * tx * P;
  dfc* R0 = tw + NF;            // 3 tx: T_R E(plane 0)
  dfc* ptab = R0 + 3 * tx;      // tx PP: exp(i beta dz j), j < 8, and exp(i beta 8 dz j')
  double2* cbeta = reinterpret_cast<double2*>(ptab + tx * PP);
  double2* cebl = cbeta + tx;   // exp(i beta L)
  dfc* ce1 = reinterpret_cast<dfc*>(cebl + tx);  // exp(i beta dz)
  dfc* ce8 = ce1 + tx;                            // exp(i beta 8 dz)
  dfc* cbeta_d = ce8 + tx;                        // beta
  dfc* cebl_d = cbeta_d + tx;                      // exp(i beta L)
  dfr* cq = reinterpret_cast<dfr*>(cebl_d + tx);  // 2 tx: qx, qy
  dfr* kzd = cq + 2 * tx;       // signed kz_l
  double* kz64 = reinterpret_cast<double*>(kzd + NF);

  const int x0 = blockIdx.x * tx, y = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  const int nx = a.nx, ny = a.ny, ns = a.nslab;
  const RhsParam& rp = a.rhsp[g];
  const size_t mbase = ((size_t)rp.slot * ny + y) * nx + x0;
  const double two_pi = 6.283185307179586476925286766559;

  for (int i = threadIdx.x; i < NF; i += NT) {
    tw[i] = to_dfc(a.twz[i]);
    kz64[i] = a.ktab64[i];
    kzd[i] = to_dfr(a.ktab64[i]);
  }
  for (int t = threadIdx.x; t < tx; t += NT) {
    const ModeEntry me = a.modes[mbase + t];
    cbeta[t] = me.beta;
    cebl[t] = me.ebL;
    cbeta_d[t] = to_dfc(me.beta);
    cebl_d[t] = to_dfc(me.ebL);
    ce1[t] = to_dfc(cexp_d(make_double2(-me.beta.y * a.dz, me.beta.x * a.dz)));
    ce8[t] = to_dfc(cexp_d(make_double2(-8.0 * me.beta.y * a.dz, 8.0 * me.beta.x * a.dz)));
    cq[2 * t] = to_dfr(rp.qix + two_pi * (double)fft_freq(x0 + t, nx) / ((double)nx * a.dx));
    cq[2 * t + 1] = to_dfr(rp.qiy + two_pi * (double)fft_freq(y, ny) / ((double)ny * a.dy));
  }
  const size_t pstride = (size_t)ny * nx;
  const int rf = threadIdx.x / N2, rj = threadIdx.x % N2;
  const bool rvalid = rf < 3 * tx;
  dfc* rex = col + (rvalid ? rf : 0) * P;  // the group's column: exchange scratch, then spectrum
  const dfc zero = mk(dfr(0.0), dfr(0.0));
  __syncthreads();  // twiddles
  {
    // forward: planes j + N2 k (k < 8, the nonzero half: ns + 1 <= NF/2) straight from HBM
    dfc v[16];
    if (rvalid) {
      const int cc = rf / tx, t = rf % tx;
      const size_t so = ((size_t)lr * 3 + cc) * ns * pstride + (size_t)y * nx + x0 + t;
      const double2* src = a.work + so;
      const dfc* srcd = reinterpret_cast<const dfc*>(a.work) + so;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int n = rj + N2 * k;
        if (n >= 1 && n <= ns) v[k] = WDF ? srcd[(size_t)(n - 1) * pstride] : to_dfc(src[(size_t)(n - 1) * pstride]);
        else v[k] = zero;
      }
#pragma unroll
      for (int k = 8; k < 16; ++k) v[k] = zero;
      reg_fft_step1<dfc, NF, false, true>(v, rj, tw);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) rex[k1 * EP + rj] = v[k1];
    }
    __syncwarp();
    dfc o[16];
    if (rvalid) reg_fft_step2<dfc, NF, false, EP>(rex, rj, o);
    __syncwarp();
    if (rvalid) {
#pragma unroll
      for (int r = 0; r < R1; ++r)
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) rex[fpad(rj + N2 * r + 16 * k2)] = o[r * N2 + k2];
    }
  }
  __syncthreads();

  // Green's scalars (one evaluation serves l and nf - l) and products in double-float
  const dfr L_d = to_dfr(0.5 * (double)NF * a.dz);
  const dfr cinv_d = to_dfr(1.0 / (a.kb * a.kb));
  const dfr scale_d = to_dfr(1.0 / ((double)NF * (double)nx * (double)ny));
  for (int i = threadIdx.x; i < tx * (HF + 1); i += NT) {
    const int t = i / (HF + 1), l = i % (HF + 1);
    dfc E = cebl_d[t];
    if (l & 1) E = cneg(E);
    const dfr kz = kzd[l];
    const dfr kap = kz.hi < 0.0f ? -kz : kz;
    dfc Sd, Ed;
    green_scalars_df(kap, cbeta_d[t], E, L_d, cinv_d, scale_d, Sd, Ed);
    const dfr qx = cq[2 * t], qy = cq[2 * t + 1];
    dfc* c0 = col + (0 * tx + t) * P;
    dfc* c1 = col + (1 * tx + t) * P;
    dfc* c2 = col + (2 * tx + t) * P;
    dyadic_apply<dfc>(c0 + fpad(l), c1 + fpad(l), c2 + fpad(l), qx, qy, kzd[l], Sd, Ed, cinv_d);
    if (l > 0 && l < HF)
      dyadic_apply<dfc>(c0 + fpad(NF - l), c1 + fpad(NF - l), c2 + fpad(NF - l), qx, qy, kzd[NF - l], Sd, Ed,
                        cinv_d);
  }
  __syncthreads();
  {
    // inverse transform; planes 0 .. NF/2 back to the group's column
    dfc v[16];
    if (rvalid) {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = rex[fpad(rj + N2 * k)];
    }
    __syncwarp();
    if (rvalid) {
      reg_fft_step1<dfc, NF, true, false>(v, rj, tw);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) rex[k1 * EP + rj] = v[k1];
    }
    __syncwarp();
    dfc o[16];
    if (rvalid) reg_fft_step2<dfc, NF, true, EP>(rex, rj, o);
    __syncwarp();
    if (rvalid) {
#pragma unroll
      for (int r = 0; r < R1; ++r)
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const int n = rj + N2 * r + 16 * k2;
          if (n <= HF) rex[fpad(n)] = o[r * N2 + k2];
        }
    }
  }
  __syncthreads();

  // normalised spectra of G*(V u) on plane 0 and plane ns+1
  if (a.side) {
    for (int i = threadIdx.x; i < 3 * tx; i += NT) {
      const int cc = i / tx, t = i % tx;
      const size_t o = (((size_t)g * 2) * 3 + cc) * ny * nx + (size_t)y * nx + x0 + t;
      a.side[o] = to_d2(col[(cc * tx + t) * P]);
      a.side[o + (size_t)3 * ny * nx] = to_d2(col[(cc * tx + t) * P + fpad(ns + 1)]);
    }
  }
  // stack reflection of the downgoing field on plane 0 (Eq. (9)) in FP64, once per column:
  // R0 = T_R E0, T_R = r_s s s^T + r_p p+ p-^T, s = z x q/|q|, p+- = (-+beta qhat, |q|)/kb
  for (int t = threadIdx.x; t < tx; t += NT) {
    const ModeEntry me = a.modes[mbase + t];
    const double qx64 = rp.qix + two_pi * (double)fft_freq(x0 + t, nx) / ((double)nx * a.dx);
    const double qy64 = rp.qiy + two_pi * (double)fft_freq(y, ny) / ((double)ny * a.dy);
    const double qn = sqrt(qx64 * qx64 + qy64 * qy64);
    const double hx = qn > 0.0 ? qx64 / qn : rp.cphi;
    const double hy = qn > 0.0 ? qy64 / qn : rp.sphi;
    const double2 e0 = to_d2(col[(0 * tx + t) * P]);
    const double2 e1 = to_d2(col[(1 * tx + t) * P]);
    const double2 e2 = to_d2(col[(2 * tx + t) * P]);
    const double ikb = 1.0 / a.kb;
    const double2 sE = make_double2(-hy * e0.x + hx * e1.x, -hy * e0.y + hx * e1.y);
    const double2 bq = cscale(me.beta, ikb);
    const double2 tq = cadd(cscale(e0, hx), cscale(e1, hy));
    const double2 pmE = cadd(cmul(bq, tq), cscale(e2, qn * ikb));
    const double2 as = cmul(me.rs, sE);
    const double2 ap = cmul(me.rp, pmE);
    const double2 mbq = cneg(bq);
    R0[0 * tx + t] = to_dfc(cadd(cscale(as, -hy), cmul(ap, cscale(mbq, hx))));
    R0[1 * tx + t] = to_dfc(cadd(cscale(as, hx), cmul(ap, cscale(mbq, hy))));
    R0[2 * tx + t] = to_dfc(cscale(ap, qn * ikb));
  }
  // phase table: powers of exp(i beta dz) (j < 8) and of exp(i beta 8 dz) (steps from FP64)
  // by binary powering in double-float
  for (int i = threadIdx.x; i < tx * PE; i += NT) {
    const int t = i / PE, j = i % PE;
    dfc w = j < 8 ? ce1[t] : ce8[t];
    int e = j < 8 ? j : j - 8;
    dfc r = mk(dfr(1.0), dfr(0.0));
    while (e) {
      if (e & 1) r = cmul(r, w);
      e >>= 1;
      if (e) w = cmul(w, w);
    }
    ptab[t * PP + j] = r;
  }
  __syncthreads();
  // planes 1 .. ns: add R0 exp(i beta (p - 1) dz), write back as FP64
  const int t0 = threadIdx.x % tx, p0 = threadIdx.x / tx, pstep = NT / tx;
  if (!a.no_reflect) {
    for (int pl = p0; pl < ns; pl += pstep) {
      const dfc ph = cmul(ptab[t0 * PP + (pl & 7)], ptab[t0 * PP + 8 + (pl >> 3)]);
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        dfc* e = col + (cc * tx + t0) * P + fpad(pl + 1);
        *e = cadd(*e, cmul(R0[cc * tx + t0], ph));
      }
    }
    __syncthreads();
  }
  const size_t go = (size_t)lr * 3 * ns * pstride + (size_t)y * nx + x0 + t0;
  double2* gcol = a.work + go;
  dfc* gcold = reinterpret_cast<dfc*>(a.work) + go;
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
#pragma unroll 4
    for (int pl = p0; pl < ns; pl += pstep) {
      const dfc v = col[(cc * tx + t0) * P + fpad(pl + 1)];
      if constexpr (WDF) gcold[((size_t)cc * ns + pl) * pstride] = v;
      else gcol[((size_t)cc * ns + pl) * pstride] = to_d2(v);
    }
  }
}

template <int NF>
int launch(const OpCall<double2>& a, bool wdf) {
  constexpr int NT = 24 * (NF / 16);
  int tx = a.nx < kDfTile ? a.nx : kDfTile;
  const size_t smem = df_smem_bytes<NF>(tx);
  auto k = wdf ? k_zcol_df<NF, NT, true> : k_zcol_df<NF, NT, false>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PSFD_E_CUDA;
  k<<<dim3(a.nx / tx, a.ny, a.nrhs), NT, smem, a.stream>>>(a, tx);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA;
}

}  // namespace

// Lengths 64 and 128, the periodic kernel, and x tiles of 1, 2, 4 or 8 modes that divide nx
// (the plane loop of the write-back needs the tile to divide the CTA).
bool zcol_df_supported(const OpCall<double2>& a) {
  const int tx = a.nx < kDfTile ? a.nx : kDfTile;
  return (a.nf == 64 || a.nf == 128) && a.sph64 == nullptr && tx >= 1 && (tx & (tx - 1)) == 0 && a.nx % tx == 0;
}

int launch_zcol_df(const OpCall<double2>& a, bool wdf) {
  if (!zcol_df_supported(a)) return PSFD_E_ARG;
  return a.nf == 64 ? launch<64>(a, wdf) : launch<128>(a, wdf);
}

}  // namespace psfd
