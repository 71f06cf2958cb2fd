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
//   - the reflection T_R E(plane 0) in double-float, from per-mode pairs (beta, exp(i beta L),
//     exp(i beta dz), exp(i beta 8 dz), r_s, r_p, q and its direction) that the FP64 stack
//     kernel prepares once per illumination set-up: the pass itself runs no FP64 operation
//     (this GPU's FP64 pipe is slow, and the per-column FP64 work ran in a few threads while
//     the rest of the CTA waited at a barrier);
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
  // per column: beta, exp(i beta L), exp(i beta dz), exp(i beta 8 dz), r_s, r_p, beta / kb
  const size_t c16col = 7 * (size_t)tx;
  const size_t c8 = (size_t)NF + 5 * (size_t)tx;  // kz_l; qx, qy, hx, hy, |q| / kb per column
  return (c16 + c16col) * 16 + c8 * 8 + (size_t)tx * sizeof(int) + 16;
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
// false (and nothing written) near the removable singularity, |delta L| < 1/2: that case is
// green_scalars_df_near's
__device__ __forceinline__ bool green_scalars_df_far(dfr kap, dfc beta, dfc E, dfr L, dfr cinv, dfr scale, dfc& S,
                                                     dfc& Es) {
  const dfc d = mk(beta.x - kap, beta.y);
  const dfc kpb = mk(kap + beta.x, beta.y);
  const dfc w = mk(-(d.y * L), d.x * L);
  if (w.x.hi * w.x.hi + w.y.hi * w.y.hi < 0.25f) return false;
  S = df_cdiv(mk(E.x - dfr(1.0f, 0.0f), E.y), cmul(d, kpb));
  S = mk(S.x * scale, S.y * scale);
  const dfr es = cinv * scale;
  Es = mk(E.x * es, E.y * es);
  return true;
}
__device__ __forceinline__ void green_scalars_df_near(dfr kap, dfc beta, dfc E, dfr L, dfr cinv, dfr scale, dfc& S,
                                                      dfc& Es) {
  const dfc d = mk(beta.x - kap, beta.y);
  const dfc kpb = mk(kap + beta.x, beta.y);
  const dfc w = mk(-(d.y * L), d.x * L);
  dfc phi = mk(dfr(1.0f, 0.0f), dfr(0.0f, 0.0f));
  df_phi1_horner<15>(w, phi);
  S = df_cdiv(mk(-(phi.y * L), phi.x * L), kpb);
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
  dfc* R0 = tw + NF;             // 3 tx: T_R E(plane 0)
  dfc* ptab = R0 + 3 * tx;       // tx PP: exp(i beta dz j), j < 8, and exp(i beta 8 dz j')
  dfc* cbeta_d = ptab + tx * PP;  // per column (from the mode table's pairs): beta
  dfc* cebl_d = cbeta_d + tx;     // exp(i beta L)
  dfc* ce1 = cebl_d + tx;         // exp(i beta dz)
  dfc* ce8 = ce1 + tx;            // exp(i beta 8 dz)
  dfc* crs = ce8 + tx;            // r_s, r_p, beta / kb
  dfc* crp = crs + tx;
  dfc* cbq = crp + tx;
  dfr* cq = reinterpret_cast<dfr*>(cbq + tx);  // 2 tx: qx, qy
  dfr* chx = cq + 2 * tx;         // unit transverse direction, |q| / kb
  dfr* chy = chx + tx;
  dfr* cqn = chy + tx;
  dfr* kzd = cqn + tx;            // signed kz_l
  int* near = reinterpret_cast<int*>(kzd + NF);  // per column: the l of phi1's series, or -1

  const int x0 = blockIdx.x * tx, y = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  const int slot = a.rhsp[g].slot;  // loaded together with the activity flag
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  const int nx = a.nx, ny = a.ny, ns = a.nslab;
  const size_t mbase = ((size_t)slot * ny + y) * nx + x0;
  const size_t pstride = (size_t)ny * nx;
  const int rf = threadIdx.x / N2, rj = threadIdx.x % N2;
  const bool rvalid = rf < 3 * tx;
  dfc* rex = col + (rvalid ? rf : 0) * P;  // the group's column: exchange scratch, then spectrum
  const dfc zero = mk(dfr(0.0), dfr(0.0));
  for (int i = threadIdx.x; i < NF; i += NT) {
    tw[i] = dfc_of(a.twzdf[i]);
    kzd[i] = dfr_of(a.kzdf[i]);
  }
  for (int t = threadIdx.x; t < tx; t += NT) {
    const ModeDF& m = a.modesdf[mbase + t];
    cbeta_d[t] = dfc_of(m.beta);
    cebl_d[t] = dfc_of(m.ebL);
    ce1[t] = dfc_of(m.e1);
    ce8[t] = dfc_of(m.e8);
    crs[t] = dfc_of(m.rs);
    crp[t] = dfc_of(m.rp);
    cbq[t] = dfc_of(m.bq);
    cq[2 * t] = dfr_of(m.qx);
    cq[2 * t + 1] = dfr_of(m.qy);
    chx[t] = dfr_of(m.hx);
    chy[t] = dfr_of(m.hy);
    cqn[t] = dfr_of(m.qnk);
    near[t] = -1;
  }
  // forward: planes j + N2 k (k < 8, the nonzero half: ns + 1 <= NF/2) straight from HBM,
  // issued before the barrier (earlier, their registers would spill under the cap)
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
  }

  __syncthreads();  // twiddles
  {
    if (rvalid) {
      reg_fft_step1<dfc, NF, false, true>(v, rj, tw);
#pragma unroll
      for (int k1 = 0; k1 < 16; ++k1) rex[k1 * EP + rj] = v[k1];
    }
    __syncwarp();
    dfc o[16];
    if (rvalid) reg_fft_step2<dfc, NF, false, EP>(rex, rj, o);
    __syncwarp();
    if (rvalid) {
      // the spectrum stays unpadded: every access to it is a run of consecutive elements
#pragma unroll
      for (int r = 0; r < R1; ++r)
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) rex[rj + N2 * r + 16 * k2] = o[r * N2 + k2];
    }
  }
  __syncthreads();

  // Green's scalars (one evaluation serves l and nf - l) and products in double-float. Items
  // run column by column (l < nf/2, then l = nf/2), so a quarter-warp's l stay in one column;
  // each column's one l near the removable singularity (|delta L| < 1/2) is left to the pass
  // after the loop, so that no warp diverges on phi1's series.
  const dfr L_d = dfr_of(a.dfL), cinv_d = dfr_of(a.dfcinv), scale_d = dfr_of(a.dfscale);
  auto apply_l = [&](int t, int l, dfc Sd, dfc Ed) {
    const dfr qx = cq[2 * t], qy = cq[2 * t + 1];
    dfc* c0 = col + (0 * tx + t) * P;
    dfc* c1 = col + (1 * tx + t) * P;
    dfc* c2 = col + (2 * tx + t) * P;
    dyadic_apply<dfc>(c0 + l, c1 + l, c2 + l, qx, qy, kzd[l], Sd, Ed, cinv_d);
    if (l > 0 && l < HF) dyadic_apply<dfc>(c0 + (NF - l), c1 + (NF - l), c2 + (NF - l), qx, qy, kzd[NF - l], Sd, Ed, cinv_d);
  };
  auto kappa = [&](int l) {
    const dfr kz = kzd[l];
    return kz.hi < 0.0f ? -kz : kz;
  };
  for (int i = threadIdx.x; i < tx * (HF + 1); i += NT) {
    const bool tail = i >= tx * HF;
    const int t = tail ? i - tx * HF : i / HF, l = tail ? HF : i % HF;
    dfc E = cebl_d[t];
    if (l & 1) E = cneg(E);
    dfc Sd, Ed;
    if (!green_scalars_df_far(kappa(l), cbeta_d[t], E, L_d, cinv_d, scale_d, Sd, Ed)) {
      near[t] = l;
      continue;
    }
    apply_l(t, l, Sd, Ed);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < tx; t += NT) {
    const int l = near[t];
    if (l < 0) continue;
    dfc E = cebl_d[t];
    if (l & 1) E = cneg(E);
    dfc Sd, Ed;
    green_scalars_df_near(kappa(l), cbeta_d[t], E, L_d, cinv_d, scale_d, Sd, Ed);
    apply_l(t, l, Sd, Ed);
  }
  __syncthreads();
  {
    // inverse transform; planes 0 .. NF/2 back to the group's column
    dfc v[16];
    if (rvalid) {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = rex[rj + N2 * k];
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
          if (n <= HF) rex[n] = o[r * N2 + k2];
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
      a.side[o + (size_t)3 * ny * nx] = to_d2(col[(cc * tx + t) * P + ns + 1]);
    }
  }
  // stack reflection of the downgoing field on plane 0 (Eq. (9)) in double-float, once per
  // column: R0 = T_R E0, T_R = r_s s s^T + r_p p+ p-^T, s = z x q/|q|, p+- = (-+beta qhat, |q|)/kb
  for (int t = threadIdx.x; t < tx; t += NT) {
    const dfr hx = chx[t], hy = chy[t], qnk = cqn[t];
    const dfc bq = cbq[t];
    const dfc e0 = col[(0 * tx + t) * P], e1 = col[(1 * tx + t) * P], e2 = col[(2 * tx + t) * P];
    const dfc sE = mk(e1.x * hx - e0.x * hy, e1.y * hx - e0.y * hy);  // s . E0
    const dfc tq = mk(e0.x * hx + e1.x * hy, e0.y * hx + e1.y * hy);  // qhat . E0
    const dfc pmE = cadd(cmul(bq, tq), mk(e2.x * qnk, e2.y * qnk));   // p- . E0
    const dfc as = cmul(crs[t], sE), ap = cmul(crp[t], pmE);
    const dfc apb = cmul(ap, bq);
    R0[0 * tx + t] = mk(-(as.x * hy) - apb.x * hx, -(as.y * hy) - apb.y * hx);
    R0[1 * tx + t] = mk(as.x * hx - apb.x * hy, as.y * hx - apb.y * hy);
    R0[2 * tx + t] = mk(ap.x * qnk, ap.y * qnk);
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
        dfc* e = col + (cc * tx + t0) * P + pl + 1;
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
      const dfc v = col[(cc * tx + t0) * P + pl + 1];
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
  return (a.nf == 64 || a.nf == 128) && a.sph64 == nullptr && a.modesdf && a.twzdf && a.kzdf && tx >= 1 &&
         (tx & (tx - 1)) == 0 && a.nx % tx == 0;
}

int launch_zcol_df(const OpCall<double2>& a, bool wdf) {
  if (!zcol_df_supported(a)) return PSFD_E_ARG;
  return a.nf == 64 ? launch<64>(a, wdf) : launch<128>(a, wdf);
}

}  // namespace psfd
