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
//   - the Green's scalars S_l, E_l, the reflection T_R E(plane 0) and the per-column
//     exponentials in FP64 (a few dozen FP64 operations per column, not per element);
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
  const size_t c16col = 5 * (size_t)tx;           // beta, exp(i beta L), exp(i beta dz), exp(i beta 8 dz), (qx, qy)
  const size_t c8 = 2 * (size_t)NF;               // kz (dfr) and kz (FP64)
  return (c16 + c16col) * 16 + c8 * 8 + 16;
}

// CTAs per SM the kernel is compiled for: at nf = 128 three (96 registers, a few bytes of
// spill) measured faster than two at 168 registers (the pass is issue- and latency-bound,
// so resident warps count more than the spill); 1 = no register cap.
template <int NF> __host__ __device__ constexpr int df_min_blocks() { return NF == 128 ? 3 : 1; }

template <int NF, int NT>
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
  dfr* cq = reinterpret_cast<dfr*>(ce8 + tx);     // 2 tx: qx, qy
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
      const double2* src = a.work + ((size_t)lr * 3 + cc) * ns * pstride + (size_t)y * nx + x0 + t;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int n = rj + N2 * k;
        v[k] = (n >= 1 && n <= ns) ? to_dfc(src[(size_t)(n - 1) * pstride]) : zero;
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

  // Green's scalars in FP64 (one evaluation serves l and nf - l), products in double-float
  const double L = 0.5 * (double)NF * a.dz;
  const double cinv = 1.0 / (a.kb * a.kb);
  const double scale = 1.0 / ((double)NF * (double)nx * (double)ny);
  const dfr cinv_d = to_dfr(cinv);
  for (int i = threadIdx.x; i < tx * (HF + 1); i += NT) {
    const int t = i / (HF + 1), l = i % (HF + 1);
    double2 E = cebl[t];
    if (l & 1) E = cneg(E);
    double2 S, Es;
    green_scalars<double2>(fabs(kz64[l]), 0.0, cbeta[t], make_double2(0.0, 0.0), E, L, cinv, scale, S, Es);
    const dfc Sd = to_dfc(S), Ed = to_dfc(Es);
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
  double2* gcol = a.work + (size_t)lr * 3 * ns * pstride + (size_t)y * nx + x0 + t0;
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
#pragma unroll 4
    for (int pl = p0; pl < ns; pl += pstep)
      gcol[((size_t)cc * ns + pl) * pstride] = to_d2(col[(cc * tx + t0) * P + fpad(pl + 1)]);
  }
}

template <int NF>
int launch(const OpCall<double2>& a) {
  constexpr int NT = 24 * (NF / 16);
  int tx = a.nx < kDfTile ? a.nx : kDfTile;
  const size_t smem = df_smem_bytes<NF>(tx);
  auto k = k_zcol_df<NF, NT>;
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

int launch_zcol_df(const OpCall<double2>& a) {
  if (!zcol_df_supported(a)) return PSFD_E_ARG;
  return a.nf == 64 ? launch<64>(a) : launch<128>(a);
}

}  // namespace psfd
