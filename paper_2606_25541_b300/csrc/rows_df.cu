// rows_df.cu -- the row passes (x transforms) of the FP64 residual's split planes with the
// transforms in double-float arithmetic.
//
// The refined solve's certifying residual r = b - A x (FP64 vectors) splits planes larger than
// 64 x 64 into a row pass and a column pass in each direction. The row passes carry the input
// stage (J = V x) and the epilogue (r = b - (x - w) with ||r||^2); their transforms along x are
// the other half of the residual's FP64 transform work. Here they run on FP32 pairs
// (dfloat.cuh), like the column and z passes, so that the FP64 pipe only converts:
//   forward: x and V converted on load (one exact FP64 operation per real), J = V x and the
//            transform in double-float;
//   inverse: the transform in double-float, w converted on output, the epilogue and the
//            norm in FP64 as before.
// With wdf set, the spectral work array between the passes holds double-float pairs
// (dfc, 16 bytes like double2) instead of FP64, so the column and z passes convert nothing;
// the whole chain then converts only x, V, b and r.
#include "../../include/psfd.h"
#include "dfloat.cuh"
#include "dfloat_ops.h"
#include "op_launch.cuh"

namespace psfd {
namespace {

constexpr int kRowNT = 256;

// Rows per CTA: the FP64 row pass's choice, so that the epilogue's partial sums have the
// layout the FP64 path (and op_blocks_per_rhs) expects.
int df_row_block(int nx, int ny) { return row_block(nx, ny, Tune<double2>::ROW_ELEMS); }

template <int NX>
size_t rows_df_smem(int rb, bool inv) {
  size_t b = (size_t)(rb * fft_phys(NX) + NX) * sizeof(dfc);
  if (inv) b += 16 + NDOT * 32 * sizeof(double2);
  return b;
}

// grid (3 nrhs, ny / rb, nslab) as k_rows_fwd (V's rows shared by neighbouring CTAs)
template <int NX, bool WDF>
__global__ void __launch_bounds__(kRowNT, 2) k_rows_fwd_df(OpCall<double2> a, int rb) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int RP = fft_phys(NX);
  dfc* tile = reinterpret_cast<dfc*>(smem);
  dfc* tw = tile + rb * RP;
  const int p = blockIdx.z, y0 = blockIdx.y * rb;
  const int c = blockIdx.x % 3, lr = blockIdx.x / 3, g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  for (int i = threadIdx.x; i < NX; i += kRowNT) tw[i] = a.twxdf ? dfc_of(a.twxdf[i]) : to_dfc(a.twx[i]);
  const size_t base = ((((size_t)lr * 3 + c) * a.nslab + p) * a.ny + y0) * (size_t)NX;
  const size_t voff = (((size_t)a.rhsp[g].clip * a.nslab + p) * a.ny + y0) * NX;
  const double2* Vp = a.V + voff;
  const float4* Vq = a.Vdf ? a.Vdf + voff : nullptr;  // V as pairs: no conversion of V here
  const int n = rb * NX;
  for (int i0 = threadIdx.x; i0 < n; i0 += 2 * kRowNT) {
    double2 uu[2];
    dfc vv[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = i0 + j * kRowNT;
      if (i < n) {
        uu[j] = a.u[base + i];
        vv[j] = Vq ? dfc_of(Vq[i]) : to_dfc(Vp[i]);
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = i0 + j * kRowNT;
      if (i < n) tile[(i / NX) * RP + fpad(i % NX)] = cmul(vv[j], to_dfc(uu[j]));
    }
  }
  __syncthreads();
  cta_fft<dfc, NX, false>(tile, rb, RP, tw);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kRowNT) {
    const dfc v = tile[(i / NX) * RP + fpad(i % NX)];
    if constexpr (WDF) reinterpret_cast<dfc*>(a.work)[base + i] = v;
    else a.work[base + i] = to_d2(v);
  }
}

// grid (nslab (ny / rb), 3, nrhs) as k_rows_inv (its partial-sum block index too)
template <int NX, int EPI, bool WDF>
__global__ void __launch_bounds__(kRowNT, 2) k_rows_inv_df(OpCall<double2> a, const double2* uin, int rb) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int RP = fft_phys(NX);
  dfc* tile = reinterpret_cast<dfc*>(smem);
  dfc* tw = tile + rb * RP;
  double2* scratch = align16<double2>(tw + NX);
  const int nrb = a.ny / rb;
  const int p = blockIdx.x / nrb, y0 = (blockIdx.x % nrb) * rb;
  const int c = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  for (int i = threadIdx.x; i < NX; i += kRowNT) tw[i] = a.twxdf ? dfc_of(a.twxdf[i]) : to_dfc(a.twx[i]);
  const size_t base = ((((size_t)lr * 3 + c) * a.nslab + p) * a.ny + y0) * (size_t)NX;
  const int n = rb * NX;
  for (int i = threadIdx.x; i < n; i += kRowNT) {
    dfc v;
    if constexpr (WDF) v = reinterpret_cast<const dfc*>(a.work)[base + i];
    else v = to_dfc(a.work[base + i]);
    tile[(i / NX) * RP + fpad(i % NX)] = v;
  }
  __syncthreads();
  cta_fft<dfc, NX, true>(tile, rb, RP, tw);
  __syncthreads();
  Dots<double2> dt;
  zero_dots(dt);
  for (int i0 = threadIdx.x; i0 < n; i0 += 2 * kRowNT) {
    EpiVals<double2> e[2];
#pragma unroll
    for (int j = 0; j < 2; ++j)
      if (i0 + j * kRowNT < n) e[j] = load_epi<double2, EPI>(a, uin, base + i0 + j * kRowNT);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = i0 + j * kRowNT;
      if (i < n) store_epi<double2, EPI>(a, base + i, e[j], to_d2(tile[(i / NX) * RP + fpad(i % NX)]), dt);
    }
  }
  if (a.dot_mask) {
    const int blk = (c * a.nslab + p) * nrb + (y0 / rb);
    block_write_dots(dt, a.dot_mask, a.partials + ((size_t)g * NDOT) * a.maxblk + blk, a.maxblk, scratch);
  }
}

template <int NX>
int launch_fwd(const OpCall<double2>& a, bool wdf) {
  const int rb = df_row_block(NX, a.ny);
  const size_t smem = rows_df_smem<NX>(rb, false);
  auto k = wdf ? k_rows_fwd_df<NX, true> : k_rows_fwd_df<NX, false>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PSFD_E_CUDA;
  k<<<dim3(3 * a.nrhs, a.ny / rb, a.nslab), kRowNT, smem, a.stream>>>(a, rb);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA;
}

template <int NX, int EPI>
int launch_inv(const OpCall<double2>& a, const double2* uin, bool wdf) {
  const int rb = df_row_block(NX, a.ny);
  const size_t smem = rows_df_smem<NX>(rb, true);
  auto k = wdf ? k_rows_inv_df<NX, EPI, true> : k_rows_inv_df<NX, EPI, false>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PSFD_E_CUDA;
  k<<<dim3(a.nslab * (a.ny / rb), 3, a.nrhs), kRowNT, smem, a.stream>>>(a, uin, rb);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA;
}

}  // namespace

// Row lengths 64, 128 and 256 of split FP64 planes, the plain input stage and the epilogues
// out = u - w and b - (u - w).
bool rows_df_supported(const OpCall<double2>& a) {
  return (a.nx == 64 || a.nx == 128 || a.nx == 256) && !use_fused<double2>(a.nx, a.ny) && a.in_mode == IN_PLAIN &&
         (a.epi == EPI_AU || a.epi == EPI_RESID);
}

int launch_rows_fwd_df(const OpCall<double2>& a, bool wdf) {
  if (!rows_df_supported(a)) return PSFD_E_ARG;
  switch (a.nx) {
    case 64: return launch_fwd<64>(a, wdf);
    case 128: return launch_fwd<128>(a, wdf);
    default: return launch_fwd<256>(a, wdf);
  }
}

int launch_rows_inv_df(const OpCall<double2>& a, const double2* uin, bool wdf) {
  if (!rows_df_supported(a)) return PSFD_E_ARG;
  const bool resid = a.epi == EPI_RESID;
  switch (a.nx) {
    case 64: return resid ? launch_inv<64, EPI_RESID>(a, uin, wdf) : launch_inv<64, EPI_AU>(a, uin, wdf);
    case 128: return resid ? launch_inv<128, EPI_RESID>(a, uin, wdf) : launch_inv<128, EPI_AU>(a, uin, wdf);
    default: return resid ? launch_inv<256, EPI_RESID>(a, uin, wdf) : launch_inv<256, EPI_AU>(a, uin, wdf);
  }
}

}  // namespace psfd
