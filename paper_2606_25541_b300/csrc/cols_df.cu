// cols_df.cu -- the y pass of the FP64 residual's split-plane transforms (planes above 64 x 64
// in FP64 do not fit one CTA and run as a row pass and a column pass) with the transform in
// double-float arithmetic.
//
// Same data movement as the FP64 column pass: tx consecutive columns of one plane of the
// spectral work array are gathered into shared memory, transformed along y in place
// (Sec. 3, Eq. (18): every convolution is an FFT), and written back; only the Stockham stages
// run on FP32 pairs (dfloat.cuh) instead of the FP64 pipe. The work array holds FP64, or
// double-float pairs when every pass of the chain is double-float (wdf).
#include "../../include/psfd.h"
#include "dfloat.cuh"
#include "dfloat_ops.h"
#include "fft.cuh"

namespace psfd {
namespace {

constexpr int kColTile = 8;  // columns per CTA
constexpr int kColNT = 256;

template <int NY>
size_t cols_df_smem(int tx) {
  return (size_t)(tx * (fft_phys(NY) | 1) + NY) * sizeof(dfc);
}

// blockIdx.x = plane * (nx / tx) + column block; blockIdx.y = component; blockIdx.z = rhs.
template <int NY, bool INV, bool WDF>
__global__ void __launch_bounds__(kColNT, 2) k_cols_df(OpCall<double2> a, int tx) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PITCH = fft_phys(NY) | 1;
  dfc* tile = reinterpret_cast<dfc*>(smem);
  dfc* tw = tile + tx * PITCH;
  const int ncb = a.nx / tx;
  const int p = blockIdx.x / ncb, x0 = (blockIdx.x % ncb) * tx;
  const int c = blockIdx.y, lr = blockIdx.z, g = a.rhs0 + lr;
  if (a.active && !a.active[g]) return;
  if (a.ctac && threadIdx.x == 0) atomicAdd(a.ctac, 1u);  // profiling: CTAs that did work
  for (int i = threadIdx.x; i < NY; i += kColNT) tw[i] = a.twydf ? dfc_of(a.twydf[i]) : to_dfc(a.twy[i]);
  const size_t base = (((size_t)lr * 3 + c) * a.nslab + p) * (size_t)NY * a.nx + x0;
  const int t0 = threadIdx.x % tx, y0 = threadIdx.x / tx, ystep = kColNT / tx;
  dfc* wd = reinterpret_cast<dfc*>(a.work);
  for (int y = y0; y < NY; y += ystep) {
    const size_t o = base + (size_t)y * a.nx + t0;
    tile[t0 * PITCH + fpad(y)] = WDF ? wd[o] : to_dfc(a.work[o]);
  }
  __syncthreads();
  cta_fft<dfc, NY, INV>(tile, tx, PITCH, tw);
  __syncthreads();
  for (int y = y0; y < NY; y += ystep) {
    const size_t o = base + (size_t)y * a.nx + t0;
    if constexpr (WDF) wd[o] = tile[t0 * PITCH + fpad(y)];
    else a.work[o] = to_d2(tile[t0 * PITCH + fpad(y)]);
  }
}

template <int NY, bool INV>
int launch(const OpCall<double2>& a, int tx, bool wdf) {
  const size_t smem = cols_df_smem<NY>(tx);
  auto k = wdf ? k_cols_df<NY, INV, true> : k_cols_df<NY, INV, false>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PSFD_E_CUDA;
  k<<<dim3(a.nslab * (a.nx / tx), 3, a.nrhs), kColNT, smem, a.stream>>>(a, tx);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA;
}

}  // namespace

// Column lengths 128 and 256 with eight-column tiles (nx a multiple of 8).
bool cols_df_supported(const OpCall<double2>& a) {
  return (a.ny == 128 || a.ny == 256) && a.nx % kColTile == 0;
}

int launch_cols_df(const OpCall<double2>& a, bool inverse, bool wdf) {
  if (!cols_df_supported(a)) return PSFD_E_ARG;
  if (a.ny == 128) return inverse ? launch<128, true>(a, kColTile, wdf) : launch<128, false>(a, kColTile, wdf);
  return inverse ? launch<256, true>(a, kColTile, wdf) : launch<256, false>(a, kColTile, wdf);
}

}  // namespace psfd
