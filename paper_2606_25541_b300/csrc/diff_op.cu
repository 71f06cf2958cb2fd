// diff_op.cu -- the conventional (differential) PSFD operator of a periodic clip with PMLs in z
// (Sec. 3, Eqs. (4)-(7)): out = curl curl E - k0^2 eps E, FP64, on Bloch envelopes.
//
// The paper's comparator for the Lippmann-Schwinger form: derivatives are spectral (Eq. (6)),
// along x and y exact per transverse mode (d/dx -> i q_x, q = q_inc + 2 pi m / P), along z by
// FFT over the column divided by the PML stretch s(z) = 1 + i sigma(z) (Eq. (7)). The PML
// profile is not given in the paper; this one is cubic, sigma(z) = sigma_max (depth/L)^3 over
// n_pml planes at both ends, sigma_max = -4 ln(1e-8) / (2 kb L). Three passes:
//   D1  FFT_xy of every (component, plane)                          -> work
//   D2  per mode: the two curls, each z derivative an FFT_z pair    -> work
//   D3  inverse FFT_xy, out = W / (nx ny) - k0^2 eps E
#include <cmath>

#include "../../include/psfd.h"
#include "fft.cuh"
#include "internal.h"

namespace psfd {
namespace {

struct DiffArgs {
  int nx, ny, nz, n_pml;
  double dx, dy, dz, k0, kb, qix, qiy, smax;
  const double2* eps;  // [z][y][x]
  const double2* E;    // [3][z][y][x]
  double2* out;        // [3][z][y][x]
  double2* work;       // [3][z][y][x]
};

__device__ void fill_twiddles(double2* tw, int n) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    double s, c;
    sincospi(-2.0 * t / n, &s, &c);
    tw[t] = make_double2(c, s);
  }
}

__device__ __forceinline__ double2 pml_inv_stretch(const DiffArgs& a, int z) {
  const double Lp = a.n_pml * a.dz, zc = (z + 0.5) * a.dz;
  const double depth = fmax(fmax(Lp - zc, zc - (a.nz * a.dz - Lp)), 0.0);
  const double t = a.n_pml > 0 ? depth / Lp : 0.0;
  const double2 s = make_double2(1.0, a.smax * t * t * t);
  return cdiv(make_double2(1.0, 0.0), s);
}

// D1 / D3: one CTA per (plane, component); the plane sits in shared memory at
// fpad(y) * PITCH + fpad(x) and is transformed along x, then y (inverse: y, then x).
template <int N, bool INV>
__global__ void __launch_bounds__(256) k_diff_plane(DiffArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PITCH = fft_phys(N) | 1;
  double2* tile = reinterpret_cast<double2*>(smem);
  double2* tw = tile + fft_phys(N) * PITCH;
  const int z = blockIdx.x, c = blockIdx.y;
  fill_twiddles(tw, N);
  const size_t base = ((size_t)c * a.nz + z) * N * N;
  const double2* src = INV ? a.work : a.E;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) tile[fpad(i / N) * PITCH + fpad(i % N)] = src[base + i];
  __syncthreads();
  if (!INV) {
    cta_fft<double2, N, false, true, 1>(tile, N, PITCH, tw);
    __syncthreads();
    cta_fft<double2, N, false, true, PITCH>(tile, N, 1, tw);
  } else {
    cta_fft<double2, N, true, true, PITCH>(tile, N, 1, tw);
    __syncthreads();
    cta_fft<double2, N, true, true, 1>(tile, N, PITCH, tw);
  }
  __syncthreads();
  if (!INV) {
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) a.work[base + i] = tile[fpad(i / N) * PITCH + fpad(i % N)];
  } else {
    const double inv = 1.0 / ((double)N * N), k02 = a.k0 * a.k0;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
      const size_t pz = (size_t)z * N * N + i;
      const double2 w = cscale(tile[fpad(i / N) * PITCH + fpad(i % N)], inv);
      a.out[base + i] = csub(w, cscale(cmul(a.eps[pz], a.E[base + i]), k02));
    }
  }
}

// D2: one CTA per transverse mode; columns of length NZ in shared memory.
template <int NZ>
__global__ void __launch_bounds__(128) k_diff_column(DiffArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int P = fft_phys(NZ) | 1;
  double2* col = reinterpret_cast<double2*>(smem);  // [8][P]: E x,y,z; C x,y,z; T0, T1
  double2* tw = col + 8 * P;
  double2* sinv = tw + NZ;  // 1 / s(z)
  const int x = blockIdx.x, y = blockIdx.y, nx = a.nx, ny = a.ny;
  fill_twiddles(tw, NZ);
  for (int z = threadIdx.x; z < NZ; z += blockDim.x) sinv[z] = pml_inv_stretch(a, z);
  const double two_pi = 6.283185307179586476925286766559;
  const double qx = a.qix + two_pi * fft_freq(x, nx) / (nx * a.dx);
  const double qy = a.qiy + two_pi * fft_freq(y, ny) / (ny * a.dy);
  const size_t pstride = (size_t)nx * ny, cstride = (size_t)a.nz * pstride, off = (size_t)y * nx + x;
  for (int i = threadIdx.x; i < 3 * NZ; i += blockDim.x) {
    const int c = i / NZ, z = i % NZ;
    col[c * P + fpad(z)] = a.work[c * cstride + z * pstride + off];
  }
  __syncthreads();
  double2* E = col;
  double2* Cc = col + 3 * P;
  double2* T = col + 6 * P;
  // T0 = d/dz f0, T1 = d/dz f1 (spectral, stretched)
  auto dz2 = [&](const double2* f0, const double2* f1) {
    for (int z = threadIdx.x; z < NZ; z += blockDim.x) {
      T[fpad(z)] = f0[fpad(z)];
      T[P + fpad(z)] = f1[fpad(z)];
    }
    __syncthreads();
    cta_fft<double2, NZ, false>(T, 2, P, tw);
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * NZ; i += blockDim.x) {
      const int c = i / NZ, l = i % NZ;
      const double kz = two_pi * fft_freq(l, NZ) / (NZ * a.dz);
      double2& v = T[c * P + fpad(l)];
      v = cscale(cmul_i(v), kz / NZ);
    }
    __syncthreads();
    cta_fft<double2, NZ, true>(T, 2, P, tw);
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * NZ; i += blockDim.x) {
      const int c = i / NZ, z = i % NZ;
      double2& v = T[c * P + fpad(z)];
      v = cmul(v, sinv[z]);
    }
    __syncthreads();
  };
  // curl E: (i qy Ez - dz Ey, dz Ex - i qx Ez, i qx Ey - i qy Ex)
  dz2(E + 1 * P, E + 0 * P);
  for (int z = threadIdx.x; z < NZ; z += blockDim.x) {
    const int o = fpad(z);
    const double2 ex = E[o], ey = E[P + o], ez = E[2 * P + o];
    Cc[o] = csub(cscale(cmul_i(ez), qy), T[o]);
    Cc[P + o] = csub(T[P + o], cscale(cmul_i(ez), qx));
    Cc[2 * P + o] = csub(cscale(cmul_i(ey), qx), cscale(cmul_i(ex), qy));
  }
  __syncthreads();
  // curl curl E, written back to the work buffer
  dz2(Cc + 1 * P, Cc + 0 * P);
  for (int z = threadIdx.x; z < NZ; z += blockDim.x) {
    const int o = fpad(z);
    const double2 cx = Cc[o], cy = Cc[P + o], cz = Cc[2 * P + o];
    a.work[0 * cstride + z * pstride + off] = csub(cscale(cmul_i(cz), qy), T[o]);
    a.work[1 * cstride + z * pstride + off] = csub(T[P + o], cscale(cmul_i(cz), qx));
    a.work[2 * cstride + z * pstride + off] = csub(cscale(cmul_i(cy), qx), cscale(cmul_i(cx), qy));
  }
}

template <int N>
int launch_plane(const DiffArgs& a, bool inv, cudaStream_t st) {
  const size_t smem = (size_t)(fft_phys(N) * (fft_phys(N) | 1) + N) * sizeof(double2);
  auto k = inv ? k_diff_plane<N, true> : k_diff_plane<N, false>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PSFD_E_CUDA;
  k<<<dim3(a.nz, 3), 256, smem, st>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA;
}

template <int NZ>
int launch_column(const DiffArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(8 * (fft_phys(NZ) | 1) + 2 * NZ) * sizeof(double2);
  auto k = k_diff_column<NZ>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return PSFD_E_CUDA;
  k<<<dim3(a.nx, a.ny), 128, smem, st>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA;
}

}  // namespace
}  // namespace psfd

extern "C" int psfd_apply_differential(int n, int nz, int n_pml, double dx, double dz, double wavelength,
                                       double eps_bg, double theta_deg, double phi_deg, const double* eps,
                                       const double* E, double* out, double* work, void* stream) {
  using namespace psfd;
  if (!(n == 8 || n == 16 || n == 32 || n == 64) || !(nz == 32 || nz == 64 || nz == 128) || n_pml < 0 ||
      2 * n_pml >= nz || !(dx > 0) || !(dz > 0) || !(wavelength > 0) || !(eps_bg > 0) || !eps || !E || !out || !work)
    return PSFD_E_ARG;
  DiffArgs a;
  a.nx = a.ny = n;
  a.nz = nz;
  a.n_pml = n_pml;
  a.dx = a.dy = dx;
  a.dz = dz;
  const double pi = 3.14159265358979323846;
  a.k0 = 2.0 * pi / wavelength;
  a.kb = a.k0 * std::sqrt(eps_bg);
  const double th = theta_deg * pi / 180.0, ph = phi_deg * pi / 180.0;
  a.qix = a.kb * std::sin(th) * std::cos(ph);
  a.qiy = a.kb * std::sin(th) * std::sin(ph);
  a.smax = n_pml > 0 ? -4.0 * std::log(1e-8) / (2.0 * a.kb * n_pml * dz) : 0.0;
  a.eps = reinterpret_cast<const double2*>(eps);
  a.E = reinterpret_cast<const double2*>(E);
  a.out = reinterpret_cast<double2*>(out);
  a.work = reinterpret_cast<double2*>(work);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = PSFD_E_ARG;
  auto planes = [&](bool inv) {
    switch (n) {
      case 8: return launch_plane<8>(a, inv, st);
      case 16: return launch_plane<16>(a, inv, st);
      case 32: return launch_plane<32>(a, inv, st);
      default: return launch_plane<64>(a, inv, st);
    }
  };
  if ((rc = planes(false)) != PSFD_OK) return rc;
  switch (nz) {
    case 32: rc = launch_column<32>(a, st); break;
    case 64: rc = launch_column<64>(a, st); break;
    default: rc = launch_column<128>(a, st); break;
  }
  if (rc != PSFD_OK) return rc;
  return planes(true);
}
