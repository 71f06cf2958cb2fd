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
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

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
      // without eps: the plain inverse transform (the spectral damping preconditioner)
      a.out[base + i] = a.eps ? csub(w, cscale(cmul(a.eps[pz], a.E[base + i]), k02)) : w;
    }
  }
}

// Spectral damping on the column's 3-D Fourier grid (the middle pass): per transverse mode,
// FFT_z of the three components, times D(k) = min(1, kb^2 / |k|^2) / nz, inverse FFT_z.
template <int NZ>
__global__ void __launch_bounds__(128) k_damp_column(DiffArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int P = fft_phys(NZ) | 1;
  double2* col = reinterpret_cast<double2*>(smem);  // [3][P]
  double2* tw = col + 3 * P;
  const int x = blockIdx.x, y = blockIdx.y, nx = a.nx, ny = a.ny;
  fill_twiddles(tw, NZ);
  const double two_pi = 6.283185307179586476925286766559;
  const double qx = a.qix + two_pi * fft_freq(x, nx) / (nx * a.dx);
  const double qy = a.qiy + two_pi * fft_freq(y, ny) / (ny * a.dy);
  const size_t pstride = (size_t)nx * ny, cstride = (size_t)a.nz * pstride, off = (size_t)y * nx + x;
  for (int i = threadIdx.x; i < 3 * NZ; i += blockDim.x) {
    const int c = i / NZ, z = i % NZ;
    col[c * P + fpad(z)] = a.work[c * cstride + z * pstride + off];
  }
  __syncthreads();
  cta_fft<double2, NZ, false>(col, 3, P, tw);
  __syncthreads();
  const double kb2 = a.kb * a.kb;
  for (int i = threadIdx.x; i < 3 * NZ; i += blockDim.x) {
    const int c = i / NZ, l = i % NZ;
    const double kz = two_pi * fft_freq(l, NZ) / (NZ * a.dz);
    const double k2 = qx * qx + qy * qy + kz * kz;
    const double d = (k2 > kb2 ? kb2 / k2 : 1.0) / NZ;
    col[c * P + fpad(l)] = cscale(col[c * P + fpad(l)], d);
  }
  __syncthreads();
  cta_fft<double2, NZ, true>(col, 3, P, tw);
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * NZ; i += blockDim.x) {
    const int c = i / NZ, z = i % NZ;
    a.work[c * cstride + z * pstride + off] = col[c * P + fpad(z)];
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

template <int NZ>
int launch_damp(const DiffArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(3 * (fft_phys(NZ) | 1) + NZ) * sizeof(double2);
  k_damp_column<NZ><<<dim3(a.nx, a.ny), 128, smem, st>>>(a);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA;
}

bool diff_sizes_ok(int n, int nz, int n_pml, double dx, double dz, double wavelength, double eps_bg) {
  return (n == 8 || n == 16 || n == 32 || n == 64) && (nz == 32 || nz == 64 || nz == 128) && n_pml >= 0 &&
         2 * n_pml < nz && dx > 0 && dz > 0 && wavelength > 0 && eps_bg > 0;
}

DiffArgs diff_args(int n, int nz, int n_pml, double dx, double dz, double wavelength, double eps_bg,
                   double theta_deg, double phi_deg) {
  DiffArgs a{};
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
  return a;
}

// out = A E (curl curl E - k0^2 eps E), work: one field-sized intermediate.
int diff_apply(DiffArgs a, const double2* E, double2* out, double2* work, cudaStream_t st) {
  a.E = E;
  a.out = out;
  a.work = work;
  auto planes = [&](bool inv) {
    switch (a.nx) {
      case 8: return launch_plane<8>(a, inv, st);
      case 16: return launch_plane<16>(a, inv, st);
      case 32: return launch_plane<32>(a, inv, st);
      default: return launch_plane<64>(a, inv, st);
    }
  };
  int rc;
  if ((rc = planes(false)) != PSFD_OK) return rc;
  switch (a.nz) {
    case 32: rc = launch_column<32>(a, st); break;
    case 64: rc = launch_column<64>(a, st); break;
    default: rc = launch_column<128>(a, st); break;
  }
  if (rc != PSFD_OK) return rc;
  return planes(true);
}

// out = D r: the spectral damping preconditioner (FFT_xyz, D(k), inverse).
int diff_damp(DiffArgs a, const double2* r, double2* out, double2* work, cudaStream_t st) {
  a.E = r;
  a.out = out;
  a.work = work;
  a.eps = nullptr;
  auto planes = [&](bool inv) {
    switch (a.nx) {
      case 8: return launch_plane<8>(a, inv, st);
      case 16: return launch_plane<16>(a, inv, st);
      case 32: return launch_plane<32>(a, inv, st);
      default: return launch_plane<64>(a, inv, st);
    }
  };
  int rc;
  if ((rc = planes(false)) != PSFD_OK) return rc;
  switch (a.nz) {
    case 32: rc = launch_damp<32>(a, st); break;
    case 64: rc = launch_damp<64>(a, st); break;
    default: rc = launch_damp<128>(a, st); break;
  }
  if (rc != PSFD_OK) return rc;
  return planes(true);
}

// ---------------------------------------------------------------------------
// GMRES(m) for the differential system (the comparator's solve; FP64). Classical Gram-Schmidt
// with one reorthogonalisation pass on the device, Givens rotations and the small triangular
// solve on the host; the matrix is left-preconditioned by D when asked.
// ---------------------------------------------------------------------------
constexpr int kVecNT = 256, kVecBlocks = 64;

// part[i * kVecBlocks + blk] = partial of <v_i, w> (conj(v_i) w), i < nv
__global__ void __launch_bounds__(kVecNT) k_gm_dots(size_t n, const double2* V, size_t vstride, int nv,
                                                     const double2* w, double2* part) {
  __shared__ double2 sh[kVecNT / 32];
  const int i = blockIdx.y, blk = blockIdx.x;
  const double2* v = V + (size_t)i * vstride;
  double2 acc = make_double2(0.0, 0.0);
  for (size_t k = (size_t)blk * kVecNT + threadIdx.x; k < n; k += (size_t)kVecBlocks * kVecNT)
    acc = cadd(acc, cmulc(v[k], w[k]));
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < kVecNT / 32; ++k) s = cadd(s, sh[k]);
    part[(size_t)i * kVecBlocks + blk] = s;
  }
}

// h[i] = sum of the partials of i (fixed order), i < nv
__global__ void k_gm_sum(const double2* part, int nv, double2* h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < kVecBlocks; ++b) s = cadd(s, part[(size_t)i * kVecBlocks + b]);
  h[i] = s;
}

// w -= sum_i c_i v_i  (sign = -1) or  w += sum_i c_i v_i  (sign = +1)
__global__ void __launch_bounds__(kVecNT) k_gm_combine(size_t n, const double2* V, size_t vstride, int nv,
                                                        const double2* c, double sign, double2* w) {
  for (size_t k = (size_t)blockIdx.x * kVecNT + threadIdx.x; k < n; k += (size_t)gridDim.x * kVecNT) {
    double2 acc = w[k];
    for (int i = 0; i < nv; ++i) acc = cadd(acc, cscale(cmul(c[i], V[(size_t)i * vstride + k]), sign));
    w[k] = acc;
  }
}

// out = alpha (a - b)  (b may be null: out = alpha a)
__global__ void __launch_bounds__(kVecNT) k_gm_axpby(size_t n, double alpha, const double2* a, const double2* b,
                                                      double2* out) {
  for (size_t k = (size_t)blockIdx.x * kVecNT + threadIdx.x; k < n; k += (size_t)gridDim.x * kVecNT)
    out[k] = cscale(b ? csub(a[k], b[k]) : a[k], alpha);
}

struct GmDiff {
  DiffArgs a;
  int precond;
  size_t n;                 // complex elements of a field
  double2 *V, *w, *t, *u;   // basis [m + 1][n], w, the operator's intermediate, the preconditioner's input
  double2 *part, *h;        // partial sums [m + 1][kVecBlocks], coefficients [m + 2] (device)
  cudaStream_t st;
};

int gm_check() { return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA; }

// out = M A in, M = D (spectral damping) or the identity
int gm_apply(GmDiff& g, const double2* in, double2* out) {
  if (!g.precond) return diff_apply(g.a, in, out, g.t, g.st);
  int rc = diff_apply(g.a, in, g.u, g.t, g.st);
  if (rc != PSFD_OK) return rc;
  return diff_damp(g.a, g.u, out, g.t, g.st);
}

// c[0 .. nv) = <v_i, w> on the device
int gm_dots(GmDiff& g, int nv, const double2* w, double2* c) {
  k_gm_dots<<<dim3(kVecBlocks, nv), kVecNT, 0, g.st>>>(g.n, g.V, g.n, nv, w, g.part);
  k_gm_sum<<<(nv + 127) / 128, 128, 0, g.st>>>(g.part, nv, c);
  count_launch(2);
  return gm_check();
}

int gm_blocks(size_t n) { return (int)std::min<size_t>(1184, (n + kVecNT - 1) / kVecNT); }

// ||v|| (device dot, host copy; synchronises the stream)
int gm_norm(GmDiff& g, const double2* v, double* out) {
  k_gm_dots<<<dim3(kVecBlocks, 1), kVecNT, 0, g.st>>>(g.n, v, g.n, 1, v, g.part);
  k_gm_sum<<<1, 128, 0, g.st>>>(g.part, 1, g.h);
  count_launch(2);
  double2 r;
  if (gm_check() || cudaMemcpyAsync(&r, g.h, sizeof(r), cudaMemcpyDeviceToHost, g.st) != cudaSuccess ||
      cudaStreamSynchronize(g.st) != cudaSuccess)
    return PSFD_E_CUDA;
  *out = std::sqrt(std::max(r.x, 0.0));
  return PSFD_OK;
}

}  // namespace
}  // namespace psfd

extern "C" int psfd_solve_differential(int n, int nz, int n_pml, double dx, double dz, double wavelength,
                                       double eps_bg, double theta_deg, double phi_deg, int precond, const double* eps,
                                       const double* b, double* x, double* work, int restart, int max_matvecs,
                                       double rtol, int* matvecs, double* relres, void* stream) {
  using namespace psfd;
  if (!diff_sizes_ok(n, nz, n_pml, dx, dz, wavelength, eps_bg) || !eps || !b || !x || !work || restart < 1 ||
      restart > 512 || max_matvecs < 1 || !(rtol > 0) || (precond != 0 && precond != 1))
    return PSFD_E_ARG;
  GmDiff g;
  g.a = diff_args(n, nz, n_pml, dx, dz, wavelength, eps_bg, theta_deg, phi_deg);
  g.a.eps = reinterpret_cast<const double2*>(eps);
  g.precond = precond;
  g.n = (size_t)3 * nz * n * n;
  g.st = (cudaStream_t)stream;
  const int m = restart;
  double2* wk = reinterpret_cast<double2*>(work);
  g.V = wk;
  g.w = wk + (size_t)(m + 1) * g.n;
  g.t = g.w + g.n;
  g.u = g.t + g.n;
  // partial sums and coefficients at the end of the work space: (m + 1) kVecBlocks + m + 2 entries
  g.part = g.u + g.n;
  g.h = g.part + (size_t)(m + 1) * kVecBlocks;
  const double2* bd = reinterpret_cast<const double2*>(b);
  double2* xd = reinterpret_cast<double2*>(x);
  const int nb = gm_blocks(g.n);
  int rc;
  // ||M b||, x = 0
  if (cudaMemsetAsync(xd, 0, sizeof(double2) * g.n, g.st) != cudaSuccess) return PSFD_E_CUDA;
  if (precond) {
    if ((rc = diff_damp(g.a, bd, g.V, g.t, g.st)) != PSFD_OK) return rc;
  } else {
    k_gm_axpby<<<nb, kVecNT, 0, g.st>>>(g.n, 1.0, bd, nullptr, g.V);
    count_launch();
  }
  double bn = 0.0;
  if ((rc = gm_norm(g, g.V, &bn)) != PSFD_OK) return rc;
  int mv = 0;
  double res = 1.0;
  if (matvecs) *matvecs = 0;
  if (relres) *relres = 0.0;
  if (bn == 0.0) return PSFD_OK;
  std::vector<std::complex<double>> H((size_t)(m + 1) * m), cs(m), gv(m + 1), hcol(m + 2);
  std::vector<double> sn(m);
  bool first = true;
  while (mv < max_matvecs) {
    // r = M (b - A x) into V[0] (the first cycle has it already)
    if (!first) {
      if ((rc = diff_apply(g.a, xd, g.w, g.t, g.st)) != PSFD_OK) return rc;
      k_gm_axpby<<<nb, kVecNT, 0, g.st>>>(g.n, 1.0, bd, g.w, precond ? g.u : g.V);
      count_launch();
      if (precond && (rc = diff_damp(g.a, g.u, g.V, g.t, g.st)) != PSFD_OK) return rc;
    }
    first = false;
    double beta = 0.0;
    if ((rc = gm_norm(g, g.V, &beta)) != PSFD_OK) return rc;
    res = beta / bn;
    if (res <= rtol) break;
    k_gm_axpby<<<nb, kVecNT, 0, g.st>>>(g.n, 1.0 / beta, g.V, nullptr, g.V);
    count_launch();
    const int mc = std::min(m, max_matvecs - mv);
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0, cols = 0;
    for (j = 0; j < mc; ++j) {
      if ((rc = gm_apply(g, g.V + (size_t)j * g.n, g.w)) != PSFD_OK) return rc;
      ++mv;
      // two passes of classical Gram-Schmidt against v_0 .. v_j; coefficients summed on the host
      std::fill(hcol.begin(), hcol.end(), 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        if ((rc = gm_dots(g, j + 1, g.w, g.h)) != PSFD_OK) return rc;
        k_gm_combine<<<nb, kVecNT, 0, g.st>>>(g.n, g.V, g.n, j + 1, g.h, -1.0, g.w);
        count_launch();
        std::vector<double2> hv(j + 1);
        if (gm_check() || cudaMemcpyAsync(hv.data(), g.h, sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost,
                                          g.st) != cudaSuccess || cudaStreamSynchronize(g.st) != cudaSuccess)
          return PSFD_E_CUDA;
        for (int i = 0; i <= j; ++i) hcol[i] += std::complex<double>(hv[i].x, hv[i].y);
      }
      double hn = 0.0;
      if ((rc = gm_norm(g, g.w, &hn)) != PSFD_OK) return rc;
      if (hn > 0.0) {
        k_gm_axpby<<<nb, kVecNT, 0, g.st>>>(g.n, 1.0 / hn, g.w, nullptr, g.V + (size_t)(j + 1) * g.n);
        count_launch();
      }
      // earlier rotations G_i = [[conj(c), s], [-s, c]] (s real), then the new one
      for (int i = 0; i < j; ++i) {
        const std::complex<double> t = std::conj(cs[i]) * hcol[i] + sn[i] * hcol[i + 1];
        hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = t;
      }
      const double den = std::hypot(std::abs(hcol[j]), hn);
      cs[j] = den > 0.0 ? hcol[j] / den : 1.0;
      sn[j] = den > 0.0 ? hn / den : 0.0;
      hcol[j] = den;
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = std::conj(cs[j]) * gv[j];
      res = std::abs(gv[j + 1]) / bn;
      cols = j + 1;
      if (res <= rtol || hn == 0.0) break;
    }
    // x += V y with the upper triangular H y = g
    std::vector<std::complex<double>> y(cols);
    for (int i = cols - 1; i >= 0; --i) {
      std::complex<double> acc = gv[i];
      for (int k = i + 1; k < cols; ++k) acc -= H[(size_t)i * m + k] * y[k];
      y[i] = acc / H[(size_t)i * m + i];
    }
    std::vector<double2> yd(cols);
    for (int i = 0; i < cols; ++i) yd[i] = make_double2(y[i].real(), y[i].imag());
    if (cudaMemcpyAsync(g.h, yd.data(), sizeof(double2) * cols, cudaMemcpyHostToDevice, g.st) != cudaSuccess)
      return PSFD_E_CUDA;
    k_gm_combine<<<nb, kVecNT, 0, g.st>>>(g.n, g.V, g.n, cols, g.h, 1.0, xd);
    count_launch();
    if (gm_check() || cudaStreamSynchronize(g.st) != cudaSuccess) return PSFD_E_CUDA;
    if (res <= rtol) break;
  }
  if (matvecs) *matvecs = mv;
  if (relres) *relres = res;
  return res <= rtol ? PSFD_OK : PSFD_E_NOT_CONVERGED;
}

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

extern "C" size_t psfd_solve_differential_work(int n, int nz, int restart) {
  if (n < 1 || nz < 1 || restart < 1) return 0;
  const size_t field = (size_t)3 * nz * n * n;
  return (size_t)(restart + 4) * field + (size_t)(restart + 1) * psfd::kVecBlocks + (size_t)restart + 2;
}
