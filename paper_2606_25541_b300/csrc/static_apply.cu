// static_apply.cu -- psfd_apply_fp32_static: one FP32 operator application that
// allocates no memory.
//
// Some callers cannot call cudaMalloc: deployments whose device memory is fixed when
// the process starts (real-time or certified systems that forbid allocation after
// initialisation), and hosts whose own allocator owns the whole device, where a stray
// cudaMalloc/cudaFree would break its accounting or force a device-wide
// synchronisation. They cannot create a psfd context either, since psfd_create
// allocates. This entry point needs no context: the caller passes the grid, the stack,
// one illumination, the permittivity, the input field and the output buffer, and every
// intermediate (twiddle tables, stack tables, FP32 potential, spectral work buffer)
// lives in one statically sized device array that the library owns for the life of
// the process.
//
// It runs the same kernels as psfd_apply with precision PSFD_FP32_REFINED.
#include <cmath>
#include <mutex>

#include "../../include/psfd.h"
#include "common.cuh"
#include "internal.h"
#include "tables.h"

using namespace psfd;

namespace {

// The shared scratch. Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[PSFD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr int kMaxLayers = 256;
std::mutex g_mu;
void* g_base[kMaxDevices] = {};

// Host-side address of g_static_scratch on the current device, looked up once per device.
int scratch_base(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PSFD_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return PSFD_E_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return PSFD_E_CUDA;
    g_base[dev] = p;
  }
  *out = g_base[dev];
  return PSFD_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void k_static_twiddles(double2* tw, float2* tw32, int n) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)t / (double)n, &s, &c);
    tw[t] = make_double2(c, s);
    tw32[t] = make_float2((float)c, (float)s);
  }
}

__global__ void k_static_params(RhsParam* rp, double* sq, double qix, double qiy, double cphi, double sphi) {
  RhsParam p = {};
  p.qix = qix;
  p.qiy = qiy;
  p.cphi = cphi;
  p.sphi = sphi;
  p.slot = 0;
  p.pol = 0;
  *rp = p;
  sq[0] = qix;
  sq[1] = qiy;
  sq[2] = cphi;
  sq[3] = sphi;
}

// kz_l = 2 pi l / (nf dz): FP32 |kz| hi / lo and signed kz, FP64 signed kz.
__global__ void k_static_ktab(float* k32, double* k64, int nf, double dz) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nf; l += gridDim.x * blockDim.x) {
    const int lf = fft_freq(l, nf);
    const double k = 6.283185307179586476925286766559 * (double)lf / ((double)nf * dz);
    k64[l] = k;
    const float hi = (float)fabs(k);
    k32[l] = hi;
    k32[nf + l] = (float)(fabs(k) - (double)hi);
    k32[2 * nf + l] = (float)k;
  }
}

// V = k0^2 (eps - eps_bg) formed in FP64 and rounded to FP32 (as psfd_set_potential does).
__global__ void k_static_potential(size_t n, const double2* eps, double k02, double eps_bg, float2* V32) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 e = eps[i];
    V32[i] = make_float2((float)(k02 * (e.x - eps_bg)), (float)(k02 * e.y));
  }
}

}  // namespace

extern "C" int psfd_apply_fp32_static(const psfd_grid* g, int n_layers, const double* n_complex,
                                      const double* thickness_nm, const double* n_sub, double theta_deg,
                                      double phi_deg, const void* eps, const void* u, void* out, void* stream) {
  constexpr double kPi = 3.14159265358979323846264338327950288;
  if (!g || !eps || !u || !out || !n_sub || n_layers < 0 || n_layers > kMaxLayers ||
      (n_layers > 0 && (!n_complex || !thickness_nm)))
    return PSFD_E_ARG;
  if (!fft_length_supported(g->nx) || !fft_length_supported(g->ny) || !fft_length_supported(g->nf) ||
      g->nslab < 1 || g->nf < 2 * g->nslab + 2 || !(g->dx > 0 && g->dy > 0 && g->dz > 0) ||
      !(g->wavelength > 0 && g->eps_bg > 0) || !std::isfinite(theta_deg) || !std::isfinite(phi_deg))
    return PSFD_E_ARG;
  const size_t plane = (size_t)g->nx * g->ny;
  const size_t U = 3 * (size_t)g->nslab * plane;

  // scratch layout, every block 256-byte aligned
  size_t off = 0;
  const size_t o_twx = off; off = align256(off + g->nx * sizeof(double2));
  const size_t o_twy = off; off = align256(off + g->ny * sizeof(double2));
  const size_t o_twz = off; off = align256(off + g->nf * sizeof(double2));
  const size_t o_twx32 = off; off = align256(off + g->nx * sizeof(float2));
  const size_t o_twy32 = off; off = align256(off + g->ny * sizeof(float2));
  const size_t o_twz32 = off; off = align256(off + g->nf * sizeof(float2));
  const size_t o_rhs = off; off = align256(off + sizeof(RhsParam));
  const size_t o_sq = off; off = align256(off + 4 * sizeof(double));
  const size_t o_k32 = off; off = align256(off + 3 * (size_t)g->nf * sizeof(float));
  const size_t o_k64 = off; off = align256(off + (size_t)g->nf * sizeof(double));
  const size_t o_m32 = off; off = align256(off + plane * sizeof(ModeF32));
  const size_t o_epsl = off; off = align256(off + kMaxLayers * sizeof(double2));
  const size_t o_dl = off; off = align256(off + kMaxLayers * sizeof(double));
  const size_t o_anom = off; off = align256(off + sizeof(int));
  const size_t o_modes = off; off = align256(off + plane * sizeof(ModeEntry));
  const size_t o_V = off; off = align256(off + (size_t)g->nslab * plane * sizeof(float2));
  const size_t o_work = off; off = align256(off + U * sizeof(float2));
  if (off > (size_t)PSFD_STATIC_SCRATCH_BYTES) return PSFD_E_BUDGET;

  const double k0 = 2.0 * kPi / g->wavelength;
  const double kb = k0 * std::sqrt(g->eps_bg);
  const double th = theta_deg * kPi / 180.0, ph = phi_deg * kPi / 180.0;
  const double qix = kb * std::sin(th) * std::cos(ph), qiy = kb * std::sin(th) * std::sin(ph);
  // Rayleigh anomaly check, on the host, before any device work
  for (int y = 0; y < g->ny; ++y) {
    const double qy = qiy + 2.0 * kPi * fft_freq(y, g->ny) / (g->ny * g->dy);
    for (int x = 0; x < g->nx; ++x) {
      const double qx = qix + 2.0 * kPi * fft_freq(x, g->nx) / (g->nx * g->dx);
      if (std::sqrt(std::fabs(kb * kb - qx * qx - qy * qy)) < 1e-9 * k0) return PSFD_E_ANOMALY;
    }
  }

  void* basev = nullptr;
  int rc = scratch_base(&basev);
  if (rc) return rc;
  unsigned char* base = static_cast<unsigned char*>(basev);
  cudaStream_t st = (cudaStream_t)stream;

  // stack permittivities and thicknesses, staged in fixed-size host arrays
  double2 eps_l[kMaxLayers];
  double d_l[kMaxLayers];
  for (int j = 0; j < n_layers; ++j) {
    const double a = n_complex[2 * j], b = n_complex[2 * j + 1];
    if (!(thickness_nm[j] >= 0.0)) return PSFD_E_ARG;
    eps_l[j] = make_double2(a * a - b * b, 2.0 * a * b);
    d_l[j] = thickness_nm[j];
  }
  // A stack of few distinct media, interfaces and layers (the periodic EUV stacks) is carried
  // by value in the kernel arguments; only one that does not deduplicate goes through the
  // scratch, copied from the stack arrays above and synchronised before they go out of scope.
  StackDev stack = {};
  stack.n_layers = n_layers;
  stack.reflect = 1;
  stack.eps = reinterpret_cast<const double2*>(base + o_epsl);
  stack.d = reinterpret_cast<const double*>(base + o_dl);
  stack.eps_sub = make_double2(n_sub[0] * n_sub[0] - n_sub[1] * n_sub[1], 2.0 * n_sub[0] * n_sub[1]);
  stack_dedup(stack, eps_l, d_l, n_layers, make_double2(g->eps_bg, 0.0), stack.eps_sub);
  if (n_layers > 0 && stack.n_mat == 0) {
    if (cudaMemcpyAsync(base + o_epsl, eps_l, sizeof(double2) * n_layers, cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(base + o_dl, d_l, sizeof(double) * n_layers, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return PSFD_E_CUDA;
  }
  // the anomaly flag is accumulated with atomicOr and must start at zero
  if (cudaMemsetAsync(base + o_anom, 0, sizeof(int), st) != cudaSuccess) return PSFD_E_CUDA;

  double2* twx = reinterpret_cast<double2*>(base + o_twx);
  double2* twy = reinterpret_cast<double2*>(base + o_twy);
  double2* twz = reinterpret_cast<double2*>(base + o_twz);
  float2* twx32 = reinterpret_cast<float2*>(base + o_twx32);
  float2* twy32 = reinterpret_cast<float2*>(base + o_twy32);
  float2* twz32 = reinterpret_cast<float2*>(base + o_twz32);
  k_static_twiddles<<<4, 256, 0, st>>>(twx, twx32, g->nx);
  k_static_twiddles<<<4, 256, 0, st>>>(twy, twy32, g->ny);
  k_static_twiddles<<<4, 256, 0, st>>>(twz, twz32, g->nf);
  RhsParam* rhsp = reinterpret_cast<RhsParam*>(base + o_rhs);
  double* sq = reinterpret_cast<double*>(base + o_sq);
  k_static_params<<<1, 1, 0, st>>>(rhsp, sq, qix, qiy, std::cos(ph), std::sin(ph));
  float* k32 = reinterpret_cast<float*>(base + o_k32);
  double* k64 = reinterpret_cast<double*>(base + o_k64);
  k_static_ktab<<<1, 256, 0, st>>>(k32, k64, g->nf, g->dz);
  float2* V32 = reinterpret_cast<float2*>(base + o_V);
  k_static_potential<<<592, 256, 0, st>>>((size_t)g->nslab * plane, static_cast<const double2*>(eps), k0 * k0,
                                          g->eps_bg, V32);
  count_launch(6);
  if (cudaGetLastError() != cudaSuccess) return PSFD_E_CUDA;

  ModeEntry* modes = reinterpret_cast<ModeEntry*>(base + o_modes);
  ModesArgs m;
  m.slot0 = 0;
  m.slots = nullptr;
  m.nx = g->nx;
  m.ny = g->ny;
  m.dx = g->dx;
  m.dy = g->dy;
  m.k0 = k0;
  m.eps_bg = g->eps_bg;
  m.L = 0.5 * g->nf * g->dz;
  m.dz = g->dz;
  m.kb = kb;
  m.slot_par = sq;
  m.stack = stack;
  m.modes = modes;
  m.modes32 = reinterpret_cast<ModeF32*>(base + o_m32);
  m.modesdf = nullptr;
  m.anomaly = reinterpret_cast<int*>(base + o_anom);
  if ((rc = launch_modes(m, 1, st))) return rc;

  OpCall<float2> a = {};
  a.nx = g->nx;
  a.ny = g->ny;
  a.nslab = g->nslab;
  a.nf = g->nf;
  a.rhs0 = 0;
  a.nrhs = 1;
  a.dx = g->dx;
  a.dy = g->dy;
  a.dz = g->dz;
  a.kb = kb;
  a.dz32 = (float)g->dz;
  a.kb32 = (float)kb;
  a.V = V32;
  a.twx = twx;
  a.twy = twy;
  a.twz = twz;
  a.twx32 = twx32;
  a.twy32 = twy32;
  a.twz32 = twz32;
  a.rhsp = rhsp;
  a.modes = modes;
  a.modes32 = m.modes32;
  a.ktab32 = k32;
  a.ktab64 = k64;
  a.active = nullptr;
  a.in_mode = IN_PLAIN;
  a.u = static_cast<const float2*>(u);
  a.work = reinterpret_cast<float2*>(base + o_work);
  a.epi = EPI_AU;
  a.out = static_cast<float2*>(out);
  a.dot_mask = 0;
  a.partials = nullptr;
  a.maxblk = 0;
  a.side = nullptr;
  a.stream = st;
  rc = op_apply<float2>(a);
  return rc < 0 ? rc : PSFD_OK;
}
