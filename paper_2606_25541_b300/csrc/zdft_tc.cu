// zdft_tc.cu -- the forward z transform of the operator's z pass (K2 at nf = 128: the
// nslab absorber planes of a column, zero padded, transformed along z; Sec. 3, Eq. (18)) as
// dense DFT products on the tensor cores, and the same stage on the CUDA cores, for
// measuring one against the other.
//
// Tensor cores (method 1): X[l] = sum_{n=1..64} x[n] w^{n l}, w = exp(-2 pi i / 128), for a
// tile of 128 complex columns at once. With the columns' real and imaginary parts as the
// 256 columns of B (K = 64 rows: the planes) and the real DFT matrices Ar = cos, Ai = -sin
// (M = 128 rows: the bins l),
//     P1 = Ar B,  P2 = Ai B,  Re X = P1[2c] - P2[2c + 1],  Im X = P2[2c] + P1[2c + 1].
// Every operand is split into BF16 hi + lo (hi = RN(v), lo = RN(v - hi)) and each product
// is A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo x lo term is below the format), accumulated
// in FP32 in tensor memory: tcgen05.mma kind::f16, M = 128, N = 256, K = 16 per instruction,
// both operands K-major in shared memory with the 128-byte swizzle. The DFT matrices are
// built once (FP64 sincospi) as the exact shared-memory image and copied into each CTA by
// one bulk asynchronous copy; the data tile is converted by the CTA's threads.
// CUDA cores (method 0): the register four-step transform of K2 (16 x 8, eight lanes per
// column, one shared-memory exchange).
//
// Both write the full 128-bin spectrum: out[set][l][y][x] from in[set][p][y][x], plane p
// at z index p + 1 (plane 0 and planes above nslab are zero).
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/psfd.h"
#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

#include <cuda_bf16.h>

namespace psfd {
namespace {

constexpr int kNf = 128;         // bins (M of the products)
constexpr int kK = 64;           // planes (K of the products; nslab <= 63)
constexpr int kCols = 128;       // complex columns per CTA
constexpr int kN = 2 * kCols;    // real columns per CTA (N of the products)
constexpr int kTcThreads = 256;
constexpr int kTileA = kNf * kK * 2;      // bytes of one BF16 DFT matrix (16 KB)
constexpr int kTileB = kN * kK * 2;       // bytes of one BF16 data tile (32 KB)
constexpr int kImage = 4 * kTileA;        // Ar hi, Ar lo, Ai hi, Ai lo
constexpr size_t kTcSmem = (size_t)kImage + 2 * kTileB + 1024 + 64;
constexpr unsigned kWaitLimit = 1u << 24;  // bounded waits: try_wait polls before giving up

// Byte offset of element (row r, k) in a K-major tile of 64 BF16 values per row with the
// 128-byte swizzle: the 16-byte chunk index is XORed with the row's position in its 8-row
// group (the tile base must be 1024-byte aligned).
__host__ __device__ __forceinline__ uint32_t sw128(int r, int k) {
  const uint32_t b = 2u * (uint32_t)k;
  return (uint32_t)r * 128u + ((((b >> 4) ^ (uint32_t)(r & 7)) & 7u) << 4) + (b & 15u);
}

// DFT matrices as the shared-memory image: [Ar hi | Ar lo | Ai hi | Ai lo], entry (l, k) =
// exp(-2 pi i (k + 1) l / 128) split into BF16 hi + lo.
__global__ void k_dft_image(unsigned char* img) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNf * kK; i += gridDim.x * blockDim.x) {
    const int l = i / kK, k = i % kK;
    double s, c;
    sincospi(-2.0 * (double)(((k + 1) * l) % kNf) / (double)kNf, &s, &c);
    const float cr = (float)c, ci = (float)s;
    const __nv_bfloat16 rh = __float2bfloat16_rn(cr), ih = __float2bfloat16_rn(ci);
    const __nv_bfloat16 rl = __float2bfloat16_rn(cr - __bfloat162float(rh));
    const __nv_bfloat16 il = __float2bfloat16_rn(ci - __bfloat162float(ih));
    const uint32_t o = sw128(l, k);
    *reinterpret_cast<__nv_bfloat16*>(img + 0 * kTileA + o) = rh;
    *reinterpret_cast<__nv_bfloat16*>(img + 1 * kTileA + o) = rl;
    *reinterpret_cast<__nv_bfloat16*>(img + 2 * kTileA + o) = ih;
    *reinterpret_cast<__nv_bfloat16*>(img + 3 * kTileA + o) = il;
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride between 8-row groups
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// grid (nx / 128, ny, sets); 256 threads; one tile of 128 complex columns (x0 .. x0 + 127)
__global__ void __launch_bounds__(kTcThreads, 1)
    k_zdft_tc(const float2* __restrict__ in, float2* __restrict__ out, const unsigned char* __restrict__ img,
              int nx, int ny, int nslab, int* err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* A = base;                  // the image: Ar hi, Ar lo, Ai hi, Ai lo
  unsigned char* Bh = base + kImage;        // data hi
  unsigned char* Bl = Bh + kTileB;          // data lo
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bl + kTileB);  // [0]: image copied, [1]: products done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * kCols, y = blockIdx.y, set = blockIdx.z;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar[0])), "r"(kImage)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(A)),
                 "l"(img), "r"(kImage), "r"(smem_u32(&bar[0]))
                 : "memory");
  }
  // the data tile: real column 2c (Re) and 2c + 1 (Im) of complex column c, K-major
  const size_t pstride = (size_t)ny * nx;
  const float2* src = in + (size_t)set * nslab * pstride + (size_t)y * nx + x0;
  for (int i = tid; i < kCols * kK; i += kTcThreads) {
    const int c = i % kCols, k = i / kCols;
    const float2 v = k < nslab ? src[(size_t)k * pstride + c] : make_float2(0.f, 0.f);
    const __nv_bfloat16 rh = __float2bfloat16_rn(v.x), ih = __float2bfloat16_rn(v.y);
    const __nv_bfloat16 rl = __float2bfloat16_rn(v.x - __bfloat162float(rh));
    const __nv_bfloat16 il = __float2bfloat16_rn(v.y - __bfloat162float(ih));
    *reinterpret_cast<__nv_bfloat16*>(Bh + sw128(2 * c, k)) = rh;
    *reinterpret_cast<__nv_bfloat16*>(Bh + sw128(2 * c + 1, k)) = ih;
    *reinterpret_cast<__nv_bfloat16*>(Bl + sw128(2 * c, k)) = rl;
    *reinterpret_cast<__nv_bfloat16*>(Bl + sw128(2 * c + 1, k)) = il;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the tile is read by the tensor cores
  __syncthreads();

  bool ok = true;
  if (tid == 0) {
    ok = mbar_wait(smem_u32(&bar[0]), 0);
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      constexpr uint32_t id = idesc_bf16(kNf, kN);
      const uint32_t a = smem_u32(A), bh = smem_u32(Bh), bl = smem_u32(Bl);
      // P1 = Ar B (TMEM columns 0 .. 255), P2 = Ai B (256 .. 511); three split products each
      for (int part = 0; part < 2; ++part) {
        const uint32_t ah = a + (2 * part) * kTileA, al = ah + kTileA;
        const uint32_t d = tmem + part * kN;
        int acc = 0;
        const uint32_t pa[3] = {ah, ah, al}, pb[3] = {bh, bl, bh};
        for (int t = 0; t < 3; ++t)
          for (int ks = 0; ks < kK / 16; ++ks) {
            mma_bf16(d, sdesc(pa[t] + 32 * ks), sdesc(pb[t] + 32 * ks), id, acc);
            acc = 1;
          }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar[1]))
                   : "memory");
    } else {
      atomicExch(err, 1);
    }
  }
  __syncthreads();
  if (__syncthreads_or(!ok)) {  // the image never arrived: wait (bounded) for the copy, then leave
    if (tid == 0) mbar_wait(smem_u32(&bar[0]), 0);
  } else {
    // uniform across the CTA: the tensor-memory loads below are warp-synchronous
    const bool done = __syncthreads_and(mbar_wait(smem_u32(&bar[1]), 0));
    if (!done && tid == 0) atomicExch(err, 2);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (done) {
      // warp w reads TMEM lanes 32 (w % 4) .. (the bins) for the complex columns of half w / 4
      const int lg = warp & 3, half = warp >> 2, l = 32 * lg + lane;
      float2* dst = out + ((size_t)set * kNf + l) * pstride + (size_t)y * nx + x0;
      for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 8) {
        uint32_t p1[16], p2[16];
        const uint32_t ta = tmem + ((uint32_t)(32 * lg) << 16) + 2 * c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(p1[0]), "=r"(p1[1]), "=r"(p1[2]), "=r"(p1[3]), "=r"(p1[4]), "=r"(p1[5]), "=r"(p1[6]),
              "=r"(p1[7]), "=r"(p1[8]), "=r"(p1[9]), "=r"(p1[10]), "=r"(p1[11]), "=r"(p1[12]), "=r"(p1[13]),
              "=r"(p1[14]), "=r"(p1[15])
            : "r"(ta));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(p2[0]), "=r"(p2[1]), "=r"(p2[2]), "=r"(p2[3]), "=r"(p2[4]), "=r"(p2[5]), "=r"(p2[6]),
              "=r"(p2[7]), "=r"(p2[8]), "=r"(p2[9]), "=r"(p2[10]), "=r"(p2[11]), "=r"(p2[12]), "=r"(p2[13]),
              "=r"(p2[14]), "=r"(p2[15])
            : "r"(ta + kN));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float re = __uint_as_float(p1[2 * j]) - __uint_as_float(p2[2 * j + 1]);
          const float im = __uint_as_float(p2[2 * j]) + __uint_as_float(p1[2 * j + 1]);
          dst[c0 + j] = make_float2(re, im);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// CUDA cores: eight lanes per column, the register four-step transform of K2 (16 x 8).
constexpr int kFftCols = 32;  // columns per CTA (256 threads)
__global__ void __launch_bounds__(256) k_zdft_fft(const float2* __restrict__ in, float2* __restrict__ out,
                                                   const double2* __restrict__ twz, int nx, int ny, int nslab) {
  constexpr int N2 = kNf / 16, EP = N2 + 1;
  __shared__ float2 tw[kNf];
  __shared__ float2 ex[kFftCols][16 * EP];
  for (int i = threadIdx.x; i < kNf; i += blockDim.x) tw[i] = make_float2((float)twz[i].x, (float)twz[i].y);
  __syncthreads();
  const int g = threadIdx.x / N2, j = threadIdx.x % N2;
  const int x = blockIdx.x * kFftCols + g, y = blockIdx.y, set = blockIdx.z;
  const size_t pstride = (size_t)ny * nx;
  const float2* src = in + (size_t)set * nslab * pstride + (size_t)y * nx + x;
  float2 v[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int n = j + N2 * k;
    v[k] = (n >= 1 && n <= nslab) ? src[(size_t)(n - 1) * pstride] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int k = 8; k < 16; ++k) v[k] = make_float2(0.f, 0.f);
  reg_fft_step1<float2, kNf, false, true>(v, j, tw);
  float2* e = ex[g];
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) e[k1 * EP + j] = v[k1];
  __syncwarp();
  float2 o[16];
  reg_fft_step2<float2, kNf, false, EP>(e, j, o);
  float2* dst = out + (size_t)set * kNf * pstride + (size_t)y * nx + x;
#pragma unroll
  for (int r = 0; r < 16 / N2; ++r)
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) dst[(size_t)(j + N2 * r + 16 * k2) * pstride] = o[r * N2 + k2];
}

std::mutex g_mu;
unsigned char* g_img[64] = {};
double2* g_tw[64] = {};
int* g_err[64] = {};

int prepare(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_img[dev]) return PSFD_OK;
  unsigned char* img = nullptr;
  double2* tw = nullptr;
  int* err = nullptr;
  if (cudaMalloc(&img, kImage) != cudaSuccess || cudaMalloc(&tw, sizeof(double2) * kNf) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess)
    return PSFD_E_NOMEM;
  double2 h[kNf];
  for (int i = 0; i < kNf; ++i) {
    const double a = -2.0 * 3.14159265358979323846 * i / kNf;
    h[i] = make_double2(std::cos(a), std::sin(a));
  }
  if (cudaMemset(img, 0, kImage) != cudaSuccess ||
      cudaMemcpy(tw, h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(err, 0, sizeof(int)) != cudaSuccess)
    return PSFD_E_CUDA;
  k_dft_image<<<32, 256>>>(img);
  count_launch();
  if (cudaDeviceSynchronize() != cudaSuccess) return PSFD_E_CUDA;
  g_img[dev] = img;
  g_tw[dev] = tw;
  g_err[dev] = err;
  return PSFD_OK;
}

}  // namespace
}  // namespace psfd

using namespace psfd;

extern "C" int psfd_zdft_measure(int method, int nx, int ny, int nsets, int nslab, const void* in, void* out,
                                 void* stream) {
  if (!in || !out || nsets < 1 || ny < 1 || nslab < 1 || nslab >= kK) return PSFD_E_ARG;
  if (method == 1 ? nx % kCols != 0 : (method == 0 ? nx % kFftCols != 0 : true)) return PSFD_E_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PSFD_E_CUDA;
  int rc = prepare(dev);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (method == 1) {
    if (cudaFuncSetAttribute(k_zdft_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem) != cudaSuccess)
      return PSFD_E_CUDA;
    k_zdft_tc<<<dim3(nx / kCols, ny, nsets), kTcThreads, kTcSmem, st>>>(
        static_cast<const float2*>(in), static_cast<float2*>(out), g_img[dev], nx, ny, nslab, g_err[dev]);
  } else {
    k_zdft_fft<<<dim3(nx / kFftCols, ny, nsets), 256, 0, st>>>(static_cast<const float2*>(in),
                                                               static_cast<float2*>(out), g_tw[dev], nx, ny, nslab);
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? PSFD_OK : PSFD_E_CUDA;
}

extern "C" int psfd_zdft_status(int* flag) {
  if (!flag) return PSFD_E_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PSFD_E_CUDA;
  if (!g_err[dev]) {
    *flag = 0;
    return PSFD_OK;
  }
  if (cudaMemcpy(flag, g_err[dev], sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PSFD_E_CUDA;
  return PSFD_OK;
}
