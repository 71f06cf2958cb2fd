// op_launch.cuh -- host dispatch of the operator kernels (included once per precision).
#pragma once

#include <cmath>

#include "op_kernels.cuh"
#include "../../include/psfd.h"

namespace psfd {

// FFT lengths the kernels are instantiated for.
#define PSFD_FOR_EACH_LENGTH(X) \
  X(4) X(8) X(16) X(32) X(64) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512) X(640) X(768) X(1024)

template <typename C> struct Tune;
template <> struct Tune<float2> {
  static constexpr int FUSED_MAX = 128;   // largest square plane transformed in shared memory
  static constexpr int HALF_MIN = 128;    // from this size on, two CTAs per plane (half planes)
  static constexpr int COL_TILE = 16;     // columns per CTA (128-byte segments)
  static constexpr int ROW_ELEMS = 4096;  // row-pass tile size in elements
  static constexpr size_t COLS_SMEM = 64 * 1024;  // column-pass tile bound (long columns: fewer per CTA)
  static constexpr int ZCOL_TILE = 8;             // x-modes per z-column CTA (4 warps: 7 CTAs per SM)
  static constexpr int ZCOL_NT = 128;
  static constexpr size_t ZCOL_SMEM = 80 * 1024;  // z-column tile bound
  static constexpr size_t ZCOL_SMEM_REG = 80 * 1024;  // the same for the register z transform
};
template <> struct Tune<double2> {
  static constexpr int FUSED_MAX = 64;
  static constexpr int HALF_MIN = 1 << 20;  // FP64 planes are FP64-pipe bound: no split
  static constexpr int COL_TILE = 8;
  static constexpr int ROW_ELEMS = 2048;
  static constexpr size_t COLS_SMEM = 64 * 1024;
  static constexpr int ZCOL_TILE = 8;
  static constexpr int ZCOL_NT = 256;
  static constexpr size_t ZCOL_SMEM = 80 * 1024;
  // register z transform (lengths 64, 128, 256): eight x-modes per CTA even at length 256,
  // one CTA per SM there (FP64-pipe bound, so twelve warps keep the pipe busy)
  static constexpr size_t ZCOL_SMEM_REG = 120 * 1024;
};

template <typename C>
inline bool use_fused(int nx, int ny) {
  return nx == ny && nx <= Tune<C>::FUSED_MAX && (nx & (nx - 1)) == 0 && nx >= 4;
}

template <typename C>
inline bool use_half(int nx, int ny) {
  return use_fused<C>(nx, ny) && nx >= Tune<C>::HALF_MIN;
}

inline int row_block(int nx, int ny, int max_elems) {
  int rb = 1;
  while (rb * 2 * nx <= max_elems && ny % (rb * 2) == 0) rb *= 2;
  return rb;
}

template <typename C>
inline int blocks_per_rhs_t(int nx, int ny, int nslab) {
  if (use_fused<C>(nx, ny)) return (use_half<C>(nx, ny) ? 6 : 3) * nslab;
  return 3 * nslab * (ny / row_block(nx, ny, Tune<C>::ROW_ELEMS));
}

#define PSFD_CHECK_LAUNCH()                                    \
  do {                                                         \
    count_launch();                                            \
    if (cudaGetLastError() != cudaSuccess) return PSFD_E_CUDA; \
  } while (0)

template <typename K>
inline int set_smem(K kernel, size_t bytes, bool max_carveout = false) {
  if (bytes > 48 * 1024) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
      return PSFD_E_CUDA;
  }
  // kernels compiled for several CTAs per SM: shared memory for all of them
  if (max_carveout && cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
    return PSFD_E_CUDA;
  return PSFD_OK;
}

// ---------------------------------------------------------------------------
template <typename C, int N, int IN>
int launch_plane_fwd(const OpCall<C>& a) {
  constexpr int NT = N >= 128 ? 512 : 256;
  const size_t smem = (size_t)(plane_tile_elems<N, N>() + 2 * N) * sizeof(C);
  auto k = k_plane_fwd<C, N, N, IN, NT>;
  if (set_smem(k, smem)) return PSFD_E_CUDA;
  k<<<dim3(a.nslab, 3, a.nrhs), NT, smem, a.stream>>>(a);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <typename C, int N, int EPI>
int launch_plane_inv(const OpCall<C>& a, const C* uin) {
  constexpr int NT = N >= 128 ? 512 : 256;
  const size_t smem = (size_t)(plane_tile_elems<N, N>() + 2 * N) * sizeof(C) + 16 + NDOT * 32 * sizeof(double2);
  auto k = k_plane_inv<C, N, N, EPI, NT>;
  if (set_smem(k, smem)) return PSFD_E_CUDA;
  k<<<dim3(a.nslab, 3, a.nrhs), NT, smem, a.stream>>>(a, uin);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

// L2 prefetch distance of the half-plane kernels: the tuned one, or none.
template <typename C>
inline int half_pf_of(const OpCall<C>& a) {
  const int t = run_tune(sizeof(C) == 16, a.nx, a.ny, a.nslab, a.nf).pf;
  return t > 0 ? t : 0;
}

template <typename C, int N, int IN>
int launch_half_fwd(const OpCall<C>& a0) {
  constexpr int NT = 512;
  const size_t smem = (size_t)(half_tile_elems<C, N, N>() + 2 * N) * sizeof(C);
  auto k = k_half_fwd<C, N, N, IN, NT>;
  if (set_smem(k, smem)) return PSFD_E_CUDA;
  OpCall<C> a = a0;
  a.pf = half_pf_of(a0);
  k<<<dim3(2 * a.nslab, 3, a.nrhs), NT, smem, a.stream>>>(a);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <typename C, int N, int EPI>
int launch_half_inv(const OpCall<C>& a0, const C* uin) {
  constexpr int NT = 512;
  const size_t smem = (size_t)(half_tile_elems<C, N, N>() + 2 * N) * sizeof(C) + 16 + NDOT * 32 * sizeof(double2);
  auto k = k_half_inv<C, N, N, EPI, NT>;
  if (set_smem(k, smem)) return PSFD_E_CUDA;
  OpCall<C> a = a0;
  a.pf = half_pf_of(a0);
  k<<<dim3(2 * a.nslab, 3, a.nrhs), NT, smem, a.stream>>>(a, uin);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <typename C, int NX, int IN>
int launch_rows_fwd(const OpCall<C>& a) {
  constexpr int NT = 256;
  const int rb = rows_fwd_rb_of(a);
  const size_t smem = (size_t)(rb * fft_phys(NX) + NX) * sizeof(C);
  auto k = k_rows_fwd<C, NX, IN, NT>;
  if (set_smem(k, smem, split_min_blocks<C, NX>() > 1)) return PSFD_E_CUDA;
  k<<<dim3(3 * a.nrhs, a.ny / rb, a.nslab), NT, smem, a.stream>>>(a, rb);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <typename C, int NX, int EPI>
int launch_rows_inv(const OpCall<C>& a, const C* uin) {
  constexpr int NT = 256;
  const int rb = row_block(NX, a.ny, Tune<C>::ROW_ELEMS);
  const size_t smem = (size_t)(rb * fft_phys(NX) + NX) * sizeof(C) + 16 + NDOT * 32 * sizeof(double2);
  auto k = k_rows_inv<C, NX, EPI, NT>;
  if (set_smem(k, smem, split_min_blocks<C, NX>() > 1)) return PSFD_E_CUDA;
  k<<<dim3(a.nslab * (a.ny / rb), 3, a.nrhs), NT, smem, a.stream>>>(a, uin, rb);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

// Columns per CTA of the column pass: COL_TILE, halved while the tile exceeds COLS_SMEM.
template <typename C>
inline size_t cols_smem_bytes(int ny, int tx) {
  return (size_t)(tx * cols_pitch<C>(ny, tx) + ny) * sizeof(C);
}
template <typename C>
inline int cols_tile(int nx, int ny) {
  int tx = nx < Tune<C>::COL_TILE ? nx : Tune<C>::COL_TILE;
  while (tx > 1 && cols_smem_bytes<C>(ny, tx) > Tune<C>::COLS_SMEM) tx >>= 1;
  return tx;
}

// Columns per CTA of the z pass: ZCOL_TILE, halved while the tile exceeds ZCOL_SMEM.
template <typename C>
inline size_t zcol_smem_bytes(int nf, int tx) {
  using R = typename RealOf<C>::T;
  const int pe = (8 + (nf + 15) / 16) | 1;  // phase_pitch
  const bool f32reg = sizeof(C) == sizeof(float2) && (nf == 64 || nf == 128 || nf == 256);  // zcol_reg
  return (size_t)(3 * tx * zcol_pitch(nf, f32reg) + nf) * sizeof(C) + 3 * (size_t)nf * sizeof(R) +
         (size_t)(11 + pe) * tx * sizeof(C) + 5 * (size_t)tx * sizeof(R) + (size_t)tx * sizeof(int) + 16;
}
template <typename C>
inline int zcol_tile(int nx, int nf) {
  int tx = nx < Tune<C>::ZCOL_TILE ? nx : Tune<C>::ZCOL_TILE;
  const bool reg = nf == 64 || nf == 128 || nf == 256;  // zcol_reg
  const size_t bound = reg ? Tune<C>::ZCOL_SMEM_REG : Tune<C>::ZCOL_SMEM;
  while (tx > 1 && zcol_smem_bytes<C>(nf, tx) > bound) tx >>= 1;
  return tx;
}

// Lanes per column of the z pass: NF/16 for the register transform, 16 for the FP32 16 x 10
// transform, 0 for the CTA-wide Stockham transform.
__host__ __device__ constexpr int zcol_lanes_of(bool f32, int nf) {
  return (nf == 64 || nf == 128 || nf == 256) ? nf / 16 : ((f32 && nf == 160) ? 16 : 0);
}
constexpr size_t kMaxSmem = 227 * 1024;

// Run-time shapes (RunTune) must divide the grid, fit shared memory and, for the lane-group
// transforms, give one of the instantiated CTA sizes (x-modes 4, 8 or 16).
template <typename C>
inline bool zcol_tile_ok(int nx, int nf, int tx) {
  if (tx < 1 || tx > 16 || nx % tx) return false;
  const int lanes = zcol_lanes_of(sizeof(C) == 8, nf);
  if (lanes && tx != 4 && tx != 8 && tx != 16) return false;
  if (!lanes && tx > Tune<C>::ZCOL_NT) return false;
  return zcol_smem_bytes<C>(nf, tx) <= kMaxSmem;
}
template <typename C>
inline bool rows_fwd_ok(int nx, int ny, int rb) {
  return rb >= 1 && ny % rb == 0 && (size_t)(rb * fft_phys(nx) + nx) * sizeof(C) <= kMaxSmem;
}
template <typename C>
inline bool cols_tile_ok(int nx, int ny, int tx) {
  return tx >= 1 && tx <= 256 && 256 % tx == 0 && nx % tx == 0 && cols_smem_bytes<C>(ny, tx) <= kMaxSmem;
}
template <typename C>
inline RunTune tune_of(const OpCall<C>& a) {
  return run_tune(sizeof(C) == 16, a.nx, a.ny, a.nslab, a.nf);
}
// The shapes the launches use: the tuned one when set and valid, else the built-in one.
template <typename C>
inline int zcol_tx_of(const OpCall<C>& a) {
  const int t = tune_of(a).zx;
  return (t && zcol_tile_ok<C>(a.nx, a.nf, t)) ? t : zcol_tile<C>(a.nx, a.nf);
}
template <typename C>
inline int rows_fwd_rb_of(const OpCall<C>& a) {
  const int t = tune_of(a).rb;
  return (t && rows_fwd_ok<C>(a.nx, a.ny, t)) ? t : row_block(a.nx, a.ny, Tune<C>::ROW_ELEMS);
}
template <typename C>
inline int cols_tx_of(const OpCall<C>& a) {
  const int t = tune_of(a).cx;
  return (t && cols_tile_ok<C>(a.nx, a.ny, t)) ? t : cols_tile<C>(a.nx, a.ny);
}

template <typename C, int NY, bool INV>
int launch_cols(const OpCall<C>& a) {
  constexpr int NT = 256;
  const int tx = cols_tx_of(a);
  const size_t smem = cols_smem_bytes<C>(NY, tx);
  auto k = k_cols<C, NY, INV, NT>;
  if (set_smem(k, smem, split_min_blocks<C, NY>() > 1)) return PSFD_E_CUDA;
  k<<<dim3(a.nslab * (a.nx / tx), 3, a.nrhs), NT, smem, a.stream>>>(a, tx);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <typename C, int NF, int NT>
int launch_zcol_nt(const OpCall<C>& a, int tx) {
  static_assert(((8 + (NF + 15) / 16) | 1) == phase_pitch<NF>(), "phase table size");
  const size_t smem = zcol_smem_bytes<C>(NF, tx);
  auto k = k_zcol<C, NF, NT>;
  if (set_smem(k, smem, zcol_min_blocks<C, NF, NT>() > 1)) return PSFD_E_CUDA;
  k<<<dim3(a.nx / tx, a.ny, a.nrhs), NT, smem, a.stream>>>(a, tx);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

// The lane-group transforms run 3 tx groups per CTA, one per (component, x-mode): the CTA
// size follows tx (instantiated for 4, 8 and 16 x-modes; fewer leave groups idle).
template <typename C, int NF>
int launch_zcol(const OpCall<C>& a) {
  constexpr int LN = zcol_lanes_of(sizeof(C) == 8, NF);
  const int tx = zcol_tx_of(a);
  if constexpr (LN > 0) {
    if (tx == 16) return launch_zcol_nt<C, NF, 3 * 16 * LN>(a, tx);
    if (tx == 8) return launch_zcol_nt<C, NF, 3 * 8 * LN>(a, tx);
    return launch_zcol_nt<C, NF, 3 * 4 * LN>(a, tx);
  } else {
    return launch_zcol_nt<C, NF, Tune<C>::ZCOL_NT>(a, tx);
  }
}

// ---------------------------------------------------------------------------
template <typename C, int IN>
int dispatch_fwd(const OpCall<C>& a) {
  if (use_fused<C>(a.nx, a.ny)) {
    switch (a.nx) {
#define X(n) \
  case n:    \
    if constexpr (n >= Tune<C>::HALF_MIN && n <= Tune<C>::FUSED_MAX && (n & (n - 1)) == 0) \
      return launch_half_fwd<C, n, IN>(a);                                                   \
    else if constexpr (n <= Tune<C>::FUSED_MAX && (n & (n - 1)) == 0)                        \
      return launch_plane_fwd<C, n, IN>(a);                                                  \
    break;
      PSFD_FOR_EACH_LENGTH(X)
#undef X
    }
    return PSFD_E_ARG;
  }
  int rc = PSFD_E_ARG;
  switch (a.nx) {
#define X(n) \
  case n:    \
    rc = launch_rows_fwd<C, n, IN>(a); \
    break;
    PSFD_FOR_EACH_LENGTH(X)
#undef X
  }
  if (rc) return rc;
  rc = PSFD_E_ARG;
  switch (a.ny) {
#define X(n) \
  case n:    \
    rc = launch_cols<C, n, false>(a); \
    break;
    PSFD_FOR_EACH_LENGTH(X)
#undef X
  }
  return rc;
}

template <typename C, int EPI>
int dispatch_inv(const OpCall<C>& a, const C* uin) {
  if (use_fused<C>(a.nx, a.ny)) {
    switch (a.nx) {
#define X(n) \
  case n:    \
    if constexpr (n >= Tune<C>::HALF_MIN && n <= Tune<C>::FUSED_MAX && (n & (n - 1)) == 0) \
      return launch_half_inv<C, n, EPI>(a, uin);                                             \
    else if constexpr (n <= Tune<C>::FUSED_MAX && (n & (n - 1)) == 0)                        \
      return launch_plane_inv<C, n, EPI>(a, uin);                                            \
    break;
      PSFD_FOR_EACH_LENGTH(X)
#undef X
    }
    return PSFD_E_ARG;
  }
  int rc = PSFD_E_ARG;
  switch (a.ny) {
#define X(n) \
  case n:    \
    rc = launch_cols<C, n, true>(a); \
    break;
    PSFD_FOR_EACH_LENGTH(X)
#undef X
  }
  if (rc) return rc;
  rc = PSFD_E_ARG;
  switch (a.nx) {
#define X(n) \
  case n:    \
    rc = launch_rows_inv<C, n, EPI>(a, uin); \
    break;
    PSFD_FOR_EACH_LENGTH(X)
#undef X
  }
  return rc;
}

template <typename C>
int dispatch_z(const OpCall<C>& a) {
  switch (a.nf) {
#define X(n) \
  case n:    \
    return launch_zcol<C, n>(a);
    PSFD_FOR_EACH_LENGTH(X)
#undef X
  }
  return PSFD_E_ARG;
}

// Algorithmic traffic and flops of the three passes, for the optional profiler: every
// vector read or written once, V once per launch; 5 N log2 N flops per complex FFT.
struct PassCost {
  double bytes[3], flops[3];
};
template <typename C>
PassCost pass_cost(const OpCall<C>& a) {
  const double b = sizeof(C), plane = (double)a.nx * a.ny;
  const double U = (double)a.nrhs * 3.0 * a.nslab * plane;
  const double vec = U * b, Vb = a.nslab * plane * b;
  PassCost c;
  const double nin = a.in_mode == IN_PLAIN ? 1 : (a.in_mode == IN_PUPDATE ? 3 : 2);
  const double nout = a.in_mode == IN_PLAIN ? 1 : 2;
  c.bytes[0] = (nin + nout) * vec + Vb;
  c.bytes[1] = 2 * vec + (double)a.nrhs * plane * sizeof(ModeEntry);
  double ninv = 3;  // W, u, out
  if (a.epi == EPI_RESID) ninv += 1;
  if (a.dot_mask & DOT_R0_OUT) ninv += 1;
  c.bytes[2] = ninv * vec;
  const double nplanes = (double)a.nrhs * 3.0 * a.nslab;
  c.flops[0] = nplanes * (5.0 * plane * std::log2(plane) + 6.0 * plane);
  c.flops[1] = (double)a.nrhs * plane * (3.0 * 2.0 * 5.0 * a.nf * std::log2((double)a.nf) + 80.0 * a.nf);
  c.flops[2] = nplanes * (5.0 * plane * std::log2(plane) + 2.0 * plane);
  return c;
}

// CTAs the xy passes (K1 or K3) and the z pass (K2) launch when every rhs is active.
template <typename C>
void pass_ctas(const OpCall<C>& a, double* xy, double* z) {
  const double planes = (double)a.nslab * 3.0 * a.nrhs;
  if (use_fused<C>(a.nx, a.ny)) {
    *xy = use_half<C>(a.nx, a.ny) ? 2 * planes : planes;
  } else {
    const int rb = rows_fwd_rb_of(a);
    *xy = planes * ((double)(a.ny / rb) + (double)(a.nx / cols_tx_of(a)));
  }
  *z = (double)(a.nx / zcol_tx_of(a)) * a.ny * a.nrhs;
}

template <typename C>
int op_apply_impl(const OpCall<C>& a0) {
  const bool f64 = sizeof(C) == 16;
  const bool prof = prof_on();
  OpCall<C> a = a0;
  PassCost cost;
  double cx = 0, cz = 0;
  if (prof) {
    cost = pass_cost(a);
    pass_ctas(a, &cx, &cz);
  }
  int rc;
  a.ctac = prof ? prof_begin(f64 ? PK_FWD64 : PK_FWD32, a.stream) : nullptr;
  switch (a.in_mode) {
    case IN_PLAIN: rc = dispatch_fwd<C, IN_PLAIN>(a); break;
    case IN_PUPDATE: rc = dispatch_fwd<C, IN_PUPDATE>(a); break;
    case IN_SUPDATE: rc = dispatch_fwd<C, IN_SUPDATE>(a); break;
    default: return PSFD_E_ARG;
  }
  if (rc) return rc;
  if (prof) prof_end(f64 ? PK_FWD64 : PK_FWD32, a.stream, cost.bytes[0], cost.flops[0], cx);
  a.ctac = prof ? prof_begin(f64 ? PK_Z64 : PK_Z32, a.stream) : nullptr;
  if ((rc = dispatch_z<C>(a))) return rc;
  if (prof) prof_end(f64 ? PK_Z64 : PK_Z32, a.stream, cost.bytes[1], cost.flops[1], cz);
  if (a.epi == EPI_NONE) return blocks_per_rhs_t<C>(a.nx, a.ny, a.nslab);
  const C* uin = a.in_mode == IN_PLAIN ? a.u : a.ustore;
  a.ctac = prof ? prof_begin(f64 ? PK_INV64 : PK_INV32, a.stream) : nullptr;
  switch (a.epi) {
    case EPI_AU: rc = dispatch_inv<C, EPI_AU>(a, uin); break;
    case EPI_RESID: rc = dispatch_inv<C, EPI_RESID>(a, uin); break;
    default: return PSFD_E_ARG;
  }
  if (rc) return rc;
  if (prof) prof_end(f64 ? PK_INV64 : PK_INV32, a.stream, cost.bytes[2], cost.flops[2], cx);
  return blocks_per_rhs_t<C>(a.nx, a.ny, a.nslab);
}

}  // namespace psfd
