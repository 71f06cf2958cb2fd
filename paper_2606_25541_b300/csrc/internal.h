// internal.h -- structures shared by the CUDA translation units of libpsfd.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace psfd {

// Per-illumination parameters on the device.
struct RhsParam {
  double qix, qiy;    // transverse wavevector of the incident wave
  double cphi, sphi;  // azimuth; orients s at q = 0
  double2 e_inc[3];   // incident polarisation vector (bilinear unit)
  double2 r_inc[3];   // T_R(q_00) e_inc: reflected incident amplitude at z_top
  double2 beta00;     // z wavenumber of the specular order
  int slot;           // row of the mode tables
  int pol;
  int clip;           // which potential (mask clip) of the context this illumination sees
  int pad;
};

// Per transverse mode (m, n) and angle slot, computed in FP64 by the stack kernel.
struct ModeEntry {
  double2 beta;  // sqrt(k_bg^2 - |q|^2), Im >= 0
  double2 ebL;   // exp(i beta L), L = nf dz / 2
  double2 rs;    // stack reflection coefficient, s (E-field)
  double2 rp;    // stack reflection coefficient, p (H-field)
};

// FP32 copy of what the z-column kernel needs per mode, prepared by the FP64 stack
// kernel so that the FP32 hot path does no FP64 arithmetic.
struct ModeF32 {
  float qx, qy;     // transverse wavevector
  float2 bh, bl;    // beta split into FP32 hi + lo (beta - kappa stays exact near kappa)
  float2 ebL;       // exp(i beta L)
  float2 e1, e8;    // exp(i beta dz), exp(i beta 8 dz) (reflection phase table steps)
  float2 rs, rp;    // stack reflection coefficients
  float hx, hy;     // unit transverse direction (azimuth of the illumination at q = 0)
  float qnk, pad;   // |q| / kb
  float2 bq;        // beta / kb
};

// Double-float copy (unevaluated pairs hi + lo of FP32 numbers) of what the FP64 residual's
// double-float z pass needs per mode, prepared by the FP64 stack kernel once per illumination
// set-up, so that the pass itself runs no FP64 arithmetic. Complex values are float4
// (re.hi, re.lo, im.hi, im.lo), reals float2 (hi, lo).
struct ModeDF {
  float4 beta, ebL;  // beta, exp(i beta L)
  float4 e1, e8;     // exp(i beta dz), exp(i beta 8 dz)
  float4 rs, rp;     // stack reflection coefficients
  float4 bq;         // beta / kb
  float2 qx, qy;     // transverse wavevector
  float2 hx, hy;     // unit transverse direction (azimuth of the illumination at q = 0)
  float2 qnk, pad;   // |q| / kb
};

// Krylov scalars per right-hand side (BiCGStab), all FP64.
struct KScal {
  double2 rho, alpha, omega, beta;
  double bnorm2;  // ||b||^2 of the system being solved
  double rnorm2;  // ||r||^2 of the recursively updated residual
  double scale;   // defect-correction scale ||r64|| of this sweep
  double tol2;    // stop when rnorm2 <= tol2 bnorm2 (set when the solve starts)
  int iters;
  int active;  // 1 while iterating
  int status;  // PSFD_OK / PSFD_E_BREAKDOWN / PSFD_E_NOT_CONVERGED
  int pad;
};

// GMRES state per right-hand side (FP64; the Hessenberg matrix is tiny).
constexpr int KMAX = 24;  // basis vectors per cycle (PSFD_KRYLOV_MAX)
struct GmState {
  int j;       // vectors in the basis of this cycle (the newest is v_j)
  int m;       // cycle length
  int status;
  int pad;
  double beta;   // ||b|| of the system of this cycle
  double tol;    // relative residual target
  double inv_h;  // 1 / ||w|| for the normalisation of the newest vector
  double resid;  // current residual estimate |g_j| / beta
  double2 g[KMAX + 1];
  double cs[KMAX];
  double2 sn[KMAX];
  double2 H[(KMAX + 1) * KMAX];  // column j at H[j * (KMAX + 1) + i]
  double2 y[KMAX];
};

enum InMode { IN_PLAIN = 0, IN_PUPDATE = 1, IN_SUPDATE = 2 };
enum EpiMode { EPI_AU = 0, EPI_RESID = 1, EPI_NONE = 2 };
enum DotBits { DOT_R0_OUT = 1, DOT_OUT_U = 2, DOT_OUT_OUT = 4 };
constexpr int NDOT = 3;

// Everything one operator application needs. Vector pointers address the first RHS of
// the batch (local index 0); tables are indexed with rhs0 + local index.
template <typename C>
struct OpCall {
  int nx, ny, nslab, nf;
  int rhs0, nrhs;
  double dx, dy, dz, kb;
  float dz32, kb32;                             // dz and kb rounded to FP32 (FP32 kernels)
  const C* V;                                   // [nslab][ny][nx]
  const double2 *twx, *twy, *twz;               // exp(-2 pi i t / n) tables (FP64)
  const float2 *twx32, *twy32, *twz32;          // the same tables rounded to FP32 (FP32 kernels)
  const RhsParam* rhsp;
  const ModeEntry* modes;
  const ModeF32* modes32;  // FP32 column constants (used by the FP32 z-column kernel)
  const ModeDF* modesdf;   // double-float column constants (the residual's double-float z pass)
  const float4* twzdf;     // [nf]: the z twiddles as double-float pairs
  const float4 *twxdf, *twydf;  // [nx], [ny]: the x and y twiddles as pairs
  const float4* Vdf;       // V as pairs (same layout as V), or null
  const float2* kzdf;      // [nf]: signed kz_l as double-float pairs
  float2 dfL, dfcinv, dfscale;  // pairs of L = nf dz / 2, 1 / kb^2, 1 / (nf nx ny)
  const float* ktab32;     // [3][nf]: |kz_l| hi, |kz_l| lo, signed kz_l (FP32)
  const double* ktab64;    // [nf]: signed kz_l (FP64)
  const int* active;  // per global rhs, or null = all active
  int no_reflect;     // 1: leave R out, i.e. the free-space operator u - G*(V u)
  int pf;             // half-plane K1/K3: L2 prefetch of the planes of the CTA pf launches ahead (0: off)
  // isolated clip: per (slot, l <= nf/2, mode) the spherically windowed kernel's (A, B/|k|^2)
  // (FP32 float4 / FP64 pair of double2); null = the periodic z-windowed kernel
  const float4* sph32;
  const double2* sph64;
  // input stage: J = V * in, in = u | r + beta (u - omega v) | r - alpha v
  int in_mode;
  const C* u;
  C* ustore;  // updated p or s (IN_PUPDATE / IN_SUPDATE)
  const C* r;
  const C* v;
  const KScal* sc;
  C* work;  // [nrhs][3][nslab][ny][nx] spectral intermediate
  // epilogue: out = in - w (EPI_AU) or b - (in - w) (EPI_RESID), with dot products
  int epi;
  C* out;
  const C* b;
  const C* r0;
  double2* partials;  // [global rhs][NDOT][maxblk]
  int maxblk;
  int dot_mask;
  C* side;  // [global rhs][2][3][ny][nx] normalised spectra of G*(V u), planes 0, nslab+1
  cudaStream_t stream;
  unsigned* ctac;  // profiling only: counts the CTAs that did work (null otherwise)
};

// Runs K1 (V multiply + forward xy FFT), K2 (z column) and K3 (inverse xy + epilogue).
// Returns the number of partial-sum blocks per RHS written (>= 0) or a negative status.
template <typename C> int op_apply(const OpCall<C>& call);

// Partial-sum blocks per RHS that op_apply's epilogue writes for this grid.
int op_blocks_per_rhs(int nx, int ny, int nslab, bool fp64);

// Whether the kernels are built for an FFT length.
bool fft_length_supported(int n);

// Tile shapes chosen at run time by the autotuner (tune.cu), per grid and precision; a zero
// field keeps the built-in choice. Only shapes that leave every element's arithmetic and
// every reduction order unchanged are tunable, so a tuned operator gives bitwise the same
// results as the built-in one.
struct RunTune {
  int zx;  // K2: transverse x-modes per CTA of the z pass
  int rb;  // K1 on split planes: rows per CTA of the forward row pass
  int cx;  // split planes: columns per CTA of the column passes (forward and inverse)
  int pf;  // half-plane K1/K3: L2 prefetch distance in CTAs (0: no prefetch)
};
RunTune run_tune(bool fp64, int nx, int ny, int nslab, int nf);
void set_run_tune(bool fp64, int nx, int ny, int nslab, int nf, RunTune t);
bool has_run_tune(bool fp64, int nx, int ny, int nslab, int nf);
void clear_run_tune();

// Kernel-launch accounting and optional per-class CUDA-event timing (psfd.cu).
enum ProfClass {
  PK_FWD32 = 0, PK_Z32, PK_INV32, PK_FWD64, PK_Z64, PK_INV64, PK_VEC32, PK_VEC64, PK_SCALAR, PK_SETUP, PK_N
};
void count_launch(int n = 1);
unsigned long long launch_total();  // kernels launched by the library so far
bool prof_on();
// Opens a profiled launch of class cls on stream st; returns a device counter that the
// launch's CTAs increment when they do work (null when profiling is off).
unsigned* prof_begin(int cls, cudaStream_t st);
// Closes it: bytes / flops are the algorithmic figures of a launch in which all ctas_full
// CTAs work; the profile scales them by the counted fraction.
void prof_end(int cls, cudaStream_t st, double bytes, double flops, double ctas_full);

}  // namespace psfd

namespace psfd {

// One batched BiCGStab solve A x = b over right-hand sides op.rhs0 .. op.rhs0+op.nrhs-1.
template <typename C>
struct KrylovCall {
  OpCall<C> op;  // grid, tables, potential, stream, partial-sum buffer
  int n;         // complex elements per right-hand side
  const C* b;
  C *x, *r, *r0, *p, *v, *s, *t, *work;
  C* pn;  // BiCGStab: the updated p when the operator's input stage may not write p in place
  KScal* sc;           // per global rhs
  int* act;            // per global rhs, device
  const int* act_in;   // initial activity (device) or null
  int* h_act;          // pinned host mirror of act (>= rhs0 + nrhs entries)
  double tol;
  const double* tol_slot;  // per global rhs tolerance of this solve (device), or null = tol
  int max_iter;
  int check_every;
  // GMRES: basis vector i of global rhs g at basis + i * bstride + g * n; z = newest basis
  // vector (operator input), w = operator output; gpart = [rhs][KMAX + 1][gblk] partials
  C* basis;
  size_t bstride;
  C *z, *w;
  GmState* gm;
  double2* gpart;
  int gblk;
  int m;
};
// Start BiCGStab for the right-hand sides selected by mask (device, per global rhs; null =
// all): x = 0, r = r0 = b, scalars reset; others keep their state. No host synchronisation.
template <typename C> int bicg_start(const KrylovCall<C>& k, const int* mask);
// `iters` BiCGStab iterations for every right-hand side whose device flag act is set.
template <typename C> int bicg_iterate(const KrylovCall<C>& k, int iters);
// GMRES(m) with classical Gram-Schmidt: start a cycle on b for the rhs in mask, iterate the
// active ones, and form x = V y for the rhs in mask once their cycle has ended.
template <typename C> int gmres_start(const KrylovCall<C>& k, const int* mask);
template <typename C> int gmres_iterate(const KrylovCall<C>& k, int iters);
template <typename C> int gmres_finish(const KrylovCall<C>& k, const int* mask);

}  // namespace psfd
