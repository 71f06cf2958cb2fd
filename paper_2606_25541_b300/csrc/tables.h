// tables.h -- launchers of the FP64 set-up / post-processing kernels (tables.cu).
#pragma once

#include "internal.h"

namespace psfd {

struct StackDev {
  int n_layers;
  int reflect;           // 0: no stack (R = 0)
  const double2* eps;    // [n_layers] permittivity, top to bottom
  const double* d;       // [n_layers] thickness, nm
  double2 eps_sub;
};

struct ModesArgs {
  int nx, ny;
  double dx, dy, k0, eps_bg, L;
  const double* slot_qix;
  const double* slot_qiy;
  StackDev stack;
  ModeEntry* modes;  // [slot][ny][nx]
  int* anomaly;
};

struct OrdersArgs {
  int nx, ny, nslab;
  double dx, dy, dz, kb;
  const int* n_orders;  // [rhs]
  const int* mn;        // [rhs][max_orders][2]
  int max_orders;
  const RhsParam* rhsp;
  const ModeEntry* modes;
  const double2* side;  // [rhs][2][3][ny][nx]
  double* out;          // [rhs][max_orders][12]
};

int launch_potential(size_t n, const double2* eps, double k02, double eps_bg, double2* V64, float2* V32,
                     cudaStream_t st);
int launch_modes(const ModesArgs& a, int n_slots, cudaStream_t st);
int launch_rhs(int rhs0, int nrhs, RhsParam* rp, const ModeEntry* modes, int nx, int ny, int nslab, double dz,
               double kb, double2* b, cudaStream_t st);
int launch_orders(const OrdersArgs& a, int nrhs, cudaStream_t st);
int launch_norm(int n, int nblk, int rhs0, int nrhs, const double2* v, double2* partials, int maxblk, int mode,
                double tol2, KScal* sc, int* act, cudaStream_t st);
int launch_ref_scale(int n, int rhs0, int nrhs, const int* act, const KScal* sc, const double2* r64, float2* r32,
                     cudaStream_t st);
int launch_ref_update(int n, int rhs0, int nrhs, const int* act, const KScal* sc, double2* x64, const float2* x32,
                      cudaStream_t st);
int launch_test_fft(int n, int count, bool inv, bool fp64, void* data, const double2* tw);

}  // namespace psfd
