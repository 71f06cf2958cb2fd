// tables.h -- launchers of the FP64 set-up / post-processing kernels (tables.cu).
#pragma once

#include "internal.h"

namespace psfd {

constexpr int kStackMaxLayers = 256;
constexpr int kMaxMat = 8, kMaxIface = 16, kMaxPh = 8;

struct StackDev {
  int n_layers;
  int reflect;           // 0: no stack (R = 0)
  const double2* eps;    // [n_layers] permittivity, top to bottom
  const double* d;       // [n_layers] thickness, nm
  double2 eps_sub;
  // A periodic stack has few distinct media, interfaces and (medium, thickness) layers;
  // when they fit these tables (n_mat > 0) each is evaluated once per mode.
  int n_mat, n_iface, n_ph;
  double2 mat_eps[kMaxMat];                     // media: ambient, layers, substrate (deduplicated)
  unsigned char iface_a[kMaxIface], iface_b[kMaxIface];  // upper / lower medium of an interface
  unsigned char ph_mat[kMaxPh];
  double ph_d[kMaxPh];
  unsigned char iface_of[kStackMaxLayers + 1];  // interface between medium j and j+1
  unsigned char layer_ph[kStackMaxLayers];      // (medium, thickness) class of layer j
  // Periodic run: layers run_top .. run_top + 2 run_k - 1 (1-based, top to bottom) are run_k
  // copies of one two-layer unit whose upper interface is the unit's own (the medium above
  // run_top equals the unit's second layer); run_k = 0 if there is none.
  int run_top, run_k;
};

// Fills the deduplication tables of st from host copies of the media (ambient first,
// then the layers top to bottom, then the substrate); leaves n_mat = 0 if they do not fit.
void stack_dedup(StackDev& st, const double2* eps_layers, const double* d_layers, int n_layers, double2 eps_amb,
                 double2 eps_sub);

struct ModesArgs {
  int slot0;  // first table row written (one launch covers rows slot0 .. slot0 + n_slots - 1)
  const int* slots;  // or, when not null, the rows slots[0 .. n_slots - 1] (device)
  int nx, ny;
  double dx, dy, dz, k0, kb, eps_bg, L;
  const double* slot_par;  // [slot][4]: q_inc x, q_inc y, cos phi, sin phi
  StackDev stack;
  ModeEntry* modes;   // [slot][ny][nx]
  ModeF32* modes32;   // [slot][ny][nx] or null
  ModeDF* modesdf;    // [slot][ny][nx] or null
  int* anomaly;
};

// Spherically windowed dyadic Green's function of an isolated clip (Sec. 3, Eqs. (13)-(17)):
// F[G_R](k) = A(|k|) I + B(|k|) khat khat^T at k = (q_x, q_y, kz_l) for l = 0 .. nf/2, stored
// per slot, l, mode as (A, B/|k|^2) times 1/(nf nx ny) (the inverse FFT normalisation).
struct SphArgs {
  int slot0, nx, ny, nf;
  double dx, dy, dz, kb, R;
  const double* slot_par;  // [slot][4]: q_inc x, q_inc y, ...
  double2* t64;            // [slot][nf/2 + 1][ny][nx][2]
  float4* t32;             // [slot][nf/2 + 1][ny][nx]
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
  const int* mask;      // right-hand sides to evaluate (null = all)
};

int launch_potential(size_t n, const double2* eps, double k02, double eps_bg, double2* V64, float2* V32, float4* Vdf,
                     cudaStream_t st);
int launch_modes(const ModesArgs& a, int n_slots, cudaStream_t st);
int launch_rhs(int rhs0, int nrhs, RhsParam* rp, const ModeEntry* modes, int nx, int ny, int nslab, double dz,
               double kb, double2* b, cudaStream_t st);
int launch_orders(const OrdersArgs& a, int nrhs, cudaStream_t st);
int launch_sph_table(const SphArgs& a, int n_slots, cudaStream_t st);
int launch_norm(int n, int nblk, int rhs0, int nrhs, const int* mask, const double2* v, double2* partials,
                int maxblk, int mode, double tol2, KScal* sc, int* act, cudaStream_t st);
template <typename C>
int launch_ref_scale(int n, int rhs0, int nrhs, const int* act, const KScal* sc, const double2* r64, C* rs,
                     cudaStream_t st);
template <typename C>
int launch_ref_update(int n, int rhs0, int nrhs, const int* act, const KScal* sc, double2* x64, const C* xc,
                      cudaStream_t st);
// a += b on the right-hand sides in mask (vectors [rhs][n], rhs0 the first one launched)
int launch_vec_add(int n, int rhs0, int nrhs, const int* mask, double2* a, const double2* b, cudaStream_t st);
int launch_test_fft(int n, int count, bool inv, bool fp64, void* data, const double2* tw);

}  // namespace psfd
