// ctx.h -- the solver context shared by the C ABI (psfd.cu), the solve engine
// (engine.cu) and the serving loop (server.cu). Private to the library.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/psfd.h"
#include "internal.h"
#include "tables.h"

namespace psfd {

constexpr double kPi = 3.14159265358979323846264338327950288;

struct Plan {
  size_t U = 0;      // complex elements per right-hand-side vector
  size_t plane = 0;  // nx * ny
  int maxblk = 1;
  int max_orders = 1;
  size_t bytes = 0;
};
// Krylov pool vectors a context starts with: BiCGStab's r, r0, p, v, s, t and pn. GMRES(m)
// needs m + 1 basis vectors plus z and w; the pool grows to that on the first GMRES solve.
constexpr int kPoolBicg = 7;
Plan make_plan(const psfd_grid& g, int precision, int max_rhs, int max_clips);
bool grid_ok(const psfd_grid* g, std::string& why);

// Krylov estimate of one slot after one tick of a device-side sweep loop (engine.cu).
struct LoopHist {
  int iters, pad;
  double rnorm2, bnorm2;
};
constexpr int kLoopHist = 128;  // ticks recorded per slot and loop

// Life cycle of one illumination in a context (see engine.cu).
enum Phase { PH_FREE = 0, PH_NEW, PH_START, PH_INNER, PH_RESID, PH_DONE };

struct StackHost {
  std::vector<double2> eps;  // permittivity per layer, top to bottom
  std::vector<double> d;     // thickness per layer, nm
  double2 eps_sub{1.0, 0.0};
  bool set = false;
};

}  // namespace psfd

struct psfd_ctx {
  psfd_grid g{};
  int precision = PSFD_FP64;
  int max_rhs = 0, max_clips = 1;
  size_t budget = 0, allocated = 0;
  cudaStream_t stream = nullptr;
  int device = 0;  // the CUDA device current when the context was created
  psfd::Plan plan;
  double k0 = 0, kb = 0, L = 0;
  std::string err;
  std::vector<std::pair<void*, size_t>> allocs;  // device buffers and their sizes

  // host state
  bool have_potential = false, have_illum = false, orders_on_host = false;
  int n_rhs = 0;                      // illuminations of the single-clip API (rhs 0 .. n_rhs-1)
  psfd::StackHost stack;              // stack of the single-clip API
  std::vector<psfd::RhsParam> h_rhsp;  // per rhs slot
  std::vector<int> h_nord, h_mn;
  std::vector<double> h_ordout;
  std::vector<double> th, ph;  // angles per rhs slot (degrees)
  std::vector<int> pol, clip;
  // engine state per rhs slot
  std::vector<int> phase, outer, iters, status;
  std::vector<int> guess;  // 1: x64 holds an initial guess for the slot's next solve
  // Residual history per slot (the convergence curve of the latest solve): kind 1 = the FP64
  // residual ||b - A x|| / ||b||, kind 0 = the Krylov estimate of a sweep (BiCGStab's recursive
  // residual scaled by the sweep's starting residual); iteration = Krylov iterations so far.
  struct HistEntry {
    int iteration, kind;
    double relres;
  };
  std::vector<std::vector<HistEntry>> hist;
  std::vector<double> sweep_rel;  // FP64 relative residual at the start of the current sweep
  int enq_hi = 0;  // slots covered by the work enqueued by engine_enqueue
  // Outer fixed-point iteration of Eq. (8) (engine_fixed_point): while set, every operator
  // application leaves R out, so the engine solves the free-space problem of one outer step.
  int no_reflect = 0;
  std::vector<double> relres;
  int* h_act = nullptr;      // pinned
  int* h_act64 = nullptr;    // pinned
  psfd::KScal* h_sc = nullptr;    // pinned
  psfd::KScal* h_sc64 = nullptr;  // pinned
  int* h_mask = nullptr;     // pinned staging for device masks

  // device state
  double2 *V64 = nullptr, *eps_stage = nullptr, *twx = nullptr, *twy = nullptr, *twz = nullptr;
  float2 *twx32 = nullptr, *twy32 = nullptr, *twz32 = nullptr;  // the twiddle tables rounded to FP32
  float2* V32 = nullptr;
  psfd::RhsParam* rhsp = nullptr;
  double* slot_par = nullptr;  // [rhs][4]: q_inc x, q_inc y, cos phi, sin phi
  psfd::ModeEntry* modes = nullptr;
  psfd::ModeF32* modes32 = nullptr;
  psfd::ModeDF* modesdf = nullptr;  // double-float column constants of the residual's z pass
  float4* twzdf = nullptr;          // z twiddles and kz_l as double-float pairs
  float4 *twxdf = nullptr, *twydf = nullptr;  // x and y twiddles as pairs
  float4* Vdf = nullptr;            // V64 as pairs (the residual's double-float row pass)
  float2* kzdf = nullptr;
  float* ktab32 = nullptr;
  double* ktab64 = nullptr;
  double2* d_eps_l = nullptr;
  double* d_d_l = nullptr;
  int* anomaly = nullptr;
  double2 *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *work64 = nullptr, *side64 = nullptr;
  // Krylov vectors in the context's working precision: rs = r64 / ||r64|| (the system each
  // sweep solves), xc = its solution, pool = pool_vecs vectors (BiCGStab: r, r0, p, v, s, t,
  // pn; GMRES(m): m + 1 basis vectors, z, w); each vector is [max_rhs][U]. The FP32 spectral
  // work buffer work32 lives inside work64: FP32 and FP64 applications never overlap on a
  // context's stream.
  double2 *rs64 = nullptr, *xc64 = nullptr, *pool64 = nullptr;
  float2 *x32 = nullptr, *r32 = nullptr, *work32 = nullptr, *pool32 = nullptr;
  int pool_vecs = 0;
  psfd::GmState* gm = nullptr;
  double2* gpart = nullptr;  // [rhs][KMAX + 1][gblk]
  int gblk = 1;
  double2* partials = nullptr;
  psfd::KScal *sc = nullptr, *sc64 = nullptr;
  int *act = nullptr, *act64 = nullptr;
  double* d_tol = nullptr;  // [max_rhs]: relative tolerance of each slot's current sweep
  std::vector<double> h_tol;
  int* d_mask[4] = {nullptr, nullptr, nullptr, nullptr};  // per-phase selections
  int *d_nord = nullptr, *d_mn = nullptr;
  int* d_slots = nullptr;  // the distinct table rows of an illumination set-up
  double* d_ordout = nullptr;
  double2* fp_b0 = nullptr;  // [max_rhs][U]: b = E_inc + R[E_inc] during a fixed-point solve (lazy)
  // isolated clip (psfd_set_green): spherically windowed kernel of radius green_R, tabulated
  // per illumination slot when the illuminations are set; no stack reflection
  int green = 0;
  double green_R = 0.0;
  double2* sph64 = nullptr;
  float4* sph32 = nullptr;

  // CUDA graphs of the Krylov step (engine.cu): one per launch configuration, replayed on
  // `stream`; captured on the private stream cap_stream.
  struct GraphEntry {
    long long key[8];
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int kernels;                  // kernel launches the graph holds (launch accounting)
    unsigned long long last_use;  // for evicting the least recently used entry
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  bool use_graphs = true;
  // Device-side sweep loop (engine.cu): while every busy slot is inside a Krylov sweep, the
  // ticks repeat inside one graph launch (a WHILE node) until no slot is active, so the host
  // waits once per sweep instead of once per tick.
  bool device_loop = true;
  int* d_loop = nullptr;              // [0]: ticks run by the current loop
  int* d_prev_act = nullptr;          // [max_rhs]: activity at the start of the current tick
  psfd::LoopHist* d_lhist = nullptr;  // [max_rhs][kLoopHist]: Krylov estimate after each tick
  int* d_lhist_n = nullptr;           // [max_rhs]
  int* h_loop = nullptr;              // pinned mirrors of the three above
  psfd::LoopHist* h_lhist = nullptr;
  int* h_lhist_n = nullptr;
  bool loop_ran = false;              // the enqueued tick was a device-side loop
  int loop_kernels = 0;               // kernels per tick of that loop
  int loop_precounted = 0;            // of those, already counted while capturing
  int resid_arith = PSFD_RESID_DFLOAT;  // arithmetic of the refined solve's FP64 residual
  unsigned long long graph_clock = 0;
  void drop_graphs() {
    for (auto& e : graphs) {
      cudaGraphExecDestroy(e.exec);
      cudaGraphDestroy(e.graph);
    }
    graphs.clear();
  }

  int fail(int code, const std::string& what) {
    err = what;
    return code;
  }
  int cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return PSFD_E_CUDA;
  }
  template <typename T>
  int dalloc(T** p, size_t count) {
    const size_t bytes = (count > 0 ? count : 1) * sizeof(T);
    if (budget && allocated + bytes > budget)
      return fail(PSFD_E_BUDGET, "allocation of " + std::to_string(bytes) + " bytes exceeds the HBM budget");
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PSFD_E_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    allocs.push_back({q, bytes});
    allocated += bytes;
    *p = static_cast<T*>(q);
    return PSFD_OK;
  }
  void dfree(void* q) {
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i].first == q) {
        cudaFree(q);
        allocated -= allocs[i].second;
        allocs.erase(allocs.begin() + (long)i);
        return;
      }
  }
  ~psfd_ctx() {
    drop_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto& q : allocs) cudaFree(q.first);
    for (void* q : {(void*)h_act, (void*)h_act64, (void*)h_sc, (void*)h_sc64, (void*)h_mask, (void*)h_loop,
                    (void*)h_lhist, (void*)h_lhist_n})
      if (q) cudaFreeHost(q);
  }
};

#define CK(call)                                             \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call); \
  } while (0)
#define RC(call)                              \
  do {                                        \
    int rc_ = (call);                         \
    if (rc_ < 0) {                            \
      if (ctx->err.empty()) ctx->err = #call; \
      return rc_;                             \
    }                                         \
  } while (0)

namespace psfd {

// Context with room for max_rhs illuminations over up to max_clips potentials.
int ctx_create(psfd_ctx** out, const psfd_grid* grid, int precision, int max_rhs, int max_clips,
               size_t hbm_budget, cudaStream_t stream);
// Grow the Krylov pool to what opts.krylov needs; extra bytes that takes for a plan.
int ensure_pool(psfd_ctx* ctx, const psfd_solve_opts& o);
size_t pool_extra_bytes(const Plan& p, int precision, int max_rhs, const psfd_solve_opts& o);

// Potential of clip `clip` from eps (host or device, complex double [nslab][ny][nx]).
int ctx_set_potential(psfd_ctx* ctx, int clip, const double* eps, int where);

// Illuminations for rhs slots g0 .. g0+n-1 seeing clip `clip` through the given stack:
// host anomaly check and order lists, then per-mode tables and right-hand sides on the
// device. The slots' phase becomes PH_NEW.
int ctx_set_rhs(psfd_ctx* ctx, int g0, int n, const double* theta, const double* phi, const int* pol, int clip,
                const StackHost& stack);

// Solve engine: one tick advances every slot by one phase step (see engine.cu).
int engine_tick(psfd_ctx* ctx, const psfd_solve_opts& o, int* n_active);
// The two halves of a tick: enqueue the work (no host wait), then wait and transition.
// With loop_deferred non-null, a tick in which every busy slot is inside a Krylov sweep is
// only prepared (*loop_deferred = true): the caller adds the context's loop to a graph
// (add_sweep_loop), launches it, then calls loop_readback and engine_readback.
int engine_enqueue(psfd_ctx* ctx, const psfd_solve_opts& o, bool* pending, bool* loop_deferred);
int engine_complete(psfd_ctx* ctx, const psfd_solve_opts& o, int* n_active);
int engine_readback(psfd_ctx* ctx);
int add_sweep_loop(psfd_ctx* ctx, const psfd_solve_opts& o, int hi, bool f32, cudaGraph_t g, int cap, int* kernels);
int loop_readback(psfd_ctx* ctx, int hi);
// The paper's outer fixed-point loop (Eqs. (8)-(9)) over rhs slots 0 .. n_rhs-1.
int engine_fixed_point(psfd_ctx* ctx, const psfd_solve_opts& o, int max_steps, double step_tol);
psfd_solve_opts solve_defaults(const psfd_solve_opts* opts);

// Copy the orders of the finished slots to the host cache (once per batch of finishes).
int ctx_orders_to_host(psfd_ctx* ctx);

OpCall<float2> base_call32(psfd_ctx* ctx, int rhs0, int nrhs);
OpCall<double2> base_call64(psfd_ctx* ctx, int rhs0, int nrhs);

}  // namespace psfd
