// engine.cu -- the solve engine: every illumination ("rhs slot") of a context moves
// through its own phases, and one tick advances all of them with shared launches.
//
//   PH_NEW    right-hand side just built: ||b|| is taken, x64 = 0, r64 = b (with an initial
//             guess x64 is kept and the slot goes to PH_RESID)
//   PH_START  a refinement sweep starts: rs = r64 / ||r64|| in the working precision (FP32
//             for PSFD_FP32_REFINED, FP64 for PSFD_FP64) and a Krylov solve of A xc = rs
//             (BiCGStab by default, or GMRES) is initialised
//   PH_INNER  Krylov iterations (check_every per tick; the device flag of a slot drops when
//             its residual estimate reaches the sweep's tolerance, its GMRES cycle is full,
//             or it breaks down); then x64 += ||r64|| xc
//   PH_RESID  FP64 residual r64 = b - A x64 (and the spectra for the orders); done when
//             ||r64|| <= tol ||b||, else a new sweep (at most max_outer)
//   PH_DONE   orders computed
// The FP64 path is the same loop with an FP64 Krylov solve to tol/2, so one sweep normally
// suffices; the FP32 path solves each sweep to inner_tol.
//
// Slots in different phases coexist in one batch: every kernel takes a per-slot mask or
// activity flag, and all reductions are per slot and in a fixed order, so a slot's result
// does not depend on which other slots share the context or when they were admitted.
// A tick is split in two so that a caller driving several contexts can overlap them:
// engine_enqueue puts the tick's work and the read-back of the per-slot scalars on the
// context's stream; engine_complete waits for it and applies the phase transitions.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "dfloat_ops.h"

namespace psfd {

psfd_solve_opts solve_defaults(const psfd_solve_opts* opts) {
  psfd_solve_opts o{};
  if (opts) o = *opts;
  if (!(o.tol > 0)) o.tol = 1e-10;
  if (o.max_iter <= 0) o.max_iter = 500;
  if (o.max_outer <= 0) o.max_outer = 12;
  if (!(o.inner_tol > 0)) o.inner_tol = 1e-4;
  if (o.check_every <= 0) o.check_every = 4;
  return o;
}

namespace {

constexpr double kSweepSafety = 0.25;

int upload_mask(psfd_ctx* ctx, int which, const std::vector<int>& sel) {
  // pageable source: the copy is staged before the call returns, so `sel` may be reused
  CK(cudaMemcpyAsync(ctx->d_mask[which], sel.data(), sizeof(int) * sel.size(), cudaMemcpyHostToDevice, ctx->stream));
  return PSFD_OK;
}

// The Krylov solve of one refinement sweep: rs x = rs-system in the context's working
// precision; b = rs, x = xc, GMRES basis / z / w in the pool (BiCGStab uses pool vectors 0-5).
template <typename C>
KrylovCall<C> krylov_common(psfd_ctx* ctx, const psfd_solve_opts& o, OpCall<C> op, C* rs, C* xc, C* work, C* pool,
                            double tol) {
  KrylovCall<C> k;
  std::memset(&k, 0, sizeof(k));
  k.op = op;
  k.n = (int)ctx->plan.U;
  const size_t bs = (size_t)ctx->max_rhs * ctx->plan.U;
  k.b = rs;
  k.x = xc;
  k.work = work;
  k.basis = pool;
  k.bstride = bs;
  k.m = (o.restart > 0 && o.restart < KMAX) ? o.restart : KMAX;
  k.z = pool + (size_t)(k.m + 1) * bs;
  k.w = k.z + bs;
  k.r = pool;
  k.r0 = pool + bs;
  k.p = pool + 2 * bs;
  k.v = pool + 3 * bs;
  k.s = pool + 4 * bs;
  k.t = pool + 5 * bs;
  k.pn = pool + 6 * bs;
  k.gm = ctx->gm;
  k.gpart = ctx->gpart;
  k.gblk = ctx->gblk;
  k.sc = ctx->sc;
  k.act = ctx->act;
  k.h_act = ctx->h_act;
  k.tol = tol;
  k.tol_slot = ctx->precision == PSFD_FP32_REFINED ? ctx->d_tol : nullptr;
  k.max_iter = o.max_iter;
  k.check_every = o.check_every;
  return k;
}

template <typename C>
KrylovCall<C> krylov_of(psfd_ctx* ctx, const psfd_solve_opts& o, int hi);

template <>
KrylovCall<float2> krylov_of<float2>(psfd_ctx* ctx, const psfd_solve_opts& o, int hi) {
  return krylov_common<float2>(ctx, o, base_call32(ctx, 0, hi), ctx->r32, ctx->x32, ctx->work32, ctx->pool32,
                               o.inner_tol);
}

template <>
KrylovCall<double2> krylov_of<double2>(psfd_ctx* ctx, const psfd_solve_opts& o, int hi) {
  // the FP64 path converges in one sweep: inner target below the outer one
  return krylov_common<double2>(ctx, o, base_call64(ctx, 0, hi), ctx->rs64, ctx->xc64, ctx->work64, ctx->pool64,
                                0.5 * o.tol);
}

template <typename C>
int krylov_start(psfd_ctx* ctx, const psfd_solve_opts& o, int hi, const int* mask) {
  const KrylovCall<C> k = krylov_of<C>(ctx, o, hi);
  C* rs = const_cast<C*>(k.b);
  RC(launch_ref_scale<C>((int)ctx->plan.U, 0, hi, mask, ctx->sc64, ctx->r64, rs, ctx->stream));
  if (o.krylov == PSFD_BICGSTAB) return bicg_start<C>(k, mask);
  return gmres_start<C>(k, mask);
}

template <typename C>
int krylov_iterate(psfd_ctx* ctx, const psfd_solve_opts& o, int hi) {
  const KrylovCall<C> k = krylov_of<C>(ctx, o, hi);
  if (o.krylov == PSFD_BICGSTAB) return bicg_iterate<C>(k, o.check_every);
  return gmres_iterate<C>(k, o.check_every);
}

// End of a sweep for the rhs in mask: xc (GMRES: V y), then x64 += ||r64|| xc.
template <typename C>
int krylov_finish(psfd_ctx* ctx, const psfd_solve_opts& o, int hi, const int* mask) {
  const KrylovCall<C> k = krylov_of<C>(ctx, o, hi);
  if (o.krylov != PSFD_BICGSTAB) RC(gmres_finish<C>(k, mask));
  RC(launch_ref_update<C>((int)ctx->plan.U, 0, hi, mask, ctx->sc64, ctx->x64, k.x, ctx->stream));
  return PSFD_OK;
}

// End of one tick of a device-side sweep loop: record the Krylov estimate of every slot that
// was active when the tick began, and keep the loop going while some slot is still active and
// fewer than `cap` ticks have run (the cap is a backstop: the Krylov kernels drop a slot's
// flag at max_iter, so the loop ends on its own; a loop stopped by the cap leaves its active
// slots to the host's next tick).
__global__ void k_sweep_cond(cudaGraphConditionalHandle cond, int R, const int* act, const KScal* sc,
                             int* prev_act, int* tick, int cap, LoopHist* hist, int* hist_n) {
  int any = 0;
  for (int g = threadIdx.x; g < R; g += blockDim.x) {
    if (prev_act[g]) {
      const int n = hist_n[g];
      if (n < kLoopHist) {
        LoopHist h;
        h.iters = sc[g].iters;
        h.pad = 0;
        h.rnorm2 = sc[g].rnorm2;
        h.bnorm2 = sc[g].bnorm2;
        hist[(size_t)g * kLoopHist + n] = h;
        hist_n[g] = n + 1;
      }
    }
    const int a = act[g];
    prev_act[g] = a;
    any |= a;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    const int t = *tick + 1;
    *tick = t;
    cudaGraphSetConditional(cond, (any && t < cap) ? 1u : 0u);
  }
}

// Device buffers of the sweep loop (allocated on first use).
int ensure_loop_buffers(psfd_ctx* ctx) {
  if (ctx->d_loop) return PSFD_OK;
  const int n = ctx->max_rhs;
  RC(ctx->dalloc(&ctx->d_loop, 1));
  RC(ctx->dalloc(&ctx->d_prev_act, n));
  RC(ctx->dalloc(&ctx->d_lhist, (size_t)n * kLoopHist));
  RC(ctx->dalloc(&ctx->d_lhist_n, n));
  CK(cudaMallocHost(&ctx->h_loop, sizeof(int)));
  CK(cudaMallocHost(&ctx->h_lhist, sizeof(LoopHist) * (size_t)n * kLoopHist));
  CK(cudaMallocHost(&ctx->h_lhist_n, sizeof(int) * n));
  return PSFD_OK;
}

}  // namespace

// Adds to graph g one WHILE node (condition 1 at every launch of g, no dependencies) whose body
// is one tick of the context -- check_every Krylov iterations of its active slots -- followed
// by k_sweep_cond with the given tick cap; the body is captured on the context's private
// stream. *kernels: the kernels one tick launches.
int add_sweep_loop(psfd_ctx* ctx, const psfd_solve_opts& o, int hi, bool f32, cudaGraph_t g, int cap, int* kernels) {
  RC(ensure_loop_buffers(ctx));
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  cudaGraphConditionalHandle cond;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  cudaGraphNode_t node;
  cudaError_t ge = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  if (ge == cudaSuccess) {
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    ge = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  }
  if (ge == cudaSuccess)
    ge = cudaStreamBeginCaptureToGraph(ctx->cap_stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeRelaxed);
  if (ge != cudaSuccess) return ctx->cuda_fail(ge, "device loop graph");
  cudaStream_t user = ctx->stream;
  const unsigned long long n0 = launch_total();
  ctx->stream = ctx->cap_stream;
  int rc = f32 ? krylov_iterate<float2>(ctx, o, hi) : krylov_iterate<double2>(ctx, o, hi);
  if (rc == PSFD_OK) {
    k_sweep_cond<<<1, 256, 0, ctx->cap_stream>>>(cond, hi, ctx->act, ctx->sc, ctx->d_prev_act, ctx->d_loop, cap,
                                                  ctx->d_lhist, ctx->d_lhist_n);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = PSFD_E_CUDA;
  }
  ctx->stream = user;
  cudaGraph_t body = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &body);
  *kernels = (int)(launch_total() - n0);
  if (rc != PSFD_OK || ce != cudaSuccess) {
    cudaGetLastError();
    if (rc != PSFD_OK) return rc;
    return ctx->cuda_fail(ce, "cudaStreamEndCapture (device loop)");
  }
  return PSFD_OK;
}

// Before a loop launch: tick counter and history cleared, activity at the start recorded.
int loop_prepare(psfd_ctx* ctx, int hi) {
  RC(ensure_loop_buffers(ctx));
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(ctx->d_loop, 0, sizeof(int), st));
  CK(cudaMemsetAsync(ctx->d_lhist_n, 0, sizeof(int) * hi, st));
  CK(cudaMemcpyAsync(ctx->d_prev_act, ctx->act, sizeof(int) * hi, cudaMemcpyDeviceToDevice, st));
  return PSFD_OK;
}

// After a loop launch: its ticks and history, then the per-slot scalars, back to the host.
int loop_readback(psfd_ctx* ctx, int hi) {
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->h_loop, ctx->d_loop, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->h_lhist_n, ctx->d_lhist_n, sizeof(int) * hi, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->h_lhist, ctx->d_lhist, sizeof(LoopHist) * (size_t)hi * kLoopHist, cudaMemcpyDeviceToHost,
                     st));
  ctx->loop_ran = true;
  return PSFD_OK;
}

namespace {

// check_every Krylov iterations of the slots whose device flag is up. The launch sequence
// depends only on the configuration in the key below (the per-slot state -- scalars, flags,
// vectors -- lives on the device), so it is captured once into a CUDA graph and replayed:
// one launch per tick instead of about ten per iteration. Profiling runs bypass the graphs
// (their events are recorded per launch). The capture happens on the context's private
// stream in relaxed mode; nothing runs during it, and the first replay follows at once.
// With loop = true the graph is a WHILE node whose body is one tick followed by
// k_sweep_cond: one launch runs ticks until no slot is active (the whole sweep).
int inner_step(psfd_ctx* ctx, const psfd_solve_opts& o, int hi, bool f32, bool loop) {
  auto direct = [&]() { return f32 ? krylov_iterate<float2>(ctx, o, hi) : krylov_iterate<double2>(ctx, o, hi); };
  if (!ctx->use_graphs || prof_on()) return direct();
  long long tol_bits;
  const double tol = f32 ? o.inner_tol : 0.5 * o.tol;
  std::memcpy(&tol_bits, &tol, sizeof(tol_bits));
  const int cap = (o.max_iter + o.check_every - 1) / o.check_every + 1;
  const long long key[8] = {hi | ((long long)cap << 20),
                            (long long)f32 | ((long long)loop << 1),
                            o.krylov,
                            o.krylov == PSFD_BICGSTAB ? 0 : o.restart,
                            o.check_every,
                            ((long long)o.max_iter << 1) | ctx->no_reflect,
                            tol_bits,
                            (long long)(f32 ? (uintptr_t)ctx->pool32 : (uintptr_t)ctx->pool64)};
  psfd_ctx::GraphEntry* hit = nullptr;
  for (auto& e : ctx->graphs)
    if (std::memcmp(e.key, key, sizeof(key)) == 0) hit = &e;
  int precounted = 0;
  if (!hit) {
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    constexpr size_t kMaxGraphs = 32;
    if (ctx->graphs.size() >= kMaxGraphs) {  // evict the least recently used
      auto old = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                  [](const auto& a, const auto& b) { return a.last_use < b.last_use; });
      cudaGraphExecDestroy(old->exec);
      cudaGraphDestroy(old->graph);
      ctx->graphs.erase(old);
    }
    psfd_ctx::GraphEntry e{};
    std::memcpy(e.key, key, sizeof(key));
    cudaStream_t user = ctx->stream;
    const unsigned long long n0 = launch_total();
    cudaGraph_t g = nullptr;
    if (loop) {
      CK(cudaGraphCreate(&g, 0));
      int kernels = 0;
      const int rc = add_sweep_loop(ctx, o, hi, f32, g, cap, &kernels);
      if (rc != PSFD_OK) {
        cudaGraphDestroy(g);
        return rc;
      }
    } else {
      CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
      ctx->stream = ctx->cap_stream;
      const int rc = direct();
      ctx->stream = user;
      const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
      if (rc != PSFD_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (rc != PSFD_OK) return rc;
        return ctx->cuda_fail(ce, "cudaStreamEndCapture");
      }
    }
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, g, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(g);
      return ctx->cuda_fail(ie, "cudaGraphInstantiate");
    }
    e.graph = g;
    e.kernels = (int)(launch_total() - n0);  // counted during the capture, run by the first replay
    ctx->graphs.push_back(e);
    hit = &ctx->graphs.back();
    precounted = e.kernels;
  } else if (!loop) {
    count_launch(hit->kernels);
  }
  hit->last_use = ++ctx->graph_clock;
  if (loop) {  // a loop's kernel count is known once its ticks are read back (engine_complete)
    ctx->loop_kernels = hit->kernels;
    ctx->loop_precounted = precounted;
  }
  CK(cudaGraphLaunch(hit->exec, ctx->stream));
  return PSFD_OK;
}

// Whether the refined solve's FP64 residual runs its z pass in double-float.
static bool resid_df(const psfd_ctx* ctx) {
  return ctx->precision == PSFD_FP32_REFINED && ctx->resid_arith == PSFD_RESID_DFLOAT;
}

// r64 = b - A x64 with the side spectra, then ||r64||^2 into sc64 / act64, for the slots in mask.
int fp64_residual(psfd_ctx* ctx, const int* mask, double tol, int hi) {
  OpCall<double2> a = base_call64(ctx, 0, hi);
  a.active = mask;
  a.u = ctx->x64;
  a.out = ctx->r64;
  a.b = ctx->b64;
  a.epi = EPI_RESID;
  a.work = ctx->work64;
  a.dot_mask = DOT_OUT_OUT;
  a.side = ctx->side64;
  const int nb = resid_df(ctx) ? op_apply_df(a) : op_apply<double2>(a);
  RC(nb);
  RC(launch_norm((int)ctx->plan.U, nb, 0, hi, mask, nullptr, ctx->partials, ctx->plan.maxblk, 1, tol * tol,
                 ctx->sc64, ctx->act64, ctx->stream));
  return PSFD_OK;
}

int compute_orders(psfd_ctx* ctx, const int* mask, int hi) {
  OrdersArgs o;
  o.nx = ctx->g.nx;
  o.ny = ctx->g.ny;
  o.nslab = ctx->g.nslab;
  o.dx = ctx->g.dx;
  o.dy = ctx->g.dy;
  o.dz = ctx->g.dz;
  o.kb = ctx->kb;
  o.n_orders = ctx->d_nord;
  o.mn = ctx->d_mn;
  o.max_orders = ctx->plan.max_orders;
  o.rhsp = ctx->rhsp;
  o.modes = ctx->modes;
  o.side = ctx->side64;
  o.out = ctx->d_ordout;
  o.mask = mask;
  RC(launch_orders(o, hi, ctx->stream));
  ctx->orders_on_host = false;
  return PSFD_OK;
}

}  // namespace

// Launches of a tick cover slots [0, hi): hi is one past the last slot with work.
static int busy_hi(const psfd_ctx* ctx) {
  int hi = 0;
  for (int g = 0; g < ctx->max_rhs; ++g)
    if (ctx->phase[g] != PH_FREE && ctx->phase[g] != PH_DONE) hi = g + 1;
  return hi;
}

int engine_enqueue(psfd_ctx* ctx, const psfd_solve_opts& o, bool* pending, bool* loop_deferred) {
  const int R = busy_hi(ctx);
  if (loop_deferred) *loop_deferred = false;
  const size_t U = ctx->plan.U;
  const bool f32 = ctx->precision == PSFD_FP32_REFINED;
  cudaStream_t st = ctx->stream;
  const int vblk = std::max(1, std::min(ctx->plan.maxblk, (int)((U + 8191) / 8192)));
  *pending = false;
  ctx->enq_hi = R;
  if (R == 0) return PSFD_OK;
  std::vector<int> sel(R);
  auto select = [&](int ph) {
    int n = 0;
    for (int g = 0; g < R; ++g) {
      sel[g] = ctx->phase[g] == ph;
      n += sel[g];
    }
    return n;
  };
  if (select(PH_NEW)) {
    RC(upload_mask(ctx, 0, sel));
    RC(launch_norm((int)U, vblk, 0, R, ctx->d_mask[0], ctx->b64, ctx->partials, ctx->plan.maxblk, 0,
                   o.tol * o.tol, ctx->sc64, ctx->act64, st));
    for (int g = 0; g < R; ++g) {
      if (!sel[g]) continue;
      if (!ctx->guess[g]) {  // with an initial guess, x64 holds it and r64 comes from PH_RESID
        CK(cudaMemsetAsync(ctx->x64 + (size_t)g * U, 0, sizeof(double2) * U, st));
        CK(cudaMemcpyAsync(ctx->r64 + (size_t)g * U, ctx->b64 + (size_t)g * U, sizeof(double2) * U,
                           cudaMemcpyDeviceToDevice, st));
      }
      CK(cudaMemsetAsync(ctx->side64 + (size_t)g * 6 * ctx->plan.plane, 0, sizeof(double2) * 6 * ctx->plan.plane,
                         st));
    }
    *pending = true;
  }
  if (select(PH_RESID)) {
    RC(upload_mask(ctx, 1, sel));
    RC(fp64_residual(ctx, ctx->d_mask[1], o.tol, R));
    *pending = true;
  }
  ctx->loop_ran = false;
  if (select(PH_INNER)) {
    // every busy slot inside a sweep: run the sweep to its end on the device
    const bool loop = (ctx->device_loop || loop_deferred) && ctx->use_graphs && !prof_on() && !*pending;
    *pending = true;
    if (loop) {
      RC(loop_prepare(ctx, R));
      if (loop_deferred) {  // the caller launches the loop (in a graph of several contexts)
        *loop_deferred = true;
        return PSFD_OK;
      }
    }
    RC(inner_step(ctx, o, R, f32, loop));
    if (loop) RC(loop_readback(ctx, R));
  }
  if (*pending) RC(engine_readback(ctx));
  return PSFD_OK;
}

// Read-back of the per-slot scalars of the enqueued work, waited for in engine_complete.
int engine_readback(psfd_ctx* ctx) {
  const int R = ctx->enq_hi;
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->h_sc64, ctx->sc64, sizeof(KScal) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(KScal) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->h_act, ctx->act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  return PSFD_OK;
}

int engine_complete(psfd_ctx* ctx, const psfd_solve_opts& o, int* n_active) {
  const int R = ctx->enq_hi;
  const size_t U = ctx->plan.U;
  const bool f32 = ctx->precision == PSFD_FP32_REFINED;
  cudaStream_t st = ctx->stream;
  if (R > 0) {
    CK(cudaStreamSynchronize(st));
    if (ctx->loop_ran)  // kernels the loop ran: its ticks times the kernels of one tick
      count_launch(std::max(0, *ctx->h_loop * ctx->loop_kernels - ctx->loop_precounted));
    std::vector<int> to_update(R, 0), to_start(R, 0), to_done(R, 0);
    const double tol2 = o.tol * o.tol;
    auto record = [&](int g, int it, int kind, double rel) {
      auto& h = ctx->hist[g];
      if (h.size() < 100000) h.push_back({it, kind, rel});
    };
    bool any_update = false, any_start = false, any_done = false;
    for (int g = 0; g < R; ++g) {
      const KScal& s64 = ctx->h_sc64[g];
      switch (ctx->phase[g]) {
        case PH_NEW:
          ctx->outer[g] = 0;
          ctx->iters[g] = 0;
          ctx->status[g] = PSFD_OK;
          ctx->hist[g].clear();
          ctx->sweep_rel[g] = 1.0;
          if (!ctx->guess[g]) record(g, 0, 1, s64.bnorm2 > 0.0 ? 1.0 : 0.0);  // x = 0: r = b
          if (!(s64.bnorm2 > 0.0)) {  // zero right-hand side: x = 0 is exact
            if (ctx->guess[g]) CK(cudaMemsetAsync(ctx->x64 + (size_t)g * U, 0, sizeof(double2) * U, st));
            ctx->relres[g] = 0.0;
            to_done[g] = 1;
          } else if (ctx->guess[g]) {  // warm start: its FP64 residual decides what comes next
            ctx->phase[g] = PH_RESID;
          } else {
            to_start[g] = 1;
          }
          ctx->guess[g] = 0;
          break;
        case PH_RESID: {
          const double rel = std::sqrt(s64.rnorm2 / s64.bnorm2);
          ctx->relres[g] = rel;
          ctx->sweep_rel[g] = rel;
          record(g, ctx->iters[g], 1, rel);
          if (s64.rnorm2 <= tol2 * s64.bnorm2) {
            ctx->status[g] = PSFD_OK;
            to_done[g] = 1;
          } else if (ctx->outer[g] >= o.max_outer || !std::isfinite(rel)) {
            ctx->status[g] = std::isfinite(rel) ? PSFD_E_NOT_CONVERGED : PSFD_E_BREAKDOWN;
            to_done[g] = 1;
          } else {
            to_start[g] = 1;
          }
          break;
        }
        case PH_INNER: {
          const KScal& si = ctx->h_sc[g];
          if (ctx->loop_ran) {  // the estimates after every tick of the device-side loop
            for (int k = 0; k < std::min(ctx->h_lhist_n[g], kLoopHist); ++k) {
              const LoopHist& h = ctx->h_lhist[(size_t)g * kLoopHist + k];
              if (o.krylov != PSFD_GMRES && h.bnorm2 > 0.0 && h.iters > 0)
                record(g, ctx->iters[g] + h.iters, 0, std::sqrt(h.rnorm2 / h.bnorm2) * ctx->sweep_rel[g]);
            }
          } else if (o.krylov != PSFD_GMRES && si.bnorm2 > 0.0 && si.iters > 0) {
            record(g, ctx->iters[g] + si.iters, 0, std::sqrt(si.rnorm2 / si.bnorm2) * ctx->sweep_rel[g]);
          }
          if (!ctx->h_act[g]) {  // sweep ended (converged, cycle full or breakdown): correct x64
            ctx->iters[g] += si.iters;
            to_update[g] = 1;
          }
          break;
        }
        default:
          break;
      }
      any_update = any_update || to_update[g];
      any_start = any_start || to_start[g];
      any_done = any_done || to_done[g];
    }
    // sweep updates, then Krylov starts, then orders of the finished slots
    if (any_update) {
      RC(upload_mask(ctx, 2, to_update));
      if (f32) RC(krylov_finish<float2>(ctx, o, R, ctx->d_mask[2]));
      else RC(krylov_finish<double2>(ctx, o, R, ctx->d_mask[2]));
      for (int g = 0; g < R; ++g)
        if (to_update[g]) ctx->phase[g] = PH_RESID;
    }
    if (any_start) {
      if (f32) {
        // A sweep only has to take the FP64 residual from sweep_rel down to tol: its
        // tolerance is tol / sweep_rel with a safety factor, but never tighter than
        // inner_tol (what an FP32 solve reliably reaches) nor looser than one half.
        ctx->h_tol.resize(R);
        for (int g = 0; g < R; ++g) {
          if (!to_start[g]) continue;
          const double want = kSweepSafety * o.tol / std::max(ctx->sweep_rel[g], 1e-300);
          ctx->h_tol[g] = std::min(0.5, std::max(o.inner_tol, want));
        }
        CK(cudaMemcpyAsync(ctx->d_tol, ctx->h_tol.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
      }
      RC(upload_mask(ctx, 3, to_start));
      if (f32) RC(krylov_start<float2>(ctx, o, R, ctx->d_mask[3]));
      else RC(krylov_start<double2>(ctx, o, R, ctx->d_mask[3]));
      for (int g = 0; g < R; ++g) {
        if (!to_start[g]) continue;
        ctx->outer[g] += 1;  // sweeps started
        ctx->phase[g] = PH_INNER;
      }
    }
    if (any_done) {
      RC(upload_mask(ctx, 0, to_done));
      RC(compute_orders(ctx, ctx->d_mask[0], R));
      for (int g = 0; g < R; ++g)
        if (to_done[g]) ctx->phase[g] = PH_DONE;
    }
    ctx->enq_hi = 0;
    ctx->loop_ran = false;
  }
  int n = 0;
  for (int g = 0; g < ctx->max_rhs; ++g) n += ctx->phase[g] != PH_FREE && ctx->phase[g] != PH_DONE;
  *n_active = n;
  return PSFD_OK;
}

int engine_tick(psfd_ctx* ctx, const psfd_solve_opts& o, int* n_active) {
  bool pending = false;
  RC(engine_enqueue(ctx, o, &pending, nullptr));
  return engine_complete(ctx, o, n_active);
}

// ---------------------------------------------------------------------------------------
// The paper's outer fixed-point iteration (Sec. 3, Eqs. (8)-(9)), as an alternative to the
// folded operator. Outer step k solves the free-space problem
//     u_k - G*(V u_k) = b_k,   b_k = E_inc + R[E_inc + E_mask^(k-1)],   E_mask^(0) = 0,
// with the engine above (context flag no_reflect: K2 adds no reflection). With A the folded
// operator and M = I - G*V the free-space one, R[E_mask^(k-1)] on the absorber planes is
// (M - A) u_(k-1), so the next right-hand side is formed from two FP64 applications:
//     r = b_1 - A u_k  (the folded residual),   b_(k+1) = M u_k + r.
// r is also the stop test: b_1 - A u_k = (b_k - M u_k) + (R[E_mask^(k)] - R[E_mask^(k-1)]), the
// step's own residual plus the change of the reflected field, and the loop ends for a slot
// once ||r|| <= tol ||b_1||. Each step is solved to step_tol ||b_k|| from the previous
// step's field (warm start), so that the change of the reflected field dominates r.
// Slots run their outer steps together; a slot that has converged stops taking part.
// ---------------------------------------------------------------------------------------
namespace {

int run_engine(psfd_ctx* ctx, const psfd_solve_opts& o) {
  for (;;) {
    int active = 0;
    RC(engine_tick(ctx, o, &active));
    if (!active) return PSFD_OK;
  }
}

}  // namespace

int engine_fixed_point(psfd_ctx* ctx, const psfd_solve_opts& o, int max_steps, double step_tol) {
  const int R = ctx->n_rhs;
  const size_t U = ctx->plan.U;
  cudaStream_t st = ctx->stream;
  if (R <= 0) return PSFD_OK;
  if (!ctx->fp_b0) RC(ctx->dalloc(&ctx->fp_b0, (size_t)ctx->max_rhs * U));
  CK(cudaMemcpyAsync(ctx->fp_b0, ctx->b64, sizeof(double2) * U * R, cudaMemcpyDeviceToDevice, st));
  psfd_solve_opts os = o;
  os.tol = step_tol;
  std::vector<int> open(R, 1), steps(R, 0), total_iters(R, 0), status(R, PSFD_OK);
  std::vector<double> rel(R, 1.0);
  std::vector<std::vector<psfd_ctx::HistEntry>> hist(R);
  auto absorb_step = [&](int g) {  // bookkeeping after the engine solved one outer step
    for (const auto& h : ctx->hist[g])
      if (hist[g].size() < 100000) hist[g].push_back({total_iters[g] + h.iteration, h.kind, h.relres});
    total_iters[g] += ctx->iters[g];
    steps[g] += 1;
    if (ctx->status[g] != PSFD_OK) {
      status[g] = ctx->status[g];
      open[g] = 0;
    }
  };
  int rc = PSFD_OK;
  ctx->no_reflect = 1;
  // step 1: b_1 (from x = 0, or from the caller's initial guess)
  for (int g = 0; g < R; ++g) ctx->phase[g] = PH_NEW;
  rc = run_engine(ctx, os);
  for (int g = 0; rc == PSFD_OK && g < R; ++g) absorb_step(g);
  while (rc == PSFD_OK) {
    // r = b_1 - A u_k on the open slots (side spectra for the orders come with it)
    ctx->no_reflect = 0;
    if ((rc = upload_mask(ctx, 1, open)) != PSFD_OK) break;
    const int* mask = ctx->d_mask[1];
    if ((rc = launch_norm((int)U, std::max(1, std::min(ctx->plan.maxblk, (int)((U + 8191) / 8192))), 0, R, mask,
                          ctx->fp_b0, ctx->partials, ctx->plan.maxblk, 0, 0.0, ctx->sc64, ctx->act64, st)) != PSFD_OK)
      break;
    OpCall<double2> a = base_call64(ctx, 0, R);
    a.active = mask;
    a.u = ctx->x64;
    a.out = ctx->r64;
    a.b = ctx->fp_b0;
    a.epi = EPI_RESID;
    a.work = ctx->work64;
    a.dot_mask = DOT_OUT_OUT;
    a.side = ctx->side64;
    const int nb = resid_df(ctx) ? op_apply_df(a) : op_apply<double2>(a);
    if (nb < 0) {
      rc = nb;
      break;
    }
    if ((rc = launch_norm((int)U, nb, 0, R, mask, nullptr, ctx->partials, ctx->plan.maxblk, 1, 0.0, ctx->sc64,
                          ctx->act64, st)) != PSFD_OK)
      break;
    CK(cudaMemcpyAsync(ctx->h_sc64, ctx->sc64, sizeof(KScal) * R, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int n_open = 0;
    for (int g = 0; g < R; ++g) {
      if (!open[g]) continue;
      const KScal& s = ctx->h_sc64[g];
      rel[g] = std::sqrt(s.rnorm2 / s.bnorm2);
      if (hist[g].size() < 100000) hist[g].push_back({total_iters[g], 2, rel[g]});
      if (rel[g] <= o.tol) {
        open[g] = 0;
      } else if (!std::isfinite(rel[g])) {
        status[g] = PSFD_E_BREAKDOWN;
        open[g] = 0;
      } else if (steps[g] >= max_steps) {
        status[g] = PSFD_E_NOT_CONVERGED;
        open[g] = 0;
      }
      n_open += open[g];
    }
    if (!n_open) break;
    // b_(k+1) = M u_k + r for the slots that go on, then solve it from u_k
    ctx->no_reflect = 1;
    if ((rc = upload_mask(ctx, 1, open)) != PSFD_OK) break;
    OpCall<double2> m = base_call64(ctx, 0, R);
    m.active = ctx->d_mask[1];
    m.u = ctx->x64;
    m.out = ctx->b64;
    m.epi = EPI_AU;
    m.work = ctx->work64;
    const int nbm = op_apply<double2>(m);
    if (nbm < 0) {
      rc = nbm;
      break;
    }
    if ((rc = launch_vec_add((int)U, 0, R, ctx->d_mask[1], ctx->b64, ctx->r64, st)) != PSFD_OK) break;
    for (int g = 0; g < R; ++g) {
      if (!open[g]) continue;
      ctx->guess[g] = 1;
      ctx->phase[g] = PH_NEW;
    }
    if ((rc = run_engine(ctx, os)) != PSFD_OK) break;
    for (int g = 0; g < R; ++g)
      if (open[g]) absorb_step(g);
  }
  ctx->no_reflect = 0;
  if (rc != PSFD_OK) return rc;
  // the folded right-hand side back in place, and the orders of the last outer step
  CK(cudaMemcpyAsync(ctx->b64, ctx->fp_b0, sizeof(double2) * U * R, cudaMemcpyDeviceToDevice, st));
  std::vector<int> all(R, 1);
  RC(upload_mask(ctx, 0, all));
  RC(compute_orders(ctx, ctx->d_mask[0], R));
  for (int g = 0; g < R; ++g) {
    ctx->phase[g] = PH_DONE;
    ctx->relres[g] = rel[g];
    ctx->iters[g] = total_iters[g];
    ctx->outer[g] = steps[g];
    ctx->status[g] = status[g];
    ctx->hist[g] = hist[g];
  }
  return PSFD_OK;
}

}  // namespace psfd
