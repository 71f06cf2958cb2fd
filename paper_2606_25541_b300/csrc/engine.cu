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
#include <cstring>
#include <vector>

#include "ctx.h"

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
  const int nb = op_apply<double2>(a);
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

int engine_enqueue(psfd_ctx* ctx, const psfd_solve_opts& o, bool* pending) {
  const int R = busy_hi(ctx);
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
  if (select(PH_INNER)) {
    if (f32) RC(krylov_iterate<float2>(ctx, o, R));
    else RC(krylov_iterate<double2>(ctx, o, R));
    *pending = true;
  }
  if (*pending) {  // read-back of the per-slot scalars, waited for in engine_complete
    CK(cudaMemcpyAsync(ctx->h_sc64, ctx->sc64, sizeof(KScal) * R, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(KScal) * R, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ctx->h_act, ctx->act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  }
  return PSFD_OK;
}

int engine_complete(psfd_ctx* ctx, const psfd_solve_opts& o, int* n_active) {
  const int R = ctx->enq_hi;
  const size_t U = ctx->plan.U;
  const bool f32 = ctx->precision == PSFD_FP32_REFINED;
  cudaStream_t st = ctx->stream;
  if (R > 0) {
    CK(cudaStreamSynchronize(st));
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
          if (o.krylov != PSFD_GMRES && si.bnorm2 > 0.0 && si.iters > 0)
            record(g, ctx->iters[g] + si.iters, 0, std::sqrt(si.rnorm2 / si.bnorm2) * ctx->sweep_rel[g]);
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
  }
  int n = 0;
  for (int g = 0; g < ctx->max_rhs; ++g) n += ctx->phase[g] != PH_FREE && ctx->phase[g] != PH_DONE;
  *n_active = n;
  return PSFD_OK;
}

int engine_tick(psfd_ctx* ctx, const psfd_solve_opts& o, int* n_active) {
  bool pending = false;
  RC(engine_enqueue(ctx, o, &pending));
  return engine_complete(ctx, o, n_active);
}

}  // namespace psfd
