// engine.cu -- the solve engine: every illumination ("rhs slot") of a context moves
// through its own phases, and one tick advances all of them with shared launches.
//
//   PH_NEW    right-hand side just built: ||b|| is taken, x = 0, r = b
//   PH_START  start a Krylov solve: FP32 path -> r32 = r64 / ||r64||, BiCGStab init on r32;
//             FP64 path -> BiCGStab init on b
//   PH_INNER  BiCGStab iterating (check_every iterations per tick; the device flag of a slot
//             drops when its relative residual reaches the inner tolerance)
//   PH_RESID  FP64 residual r64 = b - A x64 (and the spectra for the orders); the FP32 path
//             stops when ||r64|| <= tol ||b|| or after max_outer sweeps, else starts again
//   PH_DONE   orders computed
//
// Slots in different phases coexist in one batch: every kernel takes a per-slot mask or
// activity flag, and all reductions are per slot and in a fixed order, so a slot's result
// does not depend on which other slots share the context or when they were admitted.
// One host synchronisation per tick reads the per-slot scalars.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.h"

namespace psfd {

OpCall<float2> base_call32(psfd_ctx* ctx, int rhs0, int nrhs);
OpCall<double2> base_call64(psfd_ctx* ctx, int rhs0, int nrhs);

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

template <typename C>
KrylovCall<C> krylov_of(psfd_ctx* ctx, const psfd_solve_opts& o);

template <>
KrylovCall<float2> krylov_of<float2>(psfd_ctx* ctx, const psfd_solve_opts& o) {
  KrylovCall<float2> k;
  std::memset(&k, 0, sizeof(k));
  k.op = base_call32(ctx, 0, ctx->max_rhs);
  k.n = (int)ctx->plan.U;
  // the scaled FP64 residual is both b and the running residual (init copies b into r)
  k.b = ctx->r32;
  k.r = ctx->r32;
  k.x = ctx->x32;
  k.r0 = ctx->r032;
  k.p = ctx->p32;
  k.v = ctx->v32;
  k.s = ctx->s32;
  k.t = ctx->t32;
  k.work = ctx->work32;
  k.sc = ctx->sc;
  k.act = ctx->act;
  k.h_act = ctx->h_act;
  k.tol = o.inner_tol;
  k.max_iter = o.max_iter;
  k.check_every = o.check_every;
  return k;
}

template <>
KrylovCall<double2> krylov_of<double2>(psfd_ctx* ctx, const psfd_solve_opts& o) {
  KrylovCall<double2> k;
  std::memset(&k, 0, sizeof(k));
  k.op = base_call64(ctx, 0, ctx->max_rhs);
  k.n = (int)ctx->plan.U;
  k.b = ctx->b64;
  k.x = ctx->x64;
  k.r = ctx->r64;
  k.r0 = ctx->k64[0];
  k.p = ctx->k64[1];
  k.v = ctx->k64[2];
  k.s = ctx->k64[3];
  k.t = ctx->k64[4];
  k.work = ctx->work64;
  k.sc = ctx->sc;
  k.act = ctx->act;
  k.h_act = ctx->h_act;
  k.tol = o.tol;
  k.max_iter = o.max_iter;
  k.check_every = o.check_every;
  return k;
}

// r64 = b - A x64 with the side spectra, then ||r64||^2 into sc64 / act64, for the slots in mask.
int fp64_residual(psfd_ctx* ctx, const int* mask, double tol) {
  OpCall<double2> a = base_call64(ctx, 0, ctx->max_rhs);
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
  RC(launch_norm((int)ctx->plan.U, nb, 0, ctx->max_rhs, mask, nullptr, ctx->partials, ctx->plan.maxblk, 1,
                 tol * tol, ctx->sc64, ctx->act64, ctx->stream));
  return PSFD_OK;
}

int compute_orders(psfd_ctx* ctx, const int* mask) {
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
  RC(launch_orders(o, ctx->max_rhs, ctx->stream));
  ctx->orders_on_host = false;
  return PSFD_OK;
}

}  // namespace

int engine_tick(psfd_ctx* ctx, const psfd_solve_opts& o, int* n_active) {
  const int R = ctx->max_rhs;
  const size_t U = ctx->plan.U;
  const bool f32 = ctx->precision == PSFD_FP32_REFINED;
  cudaStream_t st = ctx->stream;
  const int vblk = std::max(1, std::min(ctx->plan.maxblk, (int)((U + 8191) / 8192)));
  std::vector<int> sel(R);
  auto select = [&](int ph) {
    int n = 0;
    for (int g = 0; g < R; ++g) {
      sel[g] = ctx->phase[g] == ph;
      n += sel[g];
    }
    return n;
  };

  // ---- A: enqueue the work of every phase ------------------------------------------
  bool enqueued = false;
  if (select(PH_NEW)) {
    RC(upload_mask(ctx, 0, sel));
    RC(launch_norm((int)U, vblk, 0, R, ctx->d_mask[0], ctx->b64, ctx->partials, ctx->plan.maxblk, 0,
                   o.tol * o.tol, ctx->sc64, ctx->act64, st));
    for (int g = 0; g < R; ++g) {
      if (!sel[g]) continue;
      CK(cudaMemsetAsync(ctx->x64 + (size_t)g * U, 0, sizeof(double2) * U, st));
      CK(cudaMemcpyAsync(ctx->r64 + (size_t)g * U, ctx->b64 + (size_t)g * U, sizeof(double2) * U,
                         cudaMemcpyDeviceToDevice, st));
      CK(cudaMemsetAsync(ctx->side64 + (size_t)g * 6 * ctx->plan.plane, 0, sizeof(double2) * 6 * ctx->plan.plane,
                         st));
    }
    enqueued = true;
  }
  if (select(PH_RESID)) {
    RC(upload_mask(ctx, 1, sel));
    RC(fp64_residual(ctx, ctx->d_mask[1], o.tol));
    enqueued = true;
  }
  bool any_inner = false;
  for (int g = 0; g < R; ++g) any_inner = any_inner || ctx->phase[g] == PH_INNER;
  if (any_inner) {
    if (f32) RC(bicg_iterate<float2>(krylov_of<float2>(ctx, o), o.check_every));
    else RC(bicg_iterate<double2>(krylov_of<double2>(ctx, o), o.check_every));
    enqueued = true;
  }
  if (!enqueued) {
    int n = 0;
    for (int g = 0; g < R; ++g) n += ctx->phase[g] != PH_FREE && ctx->phase[g] != PH_DONE;
    *n_active = n;
    return PSFD_OK;
  }

  // ---- B: one synchronisation, read the per-slot scalars --------------------------
  CK(cudaMemcpyAsync(ctx->h_sc64, ctx->sc64, sizeof(KScal) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(KScal) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->h_act, ctx->act, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));

  // ---- C: transitions -------------------------------------------------------------
  std::vector<int> to_update(R, 0), to_start(R, 0), to_done(R, 0);
  const double tol2 = o.tol * o.tol;
  for (int g = 0; g < R; ++g) {
    const KScal& s64 = ctx->h_sc64[g];
    switch (ctx->phase[g]) {
      case PH_NEW:
        ctx->outer[g] = 0;
        ctx->iters[g] = 0;
        ctx->status[g] = PSFD_OK;
        if (!(s64.bnorm2 > 0.0)) {  // zero right-hand side: x = 0 is exact
          ctx->relres[g] = 0.0;
          to_done[g] = 1;
        } else {
          to_start[g] = 1;
        }
        break;
      case PH_RESID: {
        const double rel = std::sqrt(s64.rnorm2 / s64.bnorm2);
        ctx->relres[g] = rel;
        if (!f32) {
          if (!(s64.rnorm2 <= tol2 * s64.bnorm2) && ctx->status[g] == PSFD_OK) ctx->status[g] = PSFD_E_NOT_CONVERGED;
          to_done[g] = 1;
        } else if (s64.rnorm2 <= tol2 * s64.bnorm2) {
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
      case PH_INNER:
        if (!ctx->h_act[g]) {
          ctx->iters[g] += ctx->h_sc[g].iters;
          if (!f32 && ctx->h_sc[g].status != PSFD_OK) ctx->status[g] = ctx->h_sc[g].status;
          to_update[g] = 1;
        }
        break;
      default:
        break;
    }
  }

  // ---- D: enqueue sweep updates and starts -----------------------------------------
  bool any = false;
  for (int g = 0; g < R; ++g) any = any || to_update[g];
  if (any) {
    if (f32) {
      RC(upload_mask(ctx, 2, to_update));
      RC(launch_ref_update((int)U, 0, R, ctx->d_mask[2], ctx->sc64, ctx->x64, ctx->x32, st));
    }
    for (int g = 0; g < R; ++g)
      if (to_update[g]) ctx->phase[g] = PH_RESID;
  }
  any = false;
  for (int g = 0; g < R; ++g) any = any || to_start[g];
  if (any) {
    RC(upload_mask(ctx, 3, to_start));
    if (f32) {
      RC(launch_ref_scale((int)U, 0, R, ctx->d_mask[3], ctx->sc64, ctx->r64, ctx->r32, st));
      RC(bicg_start<float2>(krylov_of<float2>(ctx, o), ctx->d_mask[3]));
    } else {
      RC(bicg_start<double2>(krylov_of<double2>(ctx, o), ctx->d_mask[3]));
    }
    for (int g = 0; g < R; ++g) {
      if (!to_start[g]) continue;
      if (f32) ctx->outer[g] += 1;  // sweeps started
      ctx->phase[g] = PH_INNER;
    }
  }
  // ---- E: orders of the slots that finished ----------------------------------------
  any = false;
  for (int g = 0; g < R; ++g) any = any || to_done[g];
  if (any) {
    RC(upload_mask(ctx, 0, to_done));
    RC(compute_orders(ctx, ctx->d_mask[0]));
    for (int g = 0; g < R; ++g)
      if (to_done[g]) ctx->phase[g] = PH_DONE;
  }
  int n = 0;
  for (int g = 0; g < R; ++g) n += ctx->phase[g] != PH_FREE && ctx->phase[g] != PH_DONE;
  *n_active = n;
  return PSFD_OK;
}

}  // namespace psfd
