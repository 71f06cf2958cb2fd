// tune.cu -- the process-wide table of run-time tile shapes (RunTune) and the autotuner
// (psfd_autotune) that fills it by timing candidate shapes of the operator's passes on a
// context's own buffers.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ctx.h"
#include "op_launch.cuh"

namespace psfd {

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, RunTune> g_tune;
}  // namespace

RunTune run_tune(bool fp64, int nx, int ny, int nslab, int nf) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find({fp64, nx, ny, nslab, nf});
  return it == g_tune.end() ? RunTune{0, 0, 0, 0} : it->second;
}

bool has_run_tune(bool fp64, int nx, int ny, int nslab, int nf) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return g_tune.count({fp64, nx, ny, nslab, nf}) > 0;
}

void set_run_tune(bool fp64, int nx, int ny, int nslab, int nf, RunTune t) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[{fp64, nx, ny, nslab, nf}] = t;
}

void clear_run_tune() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
}

namespace {

// Candidate shapes of each tunable for a grid (the built-in choice among them).
template <typename C>
void candidates(const psfd_grid& g, std::vector<int>& zx, std::vector<int>& rb, std::vector<int>& cx,
                std::vector<int>& pf) {
  for (int t : {1, 2, 4, 8, 16})
    if (zcol_tile_ok<C>(g.nx, g.nf, t)) zx.push_back(t);
  if (use_half<C>(g.nx, g.ny))  // prefetch distances: a quarter to one wave of resident CTAs
    for (int d : {37, 74, 111, 148, 296}) pf.push_back(d);
  if (!use_fused<C>(g.nx, g.ny)) {
    for (int r = 1; r <= g.ny; r *= 2)
      if (rows_fwd_ok<C>(g.nx, g.ny, r)) rb.push_back(r);
    for (int t : {1, 2, 4, 8, 16, 32})
      if (cols_tile_ok<C>(g.nx, g.ny, t)) cx.push_back(t);
  }
}

// Mean time of `reps` applications of A (input stage plain, epilogue out = u - w) on all of the
// context's illuminations, after one untimed application.
template <typename C>
int time_apply(psfd_ctx* ctx, const OpCall<C>& a, int reps, cudaEvent_t e0, cudaEvent_t e1, double* ms) {
  int rc = op_apply<C>(a);
  if (rc < 0) return rc;
  CK(cudaEventRecord(e0, ctx->stream));
  for (int k = 0; k < reps; ++k)
    if ((rc = op_apply<C>(a)) < 0) return rc;
  CK(cudaEventRecord(e1, ctx->stream));
  CK(cudaEventSynchronize(e1));
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, e0, e1));
  *ms = (double)t / reps;
  return PSFD_OK;
}

template <typename C>
int autotune_impl(psfd_ctx* ctx, OpCall<C> a, psfd_tune_report* rep) {
  const psfd_grid& g = ctx->g;
  const bool fp64 = sizeof(C) == 16;
  std::vector<int> zx, rb, cx, pf;
  candidates<C>(g, zx, rb, cx, pf);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  constexpr int kReps = 3;
  RunTune best{0, 0, 0, 0};
  double t_best = 0.0, t_default = 0.0;
  int tried = 0, rc = PSFD_OK;
  auto measure = [&](RunTune t, double* ms) {
    set_run_tune(fp64, g.nx, g.ny, g.nslab, g.nf, t);
    ++tried;
    return time_apply<C>(ctx, a, kReps, e0, e1, ms);
  };
  rc = measure(best, &t_default);
  t_best = t_default;
  // one tunable at a time, each from the best shape found so far
  for (int which = 0; rc == PSFD_OK && which < 4; ++which) {
    const std::vector<int>& cand = which == 0 ? zx : (which == 1 ? rb : (which == 2 ? cx : pf));
    for (int v : cand) {
      RunTune t = best;
      (which == 0 ? t.zx : (which == 1 ? t.rb : (which == 2 ? t.cx : t.pf))) = v;
      double ms = 0.0;
      if ((rc = measure(t, &ms)) != PSFD_OK) break;
      if (ms < t_best) {
        t_best = ms;
        best = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_run_tune(fp64, g.nx, g.ny, g.nslab, g.nf, rc == PSFD_OK ? best : RunTune{0, 0, 0, 0});
  if (rc != PSFD_OK) return rc;
  if (rep) {
    rep->default_ms = t_default;
    rep->tuned_ms = t_best;
    rep->zx = best.zx;
    rep->rb = best.rb;
    rep->cx = best.cx;
    rep->pf = best.pf;
    rep->candidates = tried;
  }
  return PSFD_OK;
}

}  // namespace
}  // namespace psfd

using namespace psfd;

extern "C" int psfd_autotune(psfd_ctx* ctx, int force, psfd_tune_report* report) {
  if (!ctx) return PSFD_E_ARG;
  if (!ctx->have_illum || !ctx->have_potential)
    return ctx->fail(PSFD_E_STATE, "autotune before set_potential/illumination");
  const psfd_grid& g = ctx->g;
  const bool f32 = ctx->precision == PSFD_FP32_REFINED;
  if (!force && has_run_tune(!f32, g.nx, g.ny, g.nslab, g.nf)) {
    if (report) {
      const RunTune t = run_tune(!f32, g.nx, g.ny, g.nslab, g.nf);
      *report = psfd_tune_report{0.0, 0.0, t.zx, t.rb, t.cx, 0, t.pf};
    }
    return PSFD_OK;
  }
  // the timed applications read and write two Krylov pool vectors (scratch between solves)
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return ctx->cuda_fail(cudaGetLastError(), "autotune");
  const size_t bs = (size_t)ctx->max_rhs * ctx->plan.U;
  int rc;
  if (f32) {
    OpCall<float2> a = base_call32(ctx, 0, ctx->n_rhs);
    CK(cudaMemsetAsync(ctx->pool32, 0x3c, sizeof(float2) * bs, ctx->stream));
    a.u = ctx->pool32;
    a.out = ctx->pool32 + bs;
    a.work = ctx->work32;
    rc = autotune_impl<float2>(ctx, a, report);
  } else {
    OpCall<double2> a = base_call64(ctx, 0, ctx->n_rhs);
    CK(cudaMemsetAsync(ctx->pool64, 0x3f, sizeof(double2) * bs, ctx->stream));
    a.u = ctx->pool64;
    a.out = ctx->pool64 + bs;
    a.work = ctx->work64;
    rc = autotune_impl<double2>(ctx, a, report);
  }
  // graphs captured with the old shapes would replay them
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return ctx->cuda_fail(cudaGetLastError(), "autotune");
  ctx->drop_graphs();
  return rc;
}

extern "C" int psfd_tune_set(const psfd_grid* g, int precision, int zx, int rb, int cx, int pf) {
  if (!g || zx < 0 || rb < 0 || cx < 0 || pf < 0) return PSFD_E_ARG;
  if (precision != PSFD_FP64 && precision != PSFD_FP32_REFINED) return PSFD_E_ARG;
  const bool fp64 = precision == PSFD_FP64;
  const bool ok = fp64 ? ((!zx || zcol_tile_ok<double2>(g->nx, g->nf, zx)) &&
                          (!rb || rows_fwd_ok<double2>(g->nx, g->ny, rb)) &&
                          (!cx || cols_tile_ok<double2>(g->nx, g->ny, cx)))
                       : ((!zx || zcol_tile_ok<float2>(g->nx, g->nf, zx)) &&
                          (!rb || rows_fwd_ok<float2>(g->nx, g->ny, rb)) &&
                          (!cx || cols_tile_ok<float2>(g->nx, g->ny, cx)));
  if (!ok) return PSFD_E_ARG;
  set_run_tune(fp64, g->nx, g->ny, g->nslab, g->nf, RunTune{zx, rb, cx, pf});
  return PSFD_OK;
}

extern "C" int psfd_tune_reset(void) {
  clear_run_tune();
  return PSFD_OK;
}
