// psfd.cu -- the C ABI (include/psfd.h): solver context, device memory plan, set-up of
// potentials and illuminations, one-application entry point, read-back, and the launch
// accounting / event profiler. The solve itself is the engine in engine.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "ctx.h"
#include "dfloat.cuh"
#include "dfloat_ops.h"

using namespace psfd;

// ---------------------------------------------------------------------------
// launch accounting and the optional per-class event profiler
// ---------------------------------------------------------------------------
namespace psfd {
namespace {
std::atomic<unsigned long long> g_launches{0};
bool g_prof = false;
struct ProfRec {
  int cls;
  cudaEvent_t a, b;
  double bytes, flops, ctas;
  int counter;
};
std::vector<ProfRec> g_recs;
constexpr int kMaxCounters = 1 << 18;
unsigned* g_counters = nullptr;  // device, one per profiled launch
int g_next_counter = 0;
int g_open_counter[PK_N] = {};
std::vector<cudaEvent_t> g_pool;
cudaEvent_t g_open[PK_N] = {};
struct ProfTotal {
  unsigned long long launches = 0;
  double ms = 0, bytes = 0, flops = 0;
};
ProfTotal g_tot[PK_N];
const char* kProfNames[PK_N] = {"k1_plane_fwd_fp32", "k2_zcol_fp32", "k3_plane_inv_fp32",
                                "k1_plane_fwd_fp64", "k2_zcol_fp64", "k3_plane_inv_fp64",
                                "vec_fp32",          "vec_fp64",     "scalar",
                                "setup"};
cudaEvent_t take_event() {
  cudaEvent_t e = nullptr;
  if (!g_pool.empty()) {
    e = g_pool.back();
    g_pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  return e;
}
}  // namespace

void count_launch(int n) { g_launches += (unsigned long long)n; }
unsigned long long launch_total() { return g_launches.load(); }
bool prof_on() { return g_prof; }
unsigned* prof_begin(int cls, cudaStream_t st) {
  if (!g_prof || !g_counters || g_next_counter >= kMaxCounters) return nullptr;
  cudaEvent_t e = take_event();
  cudaEventRecord(e, st);
  g_open[cls] = e;
  g_open_counter[cls] = g_next_counter++;
  return g_counters + g_open_counter[cls];
}
void prof_end(int cls, cudaStream_t st, double bytes, double flops, double ctas) {
  if (!g_prof || !g_open[cls]) return;
  cudaEvent_t e = take_event();
  cudaEventRecord(e, st);
  g_recs.push_back({cls, g_open[cls], e, bytes, flops, ctas, g_open_counter[cls]});
  g_open[cls] = nullptr;
}

// ---------------------------------------------------------------------------
// plan, validation, tables
// ---------------------------------------------------------------------------
Plan make_plan(const psfd_grid& g, int precision, int max_rhs, int max_clips) {
  Plan p;
  p.plane = (size_t)g.nx * g.ny;
  p.U = 3 * (size_t)g.nslab * p.plane;
  p.maxblk = std::max(op_blocks_per_rhs(g.nx, g.ny, g.nslab, false), op_blocks_per_rhs(g.nx, g.ny, g.nslab, true));
  p.maxblk = std::max(p.maxblk, 1);
  const double k0 = 2.0 * kPi / g.wavelength;
  const double kb = k0 * std::sqrt(g.eps_bg);
  const double ax = kb * g.nx * g.dx / (2 * kPi), ay = kb * g.ny * g.dy / (2 * kPi);
  const double bound = (2.0 * ax + 3.0) * (2.0 * ay + 3.0);
  p.max_orders = (int)std::min<double>((double)p.plane, bound);
  const size_t R = (size_t)max_rhs, Cl = (size_t)max_clips;
  size_t b = 0;
  b += p.plane * g.nslab * (Cl * (16 + 8 + 16) + 16);        // V64, V32, V as pairs per clip, eps staging
  b += (size_t)(g.nx + g.ny + g.nf) * (16 + 8) + (size_t)(g.nx + g.ny) * 16;  // twiddles: FP64, FP32, x/y pairs
  b += R * (sizeof(RhsParam) + 4 * sizeof(double));          // illumination parameters
  b += R * p.plane * (sizeof(ModeEntry) + sizeof(ModeF32) + sizeof(ModeDF));  // mode tables (FP64, FP32, pairs)
  b += (size_t)g.nf * (3 * sizeof(float) + sizeof(double) + 16 + 8);  // kz tables, pair-format twiddles and kz
  b += R * p.U * 16 * 4;                                     // b64, x64, r64, work64
  b += R * 6 * p.plane * 16;                                 // side spectra
  const size_t kvec = precision == PSFD_FP64 ? 16 : 8;       // Krylov working precision
  b += R * p.U * kvec * (2 + kPoolBicg);                     // rs, xc, BiCGStab pool
  b += R * NDOT * (size_t)p.maxblk * 16;                     // partial sums
  b += R * (sizeof(GmState) + (size_t)(KMAX + 1) * p.maxblk * 16);  // GMRES state and partials
  b += R * (2 * sizeof(KScal) + 6 * sizeof(int) + sizeof(double));  // scalars, flags, masks, sweep tolerances
  b += R * (size_t)p.max_orders * (2 * sizeof(int) + 12 * sizeof(double)) + R * sizeof(int);
  p.bytes = b;
  return p;
}

bool grid_ok(const psfd_grid* g, std::string& why) {
  if (!g) { why = "grid is null"; return false; }
  if (!fft_length_supported(g->nx) || !fft_length_supported(g->ny)) { why = "unsupported nx or ny"; return false; }
  if (!fft_length_supported(g->nf)) { why = "unsupported nf"; return false; }
  if (g->nslab < 1) { why = "nslab must be >= 1"; return false; }
  if (g->nf < 2 * g->nslab + 2) { why = "nf must be >= 2*nslab + 2"; return false; }
  if (!(g->dx > 0 && g->dy > 0 && g->dz > 0 && g->wavelength > 0 && g->eps_bg > 0)) {
    why = "spacings, wavelength and eps_bg must be positive";
    return false;
  }
  return true;
}

static std::vector<double2> twiddles(int n) {
  std::vector<double2> t(n);
  for (int i = 0; i < n; ++i) {
    const double a = -2.0 * kPi * (double)i / (double)n;
    t[i] = make_double2(std::cos(a), std::sin(a));
  }
  return t;
}

int ctx_create(psfd_ctx** out, const psfd_grid* grid, int precision, int max_rhs, int max_clips,
               size_t hbm_budget, cudaStream_t stream) {
  if (!out) return PSFD_E_ARG;
  *out = nullptr;
  std::string why;
  if (!grid_ok(grid, why) || max_rhs < 1 || max_clips < 1 ||
      (precision != PSFD_FP64 && precision != PSFD_FP32_REFINED))
    return PSFD_E_ARG;
  psfd_ctx* ctx = new psfd_ctx();
  cudaGetDevice(&ctx->device);
  ctx->g = *grid;
  ctx->precision = precision;
  ctx->max_rhs = max_rhs;
  ctx->max_clips = max_clips;
  ctx->budget = hbm_budget;
  ctx->stream = stream;
  ctx->plan = make_plan(*grid, precision, max_rhs, max_clips);
  ctx->k0 = 2.0 * kPi / grid->wavelength;
  ctx->kb = ctx->k0 * std::sqrt(grid->eps_bg);
  ctx->L = 0.5 * grid->nf * grid->dz;
  if (hbm_budget && ctx->plan.bytes > hbm_budget) {
    delete ctx;
    return PSFD_E_BUDGET;
  }
  const Plan& P = ctx->plan;
  const size_t R = (size_t)max_rhs;
  int rc = PSFD_OK;
  auto A = [&](auto** p, size_t n) {
    if (rc == PSFD_OK) rc = ctx->dalloc(p, n);
  };
  A(&ctx->V64, P.plane * grid->nslab * max_clips);
  A(&ctx->V32, P.plane * grid->nslab * max_clips);
  A(&ctx->Vdf, P.plane * grid->nslab * max_clips);
  A(&ctx->eps_stage, P.plane * grid->nslab);
  A(&ctx->twx, grid->nx);
  A(&ctx->twy, grid->ny);
  A(&ctx->twz, grid->nf);
  A(&ctx->twx32, grid->nx);
  A(&ctx->twy32, grid->ny);
  A(&ctx->twz32, grid->nf);
  A(&ctx->twxdf, grid->nx);
  A(&ctx->twydf, grid->ny);
  A(&ctx->rhsp, R);
  A(&ctx->slot_par, 4 * R);
  A(&ctx->modes, R * P.plane);
  A(&ctx->modes32, R * P.plane);
  A(&ctx->modesdf, R * P.plane);
  A(&ctx->twzdf, grid->nf);
  A(&ctx->kzdf, grid->nf);
  A(&ctx->ktab32, 3 * (size_t)grid->nf);
  A(&ctx->ktab64, grid->nf);
  A(&ctx->d_eps_l, kStackMaxLayers);
  A(&ctx->d_d_l, kStackMaxLayers);
  A(&ctx->anomaly, 1);
  A(&ctx->b64, R * P.U);
  A(&ctx->x64, R * P.U);
  A(&ctx->r64, R * P.U);
  A(&ctx->work64, R * P.U);
  A(&ctx->side64, R * 6 * P.plane);
  if (precision == PSFD_FP64) {
    A(&ctx->rs64, R * P.U);
    A(&ctx->xc64, R * P.U);
    A(&ctx->pool64, R * P.U * kPoolBicg);
  } else {
    A(&ctx->x32, R * P.U);
    A(&ctx->r32, R * P.U);
    A(&ctx->pool32, R * P.U * kPoolBicg);
  }
  ctx->pool_vecs = kPoolBicg;
  ctx->work32 = reinterpret_cast<float2*>(ctx->work64);
  ctx->gblk = std::max(1, std::min(P.maxblk, (int)((P.U + 8191) / 8192)));
  A(&ctx->gm, R);
  A(&ctx->gpart, R * (size_t)(KMAX + 1) * ctx->gblk);
  A(&ctx->partials, R * NDOT * (size_t)P.maxblk);
  A(&ctx->sc, R);
  A(&ctx->sc64, R);
  A(&ctx->act, R);
  A(&ctx->act64, R);
  A(&ctx->d_tol, R);
  for (int i = 0; i < 4; ++i) A(&ctx->d_mask[i], R);
  A(&ctx->d_nord, R);
  A(&ctx->d_slots, R);
  A(&ctx->d_mn, R * (size_t)P.max_orders * 2);
  A(&ctx->d_ordout, R * (size_t)P.max_orders * 12);
  if (rc != PSFD_OK) {
    delete ctx;
    return rc;
  }
  if (cudaMallocHost(&ctx->h_act, sizeof(int) * R) != cudaSuccess ||
      cudaMallocHost(&ctx->h_act64, sizeof(int) * R) != cudaSuccess ||
      cudaMallocHost(&ctx->h_sc, sizeof(KScal) * R) != cudaSuccess ||
      cudaMallocHost(&ctx->h_sc64, sizeof(KScal) * R) != cudaSuccess ||
      cudaMallocHost(&ctx->h_mask, sizeof(int) * 4 * R) != cudaSuccess) {
    delete ctx;
    return PSFD_E_NOMEM;
  }
  ctx->h_rhsp.assign(R, RhsParam{});
  ctx->h_nord.assign(R, 0);
  ctx->h_mn.assign(R * (size_t)P.max_orders * 2, 0);
  ctx->th.assign(R, 0.0);
  ctx->ph.assign(R, 0.0);
  ctx->pol.assign(R, 0);
  ctx->clip.assign(R, 0);
  ctx->phase.assign(R, PH_FREE);
  ctx->guess.assign(R, 0);
  ctx->hist.assign(R, {});
  ctx->sweep_rel.assign(R, 1.0);
  ctx->outer.assign(R, 0);
  ctx->iters.assign(R, 0);
  ctx->status.assign(R, PSFD_OK);
  ctx->relres.assign(R, 0.0);
  auto tx = twiddles(grid->nx), ty = twiddles(grid->ny), tz = twiddles(grid->nf);
  cudaError_t e = cudaMemcpy(ctx->twx, tx.data(), tx.size() * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->twy, ty.data(), ty.size() * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->twz, tz.data(), tz.size() * 16, cudaMemcpyHostToDevice);
  {
    // FP32 copies for the FP32 kernels: each entry rounded to nearest, the value those kernels
    // would get by converting the FP64 entry themselves
    auto f32 = [](const std::vector<double2>& t) {
      std::vector<float2> r(t.size());
      for (size_t i = 0; i < t.size(); ++i) r[i] = make_float2((float)t[i].x, (float)t[i].y);
      return r;
    };
    const auto fx = f32(tx), fy = f32(ty), fz = f32(tz);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twx32, fx.data(), fx.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twy32, fy.data(), fy.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twz32, fz.data(), fz.size() * 8, cudaMemcpyHostToDevice);
    // pair copies of the x and y tables for the residual's double-float row and column passes
    auto df4 = [](const std::vector<double2>& t) {
      std::vector<float4> r(t.size());
      for (size_t i = 0; i < t.size(); ++i) {
        const dfc d = to_dfc(t[i]);
        r[i] = make_float4(d.x.hi, d.x.lo, d.y.hi, d.y.lo);
      }
      return r;
    };
    const auto dx4 = df4(tx), dy4 = df4(ty);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twxdf, dx4.data(), dx4.size() * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twydf, dy4.data(), dy4.size() * 16, cudaMemcpyHostToDevice);
  }
  {
    // signed z wavenumbers kz_l = 2 pi l / (nf dz), and |kz_l| split into FP32 hi + lo
    std::vector<float> k32(3 * (size_t)grid->nf);
    std::vector<double> k64(grid->nf);
    for (int l = 0; l < grid->nf; ++l) {
      const int lf = l < (grid->nf + 1) / 2 ? l : l - grid->nf;
      const double k = 2.0 * kPi * (double)lf / ((double)grid->nf * grid->dz);
      k64[l] = k;
      const float hi = (float)std::fabs(k);
      k32[l] = hi;
      k32[grid->nf + l] = (float)(std::fabs(k) - (double)hi);
      k32[2 * grid->nf + l] = (float)k;
    }
    if (e == cudaSuccess) e = cudaMemcpy(ctx->ktab32, k32.data(), sizeof(float) * k32.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->ktab64, k64.data(), sizeof(double) * k64.size(), cudaMemcpyHostToDevice);
    // pair-format copies for the double-float z pass (the host conversion gives the same
    // pairs as the device's integer-path conversion)
    std::vector<float4> tdf(grid->nf);
    std::vector<float2> kdf(grid->nf);
    for (int l = 0; l < grid->nf; ++l) {
      const dfc t = to_dfc(tz[l]);
      tdf[l] = make_float4(t.x.hi, t.x.lo, t.y.hi, t.y.lo);
      const dfr k = to_dfr(k64[l]);
      kdf[l] = make_float2(k.hi, k.lo);
    }
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twzdf, tdf.data(), sizeof(float4) * tdf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->kzdf, kdf.data(), sizeof(float2) * kdf.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(ctx->sc, 0, sizeof(KScal) * R);
  if (e == cudaSuccess) e = cudaMemset(ctx->sc64, 0, sizeof(KScal) * R);
  if (e == cudaSuccess) e = cudaMemset(ctx->act, 0, sizeof(int) * R);
  if (e == cudaSuccess) e = cudaMemset(ctx->act64, 0, sizeof(int) * R);
  if (e == cudaSuccess) e = cudaMemset(ctx->side64, 0, sizeof(double2) * R * 6 * P.plane);
  if (e != cudaSuccess) {
    delete ctx;
    return PSFD_E_CUDA;
  }
  *out = ctx;
  return PSFD_OK;
}

int ctx_set_potential(psfd_ctx* ctx, int clip, const double* eps_complex, int where) {
  if (!eps_complex || clip < 0 || clip >= ctx->max_clips || (where != PSFD_HOST && where != PSFD_DEVICE))
    return ctx->fail(PSFD_E_ARG, "invalid potential arguments");
  const size_t n = ctx->plan.plane * ctx->g.nslab;
  const double2* src = reinterpret_cast<const double2*>(eps_complex);
  if (where == PSFD_HOST) {
    CK(cudaMemcpyAsync(ctx->eps_stage, src, n * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    src = ctx->eps_stage;
  }
  RC(launch_potential(n, src, ctx->k0 * ctx->k0, ctx->g.eps_bg, ctx->V64 + (size_t)clip * n,
                      ctx->V32 + (size_t)clip * n, ctx->Vdf + (size_t)clip * n, ctx->stream));
  return PSFD_OK;
}

int ctx_set_rhs(psfd_ctx* ctx, int g0, int n, const double* theta_deg, const double* phi_deg, const int* pol,
                int clip, const StackHost& stack) {
  const psfd_grid& g = ctx->g;
  if (g0 < 0 || n < 1 || g0 + n > ctx->max_rhs || clip < 0 || clip >= ctx->max_clips ||
      (int)stack.eps.size() > kStackMaxLayers)
    return ctx->fail(PSFD_E_ARG, "invalid illumination slots");
  const int M = ctx->plan.max_orders;
  std::vector<double> spar(4 * (size_t)n);
  std::vector<int> slots;                  // the table rows this call computes
  std::vector<std::pair<int, int>> dups;   // (row, row it is copied from)
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(theta_deg[i]) || !std::isfinite(phi_deg[i]) || (pol[i] != 0 && pol[i] != 1))
      return ctx->fail(PSFD_E_ARG, "invalid angle or polarisation");
    const int gi = g0 + i;
    const double th = theta_deg[i] * kPi / 180.0, ph = phi_deg[i] * kPi / 180.0;
    RhsParam p{};
    p.qix = ctx->kb * std::sin(th) * std::cos(ph);
    p.qiy = ctx->kb * std::sin(th) * std::sin(ph);
    p.cphi = std::cos(ph);
    p.sphi = std::sin(ph);
    p.pol = pol[i];
    p.slot = gi;
    p.clip = clip;
    // The mode tables depend on the angles (and on the stack, common to the call), not on the
    // polarisation: a row whose angles an earlier illumination of this call has is copied
    // from that one's row instead of being computed again (the s and p illuminations of an
    // angle run the FP64 stack recursion once).
    int src = gi;
    for (int j = 0; j < i; ++j)
      if (theta_deg[j] == theta_deg[i] && phi_deg[j] == phi_deg[i]) {
        src = g0 + j;
        break;
      }
    if (src == gi) slots.push_back(gi);
    else dups.push_back({gi, src});
    // propagating orders (|q| < k_bg) and the anomaly check, in FFT order (y outer, x inner).
    // |beta| < 1e-9 k0 is tested as |d| < (1e-9 k0)^2; a row with qy^2 > k_bg^2 + (1e-9 k0)^2
    // holds only evanescent orders far from the anomaly and is skipped (host time here is GPU
    // idle time between solves)
    int cnt = 0;
    const double kb2 = ctx->kb * ctx->kb, an2 = (1e-9 * ctx->k0) * (1e-9 * ctx->k0);
    for (int y = 0; y < g.ny; ++y) {
      const int ni = y < (g.ny + 1) / 2 ? y : y - g.ny;
      const double qy = p.qiy + 2.0 * kPi * ni / (g.ny * g.dy);
      if (qy * qy > kb2 + an2) continue;
      for (int x = 0; x < g.nx; ++x) {
        const int mi = x < (g.nx + 1) / 2 ? x : x - g.nx;
        const double qx = p.qix + 2.0 * kPi * mi / (g.nx * g.dx);
        const double d = kb2 - (qx * qx + qy * qy);
        if (std::fabs(d) < an2)
          return ctx->fail(PSFD_E_ANOMALY, "order (" + std::to_string(mi) + ", " + std::to_string(ni) +
                                               ") of illumination " + std::to_string(gi) + " has beta = 0");
        if (d > 0) {
          if (cnt >= M) return ctx->fail(PSFD_E_ARG, "order capacity exceeded");
          ctx->h_mn[((size_t)gi * M + cnt) * 2] = mi;
          ctx->h_mn[((size_t)gi * M + cnt) * 2 + 1] = ni;
          ++cnt;
        }
      }
    }
    ctx->h_nord[gi] = cnt;
    ctx->h_rhsp[gi] = p;
    ctx->th[gi] = theta_deg[i];
    ctx->ph[gi] = phi_deg[i];
    ctx->pol[gi] = pol[i];
    ctx->clip[gi] = clip;
    spar[4 * i] = p.qix;
    spar[4 * i + 1] = p.qiy;
    spar[4 * i + 2] = p.cphi;
    spar[4 * i + 3] = p.sphi;
  }
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->slot_par + 4 * (size_t)g0, spar.data(), sizeof(double) * spar.size(),
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_nord + g0, ctx->h_nord.data() + g0, sizeof(int) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_mn + (size_t)g0 * M * 2, ctx->h_mn.data() + (size_t)g0 * M * 2,
                     sizeof(int) * (size_t)n * M * 2, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->rhsp + g0, ctx->h_rhsp.data() + g0, sizeof(RhsParam) * n, cudaMemcpyHostToDevice, st));
  ModesArgs m;
  m.slot0 = g0;
  m.nx = g.nx;
  m.ny = g.ny;
  m.dx = g.dx;
  m.dy = g.dy;
  m.dz = g.dz;
  m.k0 = ctx->k0;
  m.kb = ctx->kb;
  m.eps_bg = g.eps_bg;
  m.L = ctx->L;
  m.slot_par = ctx->slot_par;
  m.stack.n_layers = (int)stack.eps.size();
  m.stack.reflect = stack.set ? 1 : 0;
  m.stack.eps = ctx->d_eps_l;
  m.stack.d = ctx->d_d_l;
  m.stack.eps_sub = stack.eps_sub;
  stack_dedup(m.stack, stack.eps.data(), stack.d.data(), (int)stack.eps.size(), make_double2(g.eps_bg, 0.0),
              stack.eps_sub);
  if (m.stack.reflect && m.stack.n_mat == 0 && !stack.eps.empty()) {
    // general stacks go through device copies (stream order keeps each copy for its launch)
    CK(cudaMemcpyAsync(ctx->d_eps_l, stack.eps.data(), sizeof(double2) * stack.eps.size(), cudaMemcpyHostToDevice,
                       st));
    CK(cudaMemcpyAsync(ctx->d_d_l, stack.d.data(), sizeof(double) * stack.d.size(), cudaMemcpyHostToDevice, st));
  }
  m.modes = ctx->modes;
  m.modes32 = ctx->modes32;
  m.modesdf = ctx->modesdf;
  m.anomaly = ctx->anomaly;
  m.slots = ctx->d_slots;
  CK(cudaMemcpyAsync(ctx->d_slots, slots.data(), sizeof(int) * slots.size(), cudaMemcpyHostToDevice, st));
  RC(launch_modes(m, (int)slots.size(), st));
  const size_t pl = ctx->plan.plane;
  for (const auto& d : dups) {
    CK(cudaMemcpyAsync(ctx->modes + d.first * pl, ctx->modes + d.second * pl, sizeof(ModeEntry) * pl,
                       cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->modes32 + d.first * pl, ctx->modes32 + d.second * pl, sizeof(ModeF32) * pl,
                       cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->modesdf + d.first * pl, ctx->modesdf + d.second * pl, sizeof(ModeDF) * pl,
                       cudaMemcpyDeviceToDevice, st));
  }
  if (ctx->green == PSFD_GREEN_SPHERICAL) {
    SphArgs sa;
    sa.slot0 = g0;
    sa.nx = g.nx;
    sa.ny = g.ny;
    sa.nf = g.nf;
    sa.dx = g.dx;
    sa.dy = g.dy;
    sa.dz = g.dz;
    sa.kb = ctx->kb;
    sa.R = ctx->green_R;
    sa.slot_par = ctx->slot_par;
    sa.t64 = ctx->sph64;
    sa.t32 = ctx->sph32;
    RC(launch_sph_table(sa, n, st));
  }
  RC(launch_rhs(g0, n, ctx->rhsp, ctx->modes, g.nx, g.ny, g.nslab, g.dz, ctx->kb, ctx->b64 + (size_t)g0 * ctx->plan.U,
                st));
  for (int i = 0; i < n; ++i) {
    ctx->phase[g0 + i] = PH_NEW;
    ctx->guess[g0 + i] = 0;
    ctx->outer[g0 + i] = 0;
    ctx->iters[g0 + i] = 0;
    ctx->status[g0 + i] = PSFD_OK;
    ctx->relres[g0 + i] = 0.0;
  }
  ctx->orders_on_host = false;
  return PSFD_OK;
}

int ctx_orders_to_host(psfd_ctx* ctx) {
  const size_t M = (size_t)ctx->plan.max_orders;
  ctx->h_ordout.resize((size_t)ctx->max_rhs * M * 12);
  CK(cudaMemcpyAsync(ctx->h_ordout.data(), ctx->d_ordout, sizeof(double) * ctx->h_ordout.size(),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->orders_on_host = true;
  return PSFD_OK;
}

template <typename C>
static OpCall<C> base_call(psfd_ctx* ctx, int rhs0, int nrhs, const C* V) {
  OpCall<C> a;
  std::memset(&a, 0, sizeof(a));
  a.nx = ctx->g.nx;
  a.ny = ctx->g.ny;
  a.nslab = ctx->g.nslab;
  a.nf = ctx->g.nf;
  a.rhs0 = rhs0;
  a.nrhs = nrhs;
  a.dx = ctx->g.dx;
  a.dy = ctx->g.dy;
  a.dz = ctx->g.dz;
  a.kb = ctx->kb;
  a.dz32 = (float)ctx->g.dz;
  a.kb32 = (float)ctx->kb;
  a.V = V;
  a.twx = ctx->twx;
  a.twy = ctx->twy;
  a.twz = ctx->twz;
  a.twx32 = ctx->twx32;
  a.twy32 = ctx->twy32;
  a.twz32 = ctx->twz32;
  a.rhsp = ctx->rhsp;
  a.modes = ctx->modes;
  a.modes32 = ctx->modes32;
  a.modesdf = ctx->modesdf;
  a.twzdf = ctx->twzdf;
  a.kzdf = ctx->kzdf;
  a.twxdf = ctx->twxdf;
  a.twydf = ctx->twydf;
  a.Vdf = (const void*)V == (const void*)ctx->V64 ? ctx->Vdf : nullptr;
  {
    // the double-float z pass's constants, formed in FP64 and split once here
    auto r2 = [](double v) {
      const dfr d = to_dfr(v);
      return make_float2(d.hi, d.lo);
    };
    const psfd_grid& g = ctx->g;
    a.dfL = r2(0.5 * (double)g.nf * g.dz);
    a.dfcinv = r2(1.0 / (ctx->kb * ctx->kb));
    a.dfscale = r2(1.0 / ((double)g.nf * (double)g.nx * (double)g.ny));
  }
  a.ktab32 = ctx->ktab32;
  a.ktab64 = ctx->ktab64;
  a.partials = ctx->partials;
  a.maxblk = ctx->plan.maxblk;
  a.stream = ctx->stream;
  a.in_mode = IN_PLAIN;
  a.epi = EPI_AU;
  a.no_reflect = ctx->no_reflect || ctx->green == PSFD_GREEN_SPHERICAL;
  if (ctx->green == PSFD_GREEN_SPHERICAL) {
    a.sph64 = ctx->sph64;
    a.sph32 = ctx->sph32;
  }
  return a;
}
template OpCall<float2> base_call<float2>(psfd_ctx*, int, int, const float2*);
template OpCall<double2> base_call<double2>(psfd_ctx*, int, int, const double2*);

OpCall<float2> base_call32(psfd_ctx* ctx, int rhs0, int nrhs) { return base_call<float2>(ctx, rhs0, nrhs, ctx->V32); }
OpCall<double2> base_call64(psfd_ctx* ctx, int rhs0, int nrhs) {
  return base_call<double2>(ctx, rhs0, nrhs, ctx->V64);
}

static int pool_need(const psfd_solve_opts& o) {
  if (o.krylov != PSFD_GMRES) return kPoolBicg;
  const int m = (o.restart > 0 && o.restart < KMAX) ? o.restart : KMAX;
  return std::max(kPoolBicg, m + 3);
}

size_t pool_extra_bytes(const Plan& p, int precision, int max_rhs, const psfd_solve_opts& o) {
  const size_t kvec = precision == PSFD_FP64 ? 16 : 8;
  return (size_t)max_rhs * p.U * kvec * (size_t)(pool_need(o) - kPoolBicg);
}

// Grow the Krylov pool to what the requested method needs (GMRES(m): m + 3 vectors). Runs
// before any work of the solve is enqueued; waits for the context's stream first.
int ensure_pool(psfd_ctx* ctx, const psfd_solve_opts& o) {
  const int need = pool_need(o);
  if (need <= ctx->pool_vecs) return PSFD_OK;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return ctx->cuda_fail(cudaGetLastError(), "pool resize");
  ctx->drop_graphs();  // they hold the old pool's addresses
  const size_t n = (size_t)ctx->max_rhs * ctx->plan.U * need;
  if (ctx->precision == PSFD_FP64) {
    ctx->dfree(ctx->pool64);
    ctx->pool64 = nullptr;
    RC(ctx->dalloc(&ctx->pool64, n));
  } else {
    ctx->dfree(ctx->pool32);
    ctx->pool32 = nullptr;
    RC(ctx->dalloc(&ctx->pool32, n));
  }
  ctx->pool_vecs = need;
  return PSFD_OK;
}

}  // namespace psfd

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* psfd_strerror(int s) {
  switch (s) {
    case PSFD_OK: return "ok";
    case PSFD_E_ARG: return "invalid argument";
    case PSFD_E_NOMEM: return "device allocation failed";
    case PSFD_E_BUDGET: return "HBM budget exceeded";
    case PSFD_E_CUDA: return "CUDA error";
    case PSFD_E_NOT_CONVERGED: return "not converged";
    case PSFD_E_BREAKDOWN: return "Krylov breakdown";
    case PSFD_E_ANOMALY: return "Rayleigh anomaly (a diffraction order has beta = 0)";
    case PSFD_E_TIMEOUT: return "device wait timed out";
    case PSFD_E_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* psfd_last_error(const psfd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int psfd_supported_length(int n) { return fft_length_supported(n) ? 1 : 0; }

int psfd_workspace_bytes(const psfd_grid* grid, int precision, int max_rhs, size_t* bytes) {
  std::string why;
  if (!bytes || !grid_ok(grid, why) || max_rhs < 1 || (precision != PSFD_FP64 && precision != PSFD_FP32_REFINED))
    return PSFD_E_ARG;
  *bytes = make_plan(*grid, precision, max_rhs, 1).bytes;
  return PSFD_OK;
}

int psfd_create(psfd_ctx** out, const psfd_grid* grid, int precision, int max_rhs, size_t hbm_budget,
                void* stream) {
  return ctx_create(out, grid, precision, max_rhs, 1, hbm_budget, (cudaStream_t)stream);
}

int psfd_destroy(psfd_ctx* ctx) {
  if (!ctx) return PSFD_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  delete ctx;
  return PSFD_OK;
}

int psfd_set_stream(psfd_ctx* ctx, void* stream) {
  if (!ctx) return PSFD_E_ARG;
  ctx->stream = (cudaStream_t)stream;
  return PSFD_OK;
}

int psfd_set_green(psfd_ctx* ctx, int kind, double R) {
  if (!ctx) return PSFD_E_ARG;
  if (kind == PSFD_GREEN_PERIODIC) {
    ctx->green = kind;
    ctx->have_illum = false;
    return PSFD_OK;
  }
  if (kind != PSFD_GREEN_SPHERICAL) return ctx->fail(PSFD_E_ARG, "unknown Green's function kind");
  const psfd_grid& g = ctx->g;
  if (!(R > 0.0) || R > g.nx * g.dx || R > g.ny * g.dy || g.nslab * g.dz + R > g.nf * g.dz)
    return ctx->fail(PSFD_E_ARG, "window radius must be positive, within the transverse periods, and nf dz >= nslab dz + R");
  if (!ctx->sph64) {
    const size_t n = (size_t)ctx->max_rhs * (g.nf / 2 + 1) * ctx->plan.plane;
    RC(ctx->dalloc(&ctx->sph64, 2 * n));
    if (ctx->precision == PSFD_FP32_REFINED) RC(ctx->dalloc(&ctx->sph32, n));
  }
  ctx->green = kind;
  ctx->green_R = R;
  ctx->have_illum = false;  // the tables are built with the illuminations
  return PSFD_OK;
}

int psfd_set_graphs(psfd_ctx* ctx, int enable) {
  if (!ctx) return PSFD_E_ARG;
  if (!enable) {
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return ctx->cuda_fail(cudaGetLastError(), "set_graphs");
    ctx->drop_graphs();
  }
  ctx->use_graphs = enable != 0;
  return PSFD_OK;
}

int psfd_set_device_loop(psfd_ctx* ctx, int enable) {
  if (!ctx) return PSFD_E_ARG;
  ctx->device_loop = enable != 0;
  return PSFD_OK;
}

int psfd_set_residual_arith(psfd_ctx* ctx, int kind) {
  if (!ctx) return PSFD_E_ARG;
  if (kind != PSFD_RESID_FP64 && kind != PSFD_RESID_DFLOAT) return ctx->fail(PSFD_E_ARG, "unknown residual arithmetic");
  ctx->resid_arith = kind;
  return PSFD_OK;
}

int psfd_set_stack(psfd_ctx* ctx, int n_layers, const double* n_complex, const double* thickness_nm,
                   const double* n_sub) {
  if (!ctx) return PSFD_E_ARG;
  if (n_layers < 0 || n_layers > kStackMaxLayers || !n_sub || (n_layers > 0 && (!n_complex || !thickness_nm)))
    return ctx->fail(PSFD_E_ARG, "invalid stack arguments");
  StackHost s;
  s.eps.resize(n_layers);
  s.d.resize(n_layers);
  for (int j = 0; j < n_layers; ++j) {
    const double a = n_complex[2 * j], b = n_complex[2 * j + 1];
    if (!(thickness_nm[j] >= 0.0)) return ctx->fail(PSFD_E_ARG, "negative layer thickness");
    s.eps[j] = make_double2(a * a - b * b, 2.0 * a * b);
    s.d[j] = thickness_nm[j];
  }
  s.eps_sub = make_double2(n_sub[0] * n_sub[0] - n_sub[1] * n_sub[1], 2.0 * n_sub[0] * n_sub[1]);
  s.set = true;
  ctx->stack = s;
  if (ctx->have_illum)
    return ctx_set_rhs(ctx, 0, ctx->n_rhs, ctx->th.data(), ctx->ph.data(), ctx->pol.data(), 0, ctx->stack);
  return PSFD_OK;
}

int psfd_set_potential(psfd_ctx* ctx, const double* eps_complex, int where) {
  if (!ctx) return PSFD_E_ARG;
  RC(ctx_set_potential(ctx, 0, eps_complex, where));
  ctx->have_potential = true;
  for (int i = 0; i < ctx->n_rhs; ++i)
    if (ctx->phase[i] != PH_FREE) ctx->phase[i] = PH_NEW;
  return PSFD_OK;
}

int psfd_set_illumination(psfd_ctx* ctx, int n_rhs, const double* theta_deg, const double* phi_deg,
                          const int* pol) {
  if (!ctx) return PSFD_E_ARG;
  if (n_rhs < 1 || n_rhs > ctx->max_rhs || !theta_deg || !phi_deg || !pol)
    return ctx->fail(PSFD_E_ARG, "invalid illumination arguments");
  for (int i = 0; i < ctx->max_rhs; ++i) ctx->phase[i] = PH_FREE;
  RC(ctx_set_rhs(ctx, 0, n_rhs, theta_deg, phi_deg, pol, 0, ctx->stack));
  ctx->n_rhs = n_rhs;
  ctx->have_illum = true;
  return PSFD_OK;
}

int psfd_apply(psfd_ctx* ctx, int precision, int rhs0, int n_rhs, const void* u, void* out) {
  if (!ctx) return PSFD_E_ARG;
  if (!ctx->have_illum || !ctx->have_potential) return ctx->fail(PSFD_E_STATE, "apply before set_potential/illumination");
  if (!u || !out || rhs0 < 0 || n_rhs < 1 || rhs0 + n_rhs > ctx->n_rhs)
    return ctx->fail(PSFD_E_ARG, "invalid apply arguments");
  if (precision == PSFD_FP64 || precision == PSFD_FP64_DF) {
    OpCall<double2> a = base_call64(ctx, rhs0, n_rhs);
    a.u = (const double2*)u;
    a.out = (double2*)out;
    a.work = ctx->work64;
    RC(precision == PSFD_FP64 ? op_apply<double2>(a) : op_apply_df(a));
  } else if (precision == PSFD_FP32_REFINED) {
    OpCall<float2> a = base_call32(ctx, rhs0, n_rhs);
    a.u = (const float2*)u;
    a.out = (float2*)out;
    a.work = ctx->work32;
    RC(op_apply<float2>(a));
  } else {
    return ctx->fail(PSFD_E_ARG, "unknown precision");
  }
  return PSFD_OK;
}

// Worst status, iteration count and residual over the single-clip slots, into report.
static int report_slots(psfd_ctx* ctx, std::chrono::steady_clock::time_point t0, psfd_report* report) {
  int status = PSFD_OK, iters = 0, outer = 0;
  double relres = 0.0;
  for (int i = 0; i < ctx->n_rhs; ++i) {
    iters = std::max(iters, ctx->iters[i]);
    outer = std::max(outer, ctx->outer[i]);
    relres = std::max(relres, ctx->relres[i]);
    if (ctx->status[i] != PSFD_OK && status == PSFD_OK) status = ctx->status[i];
  }
  if (report) {
    report->iterations = iters;
    report->outer = outer;
    report->relres = relres;
    report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    report->status = status;
  }
  if (status != PSFD_OK) ctx->err = psfd_strerror(status);
  return status;
}

int psfd_solve(psfd_ctx* ctx, const psfd_solve_opts* opts, psfd_report* report) {
  if (!ctx) return PSFD_E_ARG;
  if (!ctx->have_illum || !ctx->have_potential) return ctx->fail(PSFD_E_STATE, "solve before set_potential/illumination");
  const auto t0 = std::chrono::steady_clock::now();
  const psfd_solve_opts o = solve_defaults(opts);
  RC(ensure_pool(ctx, o));
  for (int i = 0; i < ctx->n_rhs; ++i)
    if (ctx->phase[i] == PH_DONE) ctx->phase[i] = PH_NEW;  // re-solve from scratch
  for (;;) {
    int active = 0;
    RC(engine_tick(ctx, o, &active));
    if (!active) break;
  }
  return report_slots(ctx, t0, report);
}

int psfd_solve_group(psfd_ctx* const* ctxs, int n, const psfd_solve_opts* opts, psfd_report* reports) {
  if (!ctxs || n < 1) return PSFD_E_ARG;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return PSFD_E_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return PSFD_E_ARG;
  }
  // one host thread per context beyond the first: each drives its own context's engine on its
  // own stream, so the contexts' kernels run side by side on the device
  std::vector<int> st(n, PSFD_OK);
  std::vector<std::thread> th;
  th.reserve(n - 1);
  for (int i = 1; i < n; ++i)
    th.emplace_back([&, i] {
      if (cudaSetDevice(ctxs[i]->device) != cudaSuccess) {
        st[i] = PSFD_E_CUDA;
        return;
      }
      st[i] = psfd_solve(ctxs[i], opts, reports ? reports + i : nullptr);
    });
  st[0] = psfd_solve(ctxs[0], opts, reports);
  for (auto& t : th) t.join();
  for (int s : st)
    if (s != PSFD_OK) return s;
  return PSFD_OK;
}

int psfd_solve_fixed_point(psfd_ctx* ctx, const psfd_solve_opts* opts, int max_steps, double step_tol,
                           psfd_report* report) {
  if (!ctx) return PSFD_E_ARG;
  if (!ctx->have_illum || !ctx->have_potential)
    return ctx->fail(PSFD_E_STATE, "solve_fixed_point before set_potential/illumination");
  if (!(step_tol >= 0.0) || step_tol >= 1.0) return ctx->fail(PSFD_E_ARG, "step_tol must lie in [0, 1)");
  const auto t0 = std::chrono::steady_clock::now();
  const psfd_solve_opts o = solve_defaults(opts);
  if (max_steps <= 0) max_steps = 50;
  if (step_tol == 0.0) step_tol = 0.1 * o.tol;
  RC(ensure_pool(ctx, o));
  RC(engine_fixed_point(ctx, o, max_steps, step_tol));
  return report_slots(ctx, t0, report);
}

int psfd_num_orders(psfd_ctx* ctx, int rhs, int* n_orders) {
  if (!ctx || !n_orders || !ctx->have_illum || rhs < 0 || rhs >= ctx->n_rhs) return PSFD_E_ARG;
  *n_orders = ctx->h_nord[rhs];
  return PSFD_OK;
}

int psfd_diffraction_orders(psfd_ctx* ctx, int rhs, int capacity, int* n_orders, int* mn, double* amp, double* sp,
                            double* eff) {
  if (!ctx || !n_orders || !mn) return PSFD_E_ARG;
  if (rhs < 0 || rhs >= ctx->n_rhs) return ctx->fail(PSFD_E_ARG, "rhs out of range");
  if (ctx->phase[rhs] != PH_DONE) return ctx->fail(PSFD_E_STATE, "diffraction_orders before solve");
  const int n = ctx->h_nord[rhs];
  *n_orders = n;
  if (capacity < n) return ctx->fail(PSFD_E_ARG, "capacity smaller than the number of orders");
  if (!ctx->orders_on_host) RC(ctx_orders_to_host(ctx));
  const size_t M = (size_t)ctx->plan.max_orders;
  for (int k = 0; k < n; ++k) {
    const double* o = ctx->h_ordout.data() + ((size_t)rhs * M + k) * 12;
    mn[2 * k] = ctx->h_mn[((size_t)rhs * M + k) * 2];
    mn[2 * k + 1] = ctx->h_mn[((size_t)rhs * M + k) * 2 + 1];
    if (amp) std::memcpy(amp + 6 * k, o, 6 * sizeof(double));
    if (sp) std::memcpy(sp + 4 * k, o + 6, 4 * sizeof(double));
    if (eff) eff[k] = o[10];
  }
  return PSFD_OK;
}

static int copy_vec(psfd_ctx* ctx, const double2* src, double* dst, int where) {
  const size_t bytes = sizeof(double2) * ctx->plan.U;
  CK(cudaMemcpyAsync(dst, src, bytes, where == PSFD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return PSFD_OK;
}

int psfd_get_solution(psfd_ctx* ctx, int rhs, double* dst, int where) {
  if (!ctx || !dst || rhs < 0 || rhs >= ctx->n_rhs || (where != PSFD_HOST && where != PSFD_DEVICE)) return PSFD_E_ARG;
  if (ctx->phase[rhs] != PH_DONE) return ctx->fail(PSFD_E_STATE, "get_solution before solve");
  return copy_vec(ctx, ctx->x64 + (size_t)rhs * ctx->plan.U, dst, where);
}

int psfd_set_initial_guess(psfd_ctx* ctx, int rhs, const double* x, int where) {
  if (!ctx || !x || (where != PSFD_HOST && where != PSFD_DEVICE)) return PSFD_E_ARG;
  if (!ctx->have_illum || rhs < 0 || rhs >= ctx->n_rhs) return ctx->fail(PSFD_E_ARG, "rhs out of range");
  const size_t bytes = sizeof(double2) * ctx->plan.U;
  CK(cudaMemcpyAsync(ctx->x64 + (size_t)rhs * ctx->plan.U, x, bytes,
                     where == PSFD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->guess[rhs] = 1;
  ctx->phase[rhs] = PH_NEW;
  return PSFD_OK;
}

int psfd_residual_history(psfd_ctx* ctx, int rhs, int capacity, int* n, int* iteration, int* kind, double* relres) {
  if (!ctx || !n || rhs < 0 || rhs >= ctx->max_rhs || capacity < 0) return PSFD_E_ARG;
  const auto& h = ctx->hist[rhs];
  *n = (int)h.size();
  const int m = std::min(capacity, (int)h.size());
  if (m > 0 && (!iteration || !kind || !relres)) return PSFD_E_ARG;
  for (int k = 0; k < m; ++k) {
    iteration[k] = h[k].iteration;
    kind[k] = h[k].kind;
    relres[k] = h[k].relres;
  }
  return PSFD_OK;
}

int psfd_get_rhs(psfd_ctx* ctx, int rhs, double* dst, int where) {
  if (!ctx || !dst || rhs < 0 || rhs >= ctx->n_rhs || (where != PSFD_HOST && where != PSFD_DEVICE)) return PSFD_E_ARG;
  return copy_vec(ctx, ctx->b64 + (size_t)rhs * ctx->plan.U, dst, where);
}

int psfd_get_mode_tables(psfd_ctx* ctx, int rhs, double* beta, double* r_s, double* r_p) {
  if (!ctx || rhs < 0 || rhs >= ctx->n_rhs || !ctx->have_illum) return PSFD_E_ARG;
  const size_t plane = ctx->plan.plane;
  std::vector<ModeEntry> m(plane);
  CK(cudaMemcpyAsync(m.data(), ctx->modes + (size_t)ctx->h_rhsp[rhs].slot * plane, sizeof(ModeEntry) * plane,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (size_t i = 0; i < plane; ++i) {
    if (beta) { beta[2 * i] = m[i].beta.x; beta[2 * i + 1] = m[i].beta.y; }
    if (r_s) { r_s[2 * i] = m[i].rs.x; r_s[2 * i + 1] = m[i].rs.y; }
    if (r_p) { r_p[2 * i] = m[i].rp.x; r_p[2 * i + 1] = m[i].rp.y; }
  }
  return PSFD_OK;
}

int psfd_launch_count(unsigned long long* count) {
  if (!count) return PSFD_E_ARG;
  *count = g_launches.load();
  return PSFD_OK;
}

int psfd_profile_enable(int on) {
  if (on) {
    for (auto& r : g_recs) {
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    }
    g_recs.clear();
    for (auto& t : g_tot) t = ProfTotal{};
    if (!g_counters && cudaMalloc(&g_counters, sizeof(unsigned) * kMaxCounters) != cudaSuccess) {
      g_counters = nullptr;
      return PSFD_E_NOMEM;
    }
    if (cudaMemset(g_counters, 0, sizeof(unsigned) * kMaxCounters) != cudaSuccess) return PSFD_E_CUDA;
    g_next_counter = 0;
    g_prof = true;
  } else {
    g_prof = false;
  }
  return PSFD_OK;
}

int psfd_profile_classes(void) { return PK_N; }

int psfd_profile_get(int cls, const char** name, unsigned long long* launches, double* ms, double* bytes,
                     double* flops) {
  if (cls < 0 || cls >= PK_N) return PSFD_E_ARG;
  if (!g_recs.empty()) {  // fold finished records into the totals
    std::vector<unsigned> cnt(g_next_counter > 0 ? g_next_counter : 1, 0u);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(cnt.data(), g_counters, sizeof(unsigned) * cnt.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      return PSFD_E_CUDA;
    for (auto& r : g_recs) {
      if (cudaEventSynchronize(r.b) != cudaSuccess) return PSFD_E_CUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, r.a, r.b);
      ProfTotal& T = g_tot[r.cls];
      const double frac = r.ctas > 0 ? (double)cnt[r.counter] / r.ctas : 1.0;  // share of CTAs that worked
      T.launches += 1;
      T.ms += t;
      T.bytes += r.bytes * frac;
      T.flops += r.flops * frac;
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    }
    g_recs.clear();
  }
  if (name) *name = kProfNames[cls];
  if (launches) *launches = g_tot[cls].launches;
  if (ms) *ms = g_tot[cls].ms;
  if (bytes) *bytes = g_tot[cls].bytes;
  if (flops) *flops = g_tot[cls].flops;
  return PSFD_OK;
}

int psfd_test_fft(int n, int count, int inverse, int fp64, void* data) {
  if (!data || count < 1 || !fft_length_supported(n)) return PSFD_E_ARG;
  auto t = twiddles(n);
  double2* tw = nullptr;
  if (cudaMalloc(&tw, sizeof(double2) * n) != cudaSuccess) return PSFD_E_NOMEM;
  int rc = PSFD_OK;
  if (cudaMemcpy(tw, t.data(), sizeof(double2) * n, cudaMemcpyHostToDevice) != cudaSuccess) rc = PSFD_E_CUDA;
  if (rc == PSFD_OK) rc = launch_test_fft(n, count, inverse != 0, fp64 != 0, data, tw);
  if (rc == PSFD_OK && cudaDeviceSynchronize() != cudaSuccess) rc = PSFD_E_CUDA;
  cudaFree(tw);
  return rc;
}

}  // extern "C"
