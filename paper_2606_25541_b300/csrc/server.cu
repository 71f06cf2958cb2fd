// server.cu -- the serving loop: continuous batching of mask-clip solves.
//
// Requests (a clip: grid, stack, permittivity, 1..n illuminations) are queued on
// submit. Each progress() call
//   1. admits queued requests, in arrival order, into a context ("bucket") of the same
//      grid: a free potential slot and a run of free illumination slots are claimed, the
//      potential and the per-mode tables are built, and the slots enter the engine
//      (engine.cu) -- while other requests of the bucket are mid-solve. A bucket is created
//      when the request's grid has none and its device footprint fits the HBM budget;
//      idle buckets are released when a queued request needs their memory;
//   2. advances every bucket by one engine tick (shared launches over all its slots);
//   3. retires requests whose illuminations are all done: their orders are copied to
//      host memory, their slots freed for the next admissions.
// A request's result does not depend on the other requests of its bucket: every kernel
// masks per slot and every reduction is per slot and in a fixed order.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "ctx.h"

using namespace psfd;

namespace {

bool same_grid(const psfd_grid& a, const psfd_grid& b) {
  return a.nx == b.nx && a.ny == b.ny && a.nslab == b.nslab && a.nf == b.nf && a.dx == b.dx && a.dy == b.dy &&
         a.dz == b.dz && a.wavelength == b.wavelength && a.eps_bg == b.eps_bg;
}

// Stream priority levels a bucket can run at (rank 0 = the bucket holding the oldest
// running request).
constexpr int kPrioLevels = 4;

struct Bucket {
  psfd_grid grid{};
  psfd_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;             // the stream the context currently runs on
  cudaStream_t prio[kPrioLevels] = {};       // one stream per priority level, highest first
  cudaEvent_t handoff = nullptr;             // orders work across a stream change
  cudaEvent_t tick_done = nullptr;           // end of the bucket's enqueued engine step
  bool in_flight = false;                    // an engine step is enqueued and not completed
  std::vector<long long> rhs_owner;   // request id per illumination slot, -1 free
  std::vector<long long> clip_owner;  // request id per potential slot, -1 free
  size_t bytes = 0;
  int running = 0;
};

struct Request {
  long long id = 0;
  psfd_grid grid{};
  StackHost stack;
  std::vector<double2> eps;
  std::vector<double> th, ph;
  std::vector<int> pol;
  int state = 0;  // 0 queued, 1 running, 2 done
  int status = PSFD_OK;
  Bucket* bucket = nullptr;
  int clip = -1, g0 = -1;
  std::vector<int> nord;
  std::vector<std::vector<int>> mn;
  std::vector<std::vector<double>> out;  // per illumination: orders x 12 doubles
};

}  // namespace

// A graph that advances several buckets at once: one WHILE node per bucket (engine.cu,
// add_sweep_loop), keyed by the buckets, their batch widths and buffers.
struct RoundGraph {
  std::vector<long long> key;
  std::vector<int> kernels;  // kernels per tick of each bucket's loop
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool replayed = false;
  unsigned long long last_use = 0;
};

struct psfd_server {
  int precision = PSFD_FP32_REFINED;
  size_t budget = 0, used = 0;
  int slots = 18;
  psfd_solve_opts opts{};
  long long next_id = 1;
  std::deque<long long> queue;
  std::map<long long, std::unique_ptr<Request>> reqs;
  std::vector<std::unique_ptr<Bucket>> buckets;
  // fused rounds (psfd_server_set_rounds): every bucket runs on round_stream, and the Krylov
  // ticks of all buckets inside a sweep run as one graph launch per round
  int round_ticks = 0;  // 0: buckets advance independently on their own streams
  int max_running = 0;  // requests in flight at once over all buckets (0: as many as fit)
  cudaStream_t round_stream = nullptr;
  cudaEvent_t round_done = nullptr;
  bool round_in_flight = false;
  std::vector<RoundGraph> rounds;
  unsigned long long round_clock = 0;
};

namespace {

void drop_rounds(psfd_server* s) {
  for (auto& r : s->rounds) {
    if (r.exec) cudaGraphExecDestroy(r.exec);
    if (r.graph) cudaGraphDestroy(r.graph);
  }
  s->rounds.clear();
}

void destroy_bucket(psfd_server* s, Bucket* b) {
  drop_rounds(s);  // round graphs may refer to the bucket's buffers
  if (b->ctx) psfd_destroy(b->ctx);
  for (cudaStream_t st : b->prio)
    if (st) cudaStreamDestroy(st);
  if (b->handoff) cudaEventDestroy(b->handoff);
  if (b->tick_done) cudaEventDestroy(b->tick_done);
  s->used -= b->bytes;
  s->buckets.erase(std::remove_if(s->buckets.begin(), s->buckets.end(),
                                  [&](const std::unique_ptr<Bucket>& p) { return p.get() == b; }),
                   s->buckets.end());
}

// Create a bucket for grid g if the budget allows, releasing idle buckets if needed.
Bucket* make_bucket(psfd_server* s, const psfd_grid& g, int cap, int* rc) {
  const Plan plan = make_plan(g, s->precision, cap, cap);
  const size_t need = plan.bytes + pool_extra_bytes(plan, s->precision, cap, s->opts);
  if (s->budget && s->used + need > s->budget) {
    for (size_t i = 0; i < s->buckets.size();) {
      Bucket* b = s->buckets[i].get();
      if (b->running == 0 && s->used + need > s->budget) {
        destroy_bucket(s, b);
      } else {
        ++i;
      }
    }
  }
  if (s->budget && s->used + need > s->budget) {
    *rc = PSFD_E_BUDGET;
    return nullptr;
  }
  auto b = std::make_unique<Bucket>();
  b->grid = g;
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  bool ok = cudaEventCreateWithFlags(&b->handoff, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->tick_done, cudaEventDisableTiming) == cudaSuccess;
  for (int l = 0; l < kPrioLevels && ok; ++l) {
    const int prio = std::min(least, greatest + l);  // greatest = highest priority
    ok = cudaStreamCreateWithPriority(&b->prio[l], cudaStreamNonBlocking, prio) == cudaSuccess;
  }
  if (!ok) {
    for (cudaStream_t st : b->prio)
      if (st) cudaStreamDestroy(st);
    if (b->handoff) cudaEventDestroy(b->handoff);
    if (b->tick_done) cudaEventDestroy(b->tick_done);
    *rc = PSFD_E_CUDA;
    return nullptr;
  }
  b->stream = b->prio[kPrioLevels - 1];
  *rc = ctx_create(&b->ctx, &g, s->precision, cap, cap, 0, b->stream);
  if (*rc == PSFD_OK) b->ctx->device_loop = false;  // admission happens between ticks
  if (*rc == PSFD_OK) *rc = ensure_pool(b->ctx, s->opts);
  if (*rc != PSFD_OK) {
    if (b->ctx) psfd_destroy(b->ctx);
    for (cudaStream_t st : b->prio) cudaStreamDestroy(st);
    cudaEventDestroy(b->handoff);
    cudaEventDestroy(b->tick_done);
    return nullptr;
  }
  b->bytes = need;
  b->rhs_owner.assign(cap, -1);
  b->clip_owner.assign(cap, -1);
  s->used += need;
  s->buckets.push_back(std::move(b));
  return s->buckets.back().get();
}

// Claim a free potential slot and a run of n free illumination slots.
bool find_slots(Bucket* b, int n, int* clip, int* g0) {
  *clip = -1;
  for (size_t c = 0; c < b->clip_owner.size(); ++c)
    if (b->clip_owner[c] < 0) { *clip = (int)c; break; }
  if (*clip < 0) return false;
  const int R = (int)b->rhs_owner.size();
  for (int start = 0; start + n <= R; ++start) {
    bool ok = true;
    for (int i = 0; i < n && ok; ++i) ok = b->rhs_owner[start + i] < 0;
    if (ok) {
      *g0 = start;
      return true;
    }
  }
  return false;
}

int admit(psfd_server* s, Request* r, bool* admitted) {
  *admitted = false;
  if (s->max_running > 0) {  // the request waits, in arrival order, for a running one to retire
    int running = 0;
    for (auto& bp : s->buckets) running += bp->running;
    if (running >= s->max_running) return PSFD_OK;
  }
  Bucket* b = nullptr;
  int clip = -1, g0 = -1;
  for (auto& bp : s->buckets)
    if (!bp->in_flight && same_grid(bp->grid, r->grid) && find_slots(bp.get(), (int)r->th.size(), &clip, &g0)) {
      b = bp.get();
      break;
    }
  if (!b) {
    bool have_shape = false;
    for (auto& bp : s->buckets) have_shape = have_shape || same_grid(bp->grid, r->grid);
    if (have_shape && (int)r->th.size() <= s->slots) return PSFD_OK;  // wait for slots of that bucket
    int rc = PSFD_OK;
    const int cap = std::max(s->slots, (int)r->th.size());
    const Plan plan = make_plan(r->grid, s->precision, cap, cap);
    if (s->budget && plan.bytes + pool_extra_bytes(plan, s->precision, cap, s->opts) > s->budget) {
      r->state = 2;  // can never fit: rejected
      r->status = PSFD_E_BUDGET;
      *admitted = true;
      return PSFD_OK;
    }
    b = make_bucket(s, r->grid, cap, &rc);
    if (!b && rc == PSFD_E_NOMEM) {
      bool running = false;
      for (auto& bp : s->buckets) running = running || bp->running > 0;
      if (running) return PSFD_OK;  // device memory may free up when running requests finish
      r->state = 2;                 // nothing to wait for: the request fails, the server goes on
      r->status = PSFD_E_NOMEM;
      *admitted = true;
      return PSFD_OK;
    }
    if (!b) return rc == PSFD_E_BUDGET ? PSFD_OK : rc;  // wait for memory
    if (!find_slots(b, (int)r->th.size(), &clip, &g0)) return PSFD_E_ARG;
  }
  psfd_ctx* ctx = b->ctx;
  int rc = ctx_set_potential(ctx, clip, reinterpret_cast<const double*>(r->eps.data()), PSFD_HOST);
  if (rc == PSFD_OK)
    rc = ctx_set_rhs(ctx, g0, (int)r->th.size(), r->th.data(), r->ph.data(), r->pol.data(), clip, r->stack);
  if (rc != PSFD_OK) {
    r->state = 2;
    r->status = rc;
    *admitted = true;
    return PSFD_OK;
  }
  b->clip_owner[clip] = r->id;
  for (size_t i = 0; i < r->th.size(); ++i) b->rhs_owner[g0 + i] = r->id;
  b->running += 1;
  r->bucket = b;
  r->clip = clip;
  r->g0 = g0;
  r->state = 1;
  *admitted = true;
  return PSFD_OK;
}

int retire(psfd_server* s, Bucket* b) {
  psfd_ctx* ctx = b->ctx;
  bool copied = false;
  for (auto& kv : s->reqs) {
    Request* r = kv.second.get();
    if (r->state != 1 || r->bucket != b) continue;
    const int n = (int)r->th.size();
    bool done = true;
    for (int i = 0; i < n && done; ++i) done = ctx->phase[r->g0 + i] == PH_DONE;
    if (!done) continue;
    if (!copied) {
      int rc = ctx_orders_to_host(ctx);
      if (rc) return rc;
      copied = true;
    }
    const size_t M = (size_t)ctx->plan.max_orders;
    r->nord.assign(n, 0);
    r->mn.assign(n, {});
    r->out.assign(n, {});
    for (int i = 0; i < n; ++i) {
      const int g = r->g0 + i;
      const int k = ctx->h_nord[g];
      r->nord[i] = k;
      r->mn[i].assign(ctx->h_mn.begin() + (ptrdiff_t)(g * M * 2), ctx->h_mn.begin() + (ptrdiff_t)(g * M * 2 + 2 * k));
      r->out[i].assign(ctx->h_ordout.begin() + (ptrdiff_t)(g * M * 12),
                       ctx->h_ordout.begin() + (ptrdiff_t)(g * M * 12 + 12 * k));
      if (ctx->status[g] != PSFD_OK && r->status == PSFD_OK) r->status = ctx->status[g];
      ctx->phase[g] = PH_FREE;
      b->rhs_owner[g] = -1;
    }
    b->clip_owner[r->clip] = -1;
    b->running -= 1;
    r->state = 2;
    r->bucket = nullptr;
  }
  return PSFD_OK;
}

// One non-blocking pass: complete the buckets whose engine step has finished, admit queued
// requests into buckets between steps, then enqueue the next step of every idle bucket with
// work on its priority stream. Returns whether anything completed or was admitted.
static int progress_pass(psfd_server* s, bool* moved) {
  *moved = false;
  // 1. completions: buckets whose last step has finished on the device
  for (auto& bp : s->buckets) {
    Bucket* b = bp.get();
    if (!b->in_flight) continue;
    const cudaError_t q = cudaEventQuery(b->tick_done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return PSFD_E_CUDA;
    b->in_flight = false;
    *moved = true;
    int active = 0;
    int rc = engine_complete(b->ctx, s->opts, &active);
    if (rc != PSFD_OK) return rc;
    if ((rc = retire(s, b)) != PSFD_OK) return rc;
  }
  // 2. admissions, in arrival order; requests that do not fit yet stay queued
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    Request* r = s->reqs[*it].get();
    bool admitted = false;
    const int rc = admit(s, r, &admitted);
    if (rc != PSFD_OK) return rc;
    *moved = *moved || admitted;
    it = admitted ? s->queue.erase(it) : std::next(it);
  }
  // 3. stream priorities by age: the bucket holding the oldest running request runs at the
  //    highest priority, the next at the next level, and so on, so the block scheduler
  //    serves requests in arrival order while younger ones fill the idle SMs; then the next
  //    engine step of every idle bucket with work is enqueued (buckets advance
  //    independently: none waits for a slower one)
  std::vector<std::pair<long long, Bucket*>> order;
  for (auto& bp : s->buckets) {
    if (bp->running == 0) continue;
    long long oldest = -1;
    for (long long id : bp->rhs_owner)
      if (id >= 0 && (oldest < 0 || id < oldest)) oldest = id;
    order.push_back({oldest, bp.get()});
  }
  std::sort(order.begin(), order.end(),
            [](const std::pair<long long, Bucket*>& a, const std::pair<long long, Bucket*>& b) {
              return a.first < b.first;
            });
  for (size_t r = 0; r < order.size(); ++r) {
    Bucket* b = order[r].second;
    if (b->in_flight) continue;
    cudaStream_t want = b->prio[std::min<size_t>(r, kPrioLevels - 1)];
    if (want != b->stream) {
      // whatever the context queued on its previous stream (admission uploads) comes first
      if (cudaEventRecord(b->handoff, b->stream) != cudaSuccess ||
          cudaStreamWaitEvent(want, b->handoff, 0) != cudaSuccess)
        return PSFD_E_CUDA;
      b->stream = want;
      psfd_set_stream(b->ctx, want);
    }
    bool pending = false;
    const int rc = engine_enqueue(b->ctx, s->opts, &pending, nullptr);
    if (rc != PSFD_OK) return rc;
    if (cudaEventRecord(b->tick_done, b->stream) != cudaSuccess) return PSFD_E_CUDA;
    b->in_flight = true;
  }
  return PSFD_OK;
}

// The round graph of these buckets (built on first use; the context's loop bodies are captured
// with their current batch width and buffers, which are part of the key).
RoundGraph* round_graph(psfd_server* s, const std::vector<Bucket*>& list, int* rc) {
  const bool f32 = s->precision == PSFD_FP32_REFINED;
  std::vector<long long> key;
  for (Bucket* b : list) {
    psfd_ctx* c = b->ctx;
    key.push_back((long long)(uintptr_t)c);
    key.push_back(c->enq_hi);
    key.push_back((long long)(f32 ? (uintptr_t)c->pool32 : (uintptr_t)c->pool64));
    key.push_back(c->no_reflect);
  }
  for (auto& r : s->rounds)
    if (r.key == key) {
      r.last_use = ++s->round_clock;
      return &r;
    }
  constexpr size_t kMaxRounds = 16;
  if (s->rounds.size() >= kMaxRounds) {
    auto old = std::min_element(s->rounds.begin(), s->rounds.end(),
                                [](const RoundGraph& a, const RoundGraph& b) { return a.last_use < b.last_use; });
    if (old->exec) cudaGraphExecDestroy(old->exec);
    if (old->graph) cudaGraphDestroy(old->graph);
    s->rounds.erase(old);
  }
  RoundGraph r;
  r.key = key;
  if (cudaGraphCreate(&r.graph, 0) != cudaSuccess) {
    *rc = PSFD_E_CUDA;
    return nullptr;
  }
  for (Bucket* b : list) {
    int k = 0;
    *rc = add_sweep_loop(b->ctx, s->opts, b->ctx->enq_hi, f32, r.graph, s->round_ticks, &k);
    if (*rc != PSFD_OK) {
      cudaGraphDestroy(r.graph);
      return nullptr;
    }
    r.kernels.push_back(k);
  }
  if (cudaGraphInstantiate(&r.exec, r.graph, 0) != cudaSuccess) {
    cudaGraphDestroy(r.graph);
    *rc = PSFD_E_CUDA;
    return nullptr;
  }
  r.last_use = ++s->round_clock;
  s->rounds.push_back(std::move(r));
  *rc = PSFD_OK;
  return &s->rounds.back();
}

// One non-blocking pass of the fused rounds: when the previous round has finished, complete
// every bucket, admit, enqueue each bucket's phase work (norms, FP64 residuals, sweep starts,
// orders) on round_stream, and launch one graph whose WHILE nodes run up to round_ticks ticks
// of every bucket that is inside a Krylov sweep, side by side.
int progress_round(psfd_server* s, bool* moved) {
  *moved = false;
  if (s->round_in_flight) {
    const cudaError_t q = cudaEventQuery(s->round_done);
    if (q == cudaErrorNotReady) return PSFD_OK;
    if (q != cudaSuccess) return PSFD_E_CUDA;
    s->round_in_flight = false;
    *moved = true;
    for (auto& bp : s->buckets) {
      Bucket* b = bp.get();
      if (!b->in_flight) continue;
      b->in_flight = false;
      int active = 0;
      int rc = engine_complete(b->ctx, s->opts, &active);
      if (rc != PSFD_OK) return rc;
      if ((rc = retire(s, b)) != PSFD_OK) return rc;
    }
  }
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    Request* r = s->reqs[*it].get();
    bool admitted = false;
    const int rc = admit(s, r, &admitted);
    if (rc != PSFD_OK) return rc;
    *moved = *moved || admitted;
    it = admitted ? s->queue.erase(it) : std::next(it);
  }
  std::vector<Bucket*> looping;
  bool any = false;
  for (auto& bp : s->buckets) {
    Bucket* b = bp.get();
    if (b->running == 0) continue;
    if (b->stream != s->round_stream) {
      if (cudaEventRecord(b->handoff, b->stream) != cudaSuccess ||
          cudaStreamWaitEvent(s->round_stream, b->handoff, 0) != cudaSuccess)
        return PSFD_E_CUDA;
      b->stream = s->round_stream;
      psfd_set_stream(b->ctx, s->round_stream);
    }
    bool pending = false, deferred = false;
    const int rc = engine_enqueue(b->ctx, s->opts, &pending, &deferred);
    if (rc != PSFD_OK) return rc;
    if (deferred) looping.push_back(b);
    b->in_flight = pending;
    any = any || pending;
  }
  if (!looping.empty()) {
    int rc = PSFD_OK;
    RoundGraph* r = round_graph(s, looping, &rc);
    if (!r) return rc;
    for (size_t i = 0; i < looping.size(); ++i) {
      looping[i]->ctx->loop_kernels = r->kernels[i];
      looping[i]->ctx->loop_precounted = r->replayed ? 0 : r->kernels[i];
    }
    r->replayed = true;
    if (cudaGraphLaunch(r->exec, s->round_stream) != cudaSuccess) return PSFD_E_CUDA;
    for (Bucket* b : looping) {
      if ((rc = loop_readback(b->ctx, b->ctx->enq_hi)) != PSFD_OK) return rc;
      if ((rc = engine_readback(b->ctx)) != PSFD_OK) return rc;
    }
  }
  if (any) {
    if (cudaEventRecord(s->round_done, s->round_stream) != cudaSuccess) return PSFD_E_CUDA;
    s->round_in_flight = true;
  }
  return PSFD_OK;
}

}  // namespace

extern "C" {

int psfd_server_set_max_running(psfd_server* s, int n) {
  if (!s || n < 0) return PSFD_E_ARG;
  s->max_running = n;
  return PSFD_OK;
}

int psfd_server_set_rounds(psfd_server* s, int ticks_per_round) {
  if (!s || ticks_per_round < 0) return PSFD_E_ARG;
  // only between rounds, with every bucket idle
  if (s->round_in_flight) return PSFD_E_STATE;
  for (auto& bp : s->buckets)
    if (bp->in_flight) return PSFD_E_STATE;
  if (ticks_per_round > 0 && !s->round_stream) {
    if (cudaStreamCreateWithFlags(&s->round_stream, cudaStreamNonBlocking) != cudaSuccess) return PSFD_E_CUDA;
    if (cudaEventCreateWithFlags(&s->round_done, cudaEventDisableTiming) != cudaSuccess) return PSFD_E_CUDA;
  }
  drop_rounds(s);
  s->round_ticks = ticks_per_round;
  return PSFD_OK;
}

int psfd_server_create(psfd_server** out, int precision, size_t hbm_budget, int slots_per_context,
                       const psfd_solve_opts* opts) {
  if (!out || (precision != PSFD_FP64 && precision != PSFD_FP32_REFINED) || slots_per_context < 1)
    return PSFD_E_ARG;
  psfd_server* s = new psfd_server();
  s->precision = precision;
  s->budget = hbm_budget;
  s->slots = slots_per_context;
  s->opts = solve_defaults(opts);
  *out = s;
  return PSFD_OK;
}

int psfd_server_destroy(psfd_server* s) {
  if (!s) return PSFD_OK;
  if (s->round_stream) cudaStreamSynchronize(s->round_stream);
  while (!s->buckets.empty()) destroy_bucket(s, s->buckets.back().get());
  drop_rounds(s);
  if (s->round_done) cudaEventDestroy(s->round_done);
  if (s->round_stream) cudaStreamDestroy(s->round_stream);
  delete s;
  return PSFD_OK;
}

int psfd_server_submit(psfd_server* s, const psfd_request* q, long long* ticket) {
  if (!s || !q || !ticket || !q->eps || !q->n_sub || q->n_rhs < 1 || !q->theta_deg || !q->phi_deg || !q->pol ||
      q->n_layers < 0 || q->n_layers > kStackMaxLayers || (q->n_layers > 0 && (!q->n_complex || !q->thickness_nm)))
    return PSFD_E_ARG;
  std::string why;
  if (!grid_ok(&q->grid, why)) return PSFD_E_ARG;
  auto r = std::make_unique<Request>();
  r->id = s->next_id++;
  r->grid = q->grid;
  r->stack.eps.resize(q->n_layers);
  r->stack.d.assign(q->thickness_nm, q->thickness_nm + q->n_layers);
  for (int j = 0; j < q->n_layers; ++j) {
    const double a = q->n_complex[2 * j], b = q->n_complex[2 * j + 1];
    r->stack.eps[j] = make_double2(a * a - b * b, 2.0 * a * b);
  }
  r->stack.eps_sub = make_double2(q->n_sub[0] * q->n_sub[0] - q->n_sub[1] * q->n_sub[1], 2.0 * q->n_sub[0] * q->n_sub[1]);
  r->stack.set = true;
  const size_t n = (size_t)q->grid.nx * q->grid.ny * q->grid.nslab;
  r->eps.resize(n);
  std::memcpy(r->eps.data(), q->eps, n * sizeof(double2));
  r->th.assign(q->theta_deg, q->theta_deg + q->n_rhs);
  r->ph.assign(q->phi_deg, q->phi_deg + q->n_rhs);
  r->pol.assign(q->pol, q->pol + q->n_rhs);
  *ticket = r->id;
  s->queue.push_back(r->id);
  s->reqs[r->id] = std::move(r);
  return PSFD_OK;
}

int psfd_server_progress(psfd_server* s, int* n_pending) {
  if (!s) return PSFD_E_ARG;
  // repeat non-blocking passes until something moves (or briefly, 2 ms, if nothing can)
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    bool moved = false;
    const int rc = s->round_ticks > 0 ? progress_round(s, &moved) : progress_pass(s, &moved);
    if (rc != PSFD_OK) return rc;
    bool any_in_flight = s->round_in_flight;
    for (auto& bp : s->buckets) any_in_flight = any_in_flight || bp->in_flight;
    if (moved || !any_in_flight ||
        std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(2000))
      break;
  }
  if (n_pending) {
    int n = (int)s->queue.size();
    for (auto& bp : s->buckets) n += bp->running;
    *n_pending = n;
  }
  return PSFD_OK;
}

int psfd_server_status(psfd_server* s, long long ticket, int* state, int* status) {
  if (!s || !state) return PSFD_E_ARG;
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return PSFD_E_ARG;
  *state = it->second->state;
  if (status) *status = it->second->status;
  return PSFD_OK;
}

int psfd_server_orders(psfd_server* s, long long ticket, int rhs, int capacity, int* n_orders, int* mn, double* amp,
                       double* sp, double* eff) {
  if (!s || !n_orders || !mn) return PSFD_E_ARG;
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return PSFD_E_ARG;
  Request* r = it->second.get();
  if (r->state != 2 || r->nord.empty()) return PSFD_E_STATE;
  if (rhs < 0 || rhs >= (int)r->nord.size()) return PSFD_E_ARG;
  const int n = r->nord[rhs];
  *n_orders = n;
  if (capacity < n) return PSFD_E_ARG;
  for (int k = 0; k < n; ++k) {
    const double* o = r->out[rhs].data() + 12 * k;
    mn[2 * k] = r->mn[rhs][2 * k];
    mn[2 * k + 1] = r->mn[rhs][2 * k + 1];
    if (amp) std::memcpy(amp + 6 * k, o, 6 * sizeof(double));
    if (sp) std::memcpy(sp + 4 * k, o + 6, 4 * sizeof(double));
    if (eff) eff[k] = o[10];
  }
  return PSFD_OK;
}

int psfd_server_release(psfd_server* s, long long ticket) {
  if (!s) return PSFD_E_ARG;
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || it->second->state == 1) return PSFD_E_STATE;
  if (it->second->state == 0) s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), ticket), s->queue.end());
  s->reqs.erase(it);
  return PSFD_OK;
}

int psfd_server_memory(psfd_server* s, size_t* used, int* n_contexts) {
  if (!s) return PSFD_E_ARG;
  if (used) *used = s->used;
  if (n_contexts) *n_contexts = (int)s->buckets.size();
  return PSFD_OK;
}

}  // extern "C"
