// serve.cu -- continuous-batching request server (qaoa_server_*; not in the
// paper).  Objective (+ gradient) requests of different n and p arrive at any
// time; a scheduler thread admits them as GPU slots and device memory free up
// and runs admitted work concurrently:
//   * n <= 12 requests are packed, many per launch, into k_small_batch
//     (one CTA per request, state and lambda on chip);
//   * larger requests run qaoa_grad / qaoa_simulate on their own stream,
//     several streams at once, so mid-size requests that cannot fill the GPU
//     alone overlap with each other.
// Device memory is one caller-provided arena, sub-allocated here: each
// request takes its footprint (state, lambda, workspace, outputs) while it
// runs; cost vectors are cached by problem key and evicted least recently
// used when memory is needed.  A request whose footprint exceeds the arena is
// rejected at once.  Every request's arithmetic depends only on its own
// inputs (fixed launch shapes, deterministic reductions), so its result is
// the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/qaoa.h"
#include "kernels.h"
#include "qaoa_common.cuh"

namespace qaoa {
void set_last_error(const char *msg);
}

using namespace qaoa;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

constexpr size_t kAlign = 256;
size_t up(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

// First-fit sub-allocator over [0, size) with coalescing.
struct Arena {
  size_t size = 0, used = 0, peak = 0;
  std::map<size_t, size_t> free_;  // offset -> bytes
  void init(size_t s) {
    size = s & ~(kAlign - 1);
    free_.clear();
    free_[0] = size;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t o2 = it->first + bytes;
        free_.erase(it);
        if (rest) free_[o2] = rest;
        used += bytes;
        peak = std::max(peak, used);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = up(bytes);
    used -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct CostEntry {
  size_t off = 0, bytes = 0;
  qaoa_cost_type ct = QAOA_COST_I32;
  qaoa_cost_stats stats{};
  int refs = 0;
  uint64_t last_use = 0;
};

using CostKey = std::tuple<int, int, uint64_t>;  // problem, n, key

enum JobState { kPending, kRunning, kDone };

struct Job {
  uint64_t ticket = 0;
  int problem = 0, n = 0, p = 0, want_grad = 0;
  uint64_t key = 0;
  std::vector<int32_t> edges;
  std::vector<double> weights, g, b;
  JobState state = kPending;
  bool cancelled = false;
  qaoa_status status = QAOA_OK;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  std::vector<double> result;  // [E, O, dg.., db..]
  // device resources while running
  std::vector<std::pair<size_t, size_t>> allocs;
  CostKey ckey;
  bool holds_cost = false;
  int unit = -1;  // running unit index
  int bypassed = 0;  // later jobs admitted while this one waited for memory
};

// A unit of GPU work: one large job, or one batch of small jobs, on a stream.
struct Unit {
  bool busy = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<Job *> jobs;
  double *h_out = nullptr;  // pinned host results
  size_t h_out_cap = 0;     // doubles
  unsigned char *h_stage = nullptr;  // pinned host staging (small batches)
  size_t h_stage_cap = 0;
  std::vector<std::pair<size_t, size_t>> allocs;  // batch-wide device buffers
};

constexpr size_t kStageBytes = 4u << 20;  // pinned staging per unit
constexpr size_t kOutDoubles = 1u << 18;  // pinned result slots per unit

}  // namespace

struct qaoa_server {
  qaoa_server_config cfg{};
  unsigned char *d_arena = nullptr;
  Arena arena;
  std::map<CostKey, CostEntry> costs;
  uint64_t use_clock = 0;
  std::vector<Unit> units;
  std::deque<Job *> pending;
  std::map<uint64_t, Job *> jobs;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  int device = 0;
  // statistics
  uint64_t n_submitted = 0, n_completed = 0, n_rejected = 0, n_cancelled = 0;
  double first_submit = -1, last_finish = 0;
  std::vector<double> latencies;
};

namespace {

size_t state_bytes(int n) { return (size_t)8 << n; }  // complex64
size_t cost_bytes_of(int n) { return (size_t)4 << n; }

qaoa_cost_type cost_type_of(const Job &j) {
  if (j.problem == QAOA_PROBLEM_LABS) return QAOA_COST_I32;
  for (double w : j.weights)
    if (w != std::nearbyint(w)) return QAOA_COST_F32;
  return QAOA_COST_I32;
}

// Footprint of a large job while it runs (excluding its cost vector).
size_t large_footprint(const Job &j) {
  return up(state_bytes(j.n)) + (j.want_grad ? up(state_bytes(j.n)) : 0) + up(qaoa_workspace_bytes(j.n)) +
         up(sizeof(double) * (2 + 2 * (size_t)j.p));
}

bool alloc_or_evict(qaoa_server *S, size_t bytes, size_t *off) {
  while (!S->arena.alloc(bytes, off)) {
    // evict the least recently used cost vector nobody holds
    auto victim = S->costs.end();
    for (auto it = S->costs.begin(); it != S->costs.end(); ++it)
      if (it->second.refs == 0 && (victim == S->costs.end() || it->second.last_use < victim->second.last_use))
        victim = it;
    if (victim == S->costs.end()) return false;
    S->arena.release(victim->second.off, victim->second.bytes);
    S->costs.erase(victim);
  }
  return true;
}

// Cached cost vector of the job's problem, built on `st` if missing.
// Returns nullptr if memory does not allow it now.
CostEntry *get_cost(qaoa_server *S, Job &j, cudaStream_t st, void *d_work, size_t work_bytes,
                    qaoa_status *err) {
  const CostKey k{j.problem, j.n, j.key};
  auto it = S->costs.find(k);
  if (it != S->costs.end()) {
    it->second.last_use = ++S->use_clock;
    return &it->second;
  }
  size_t off;
  if (!alloc_or_evict(S, cost_bytes_of(j.n), &off)) return nullptr;
  CostEntry e;
  e.off = off;
  e.bytes = cost_bytes_of(j.n);
  e.ct = cost_type_of(j);
  void *d = S->d_arena + off;
  qaoa_status r;
  if (j.problem == QAOA_PROBLEM_LABS)
    r = qaoa_labs_costs(j.n, reinterpret_cast<int32_t *>(d), reinterpret_cast<qaoa_stream_t>(st));
  else
    r = qaoa_maxcut_costs(j.n, j.edges.data(), j.weights.data(), j.weights.size(), e.ct, d,
                          reinterpret_cast<qaoa_stream_t>(st));
  if (r == QAOA_OK)
    r = qaoa_cost_stats_compute(j.n, d, e.ct, d_work, work_bytes, &e.stats,
                                reinterpret_cast<qaoa_stream_t>(st));
  if (r != QAOA_OK) {
    S->arena.release(off, e.bytes);
    *err = r;
    return nullptr;
  }
  e.last_use = ++S->use_clock;
  return &(S->costs[k] = e);
}

void finish_job(qaoa_server *S, Job *j, qaoa_status st) {
  j->status = st;
  j->state = kDone;
  j->t_finish = now_s();
  for (auto &a : j->allocs) S->arena.release(a.first, a.second);
  j->allocs.clear();
  if (j->holds_cost) {
    auto it = S->costs.find(j->ckey);
    if (it != S->costs.end()) it->second.refs -= 1;
    j->holds_cost = false;
  }
  if (st == QAOA_OK) {
    S->n_completed += 1;
    S->latencies.push_back(j->t_finish - j->t_submit);
    S->last_finish = std::max(S->last_finish, j->t_finish);
  }
}

int free_unit(qaoa_server *S) {
  for (size_t i = 0; i < S->units.size(); ++i)
    if (!S->units[i].busy) return (int)i;
  return -1;
}

// Start one large job on unit u; false if memory does not allow it yet.
bool start_large(qaoa_server *S, Job *j, int u) {
  Unit &U = S->units[u];
  size_t o_state, o_lam = 0, o_work, o_out;
  std::vector<std::pair<size_t, size_t>> got;
  auto take = [&](size_t bytes, size_t *o) {
    if (!alloc_or_evict(S, bytes, o)) return false;
    got.emplace_back(*o, bytes);
    return true;
  };
  const size_t wsb = qaoa_workspace_bytes(j->n);
  if (!take(state_bytes(j->n), &o_state) || (j->want_grad && !take(state_bytes(j->n), &o_lam)) ||
      !take(wsb, &o_work) || !take(sizeof(double) * (2 + 2 * (size_t)j->p), &o_out)) {
    for (auto &a : got) S->arena.release(a.first, a.second);
    return false;
  }
  qaoa_status err = QAOA_OK;
  CostEntry *ce = get_cost(S, *j, U.stream, S->d_arena + o_work, wsb, &err);
  if (!ce) {
    for (auto &a : got) S->arena.release(a.first, a.second);
    if (err != QAOA_OK) {
      finish_job(S, j, err);
      return true;
    }
    return false;
  }
  ce->refs += 1;
  j->holds_cost = true;
  j->ckey = CostKey{j->problem, j->n, j->key};
  j->allocs = got;
  j->t_admit = now_s();
  qaoa_stream_t st = reinterpret_cast<qaoa_stream_t>(U.stream);
  double *d_out = reinterpret_cast<double *>(S->d_arena + o_out);
  qaoa_status r;
  if (j->want_grad)
    r = qaoa_grad(j->n, S->d_arena + ce->off, ce->ct, &ce->stats, j->g.data(), j->b.data(), j->p,
                  S->d_arena + o_state, S->d_arena + o_lam, QAOA_C64, S->d_arena + o_work, wsb, d_out, st);
  else
    r = qaoa_simulate(j->n, S->d_arena + ce->off, ce->ct, &ce->stats, j->g.data(), j->b.data(), j->p,
                      S->d_arena + o_state, QAOA_C64, 1, S->d_arena + o_work, wsb, d_out, st);
  const size_t nd = j->want_grad ? 2 + 2 * (size_t)j->p : 2;
  if (r == QAOA_OK && nd <= U.h_out_cap)
    r = cudaMemcpyAsync(U.h_out, d_out, nd * sizeof(double), cudaMemcpyDeviceToHost, U.stream) == cudaSuccess
            ? QAOA_OK : QAOA_ERR_CUDA;
  if (r == QAOA_OK) r = cudaEventRecord(U.done, U.stream) == cudaSuccess ? QAOA_OK : QAOA_ERR_CUDA;
  if (r != QAOA_OK) {
    finish_job(S, j, r);
    return true;
  }
  j->state = kRunning;
  j->unit = u;
  U.busy = true;
  U.jobs.assign(1, j);
  return true;
}

// Pack pending small jobs (n <= 12, p <= 128) into one launch on unit u.
bool start_small_batch(qaoa_server *S, std::vector<Job *> &cand, int u) {
  Unit &U = S->units[u];
  std::vector<Job *> batch;
  size_t stage = 0, outs = 0;
  int max_n = 1;
  for (Job *j : cand) {
    if ((int)batch.size() >= S->cfg.small_batch) break;
    const size_t need = sizeof(SmallJob<float>) + sizeof(SmallLayer<float>) * j->p;
    const size_t nd = 2 + 2 * (size_t)j->p;
    if (stage + need > U.h_stage_cap || outs + nd > U.h_out_cap) break;
    stage += need;
    outs += nd;
    max_n = std::max(max_n, j->n);
    batch.push_back(j);
  }
  if (batch.empty()) return false;
  // device buffers: descriptors + layers (staged), outputs, states, lambdas
  size_t bytes_state = 0;
  for (Job *j : batch) bytes_state += 2 * up(state_bytes(j->n));
  size_t o_stage, o_out, o_states;
  std::vector<std::pair<size_t, size_t>> got;
  auto take = [&](size_t bytes, size_t *o) {
    if (!alloc_or_evict(S, bytes, o)) return false;
    got.emplace_back(*o, bytes);
    return true;
  };
  if (!take(stage + kAlign, &o_stage) || !take(outs * sizeof(double), &o_out) || !take(bytes_state, &o_states)) {
    for (auto &a : got) S->arena.release(a.first, a.second);
    return false;
  }
  // cost vectors (built synchronously on this unit's stream when missing)
  std::vector<CostEntry *> ce(batch.size());
  size_t wsb = qaoa_workspace_bytes(kSmallMaxN);
  size_t o_ws;
  if (!take(wsb, &o_ws)) {
    for (auto &a : got) S->arena.release(a.first, a.second);
    return false;
  }
  for (size_t i = 0; i < batch.size(); ++i) {
    qaoa_status err = QAOA_OK;
    ce[i] = get_cost(S, *batch[i], U.stream, S->d_arena + o_ws, wsb, &err);
    if (!ce[i]) {
      for (size_t k = 0; k < i; ++k) ce[k]->refs -= 1;
      for (auto &a : got) S->arena.release(a.first, a.second);
      if (err != QAOA_OK) {
        finish_job(S, batch[i], err);
        S->pending.erase(std::find(S->pending.begin(), S->pending.end(), batch[i]));
      }
      return err != QAOA_OK;
    }
    ce[i]->refs += 1;
  }
  // host staging: job descriptors first, then each job's layers
  SmallJob<float> *hj = reinterpret_cast<SmallJob<float> *>(U.h_stage);
  SmallLayer<float> *hl = reinterpret_cast<SmallLayer<float> *>(U.h_stage + sizeof(SmallJob<float>) * batch.size());
  const size_t layers_off = sizeof(SmallJob<float>) * batch.size();
  size_t lcur = 0, ocur = 0, scur = 0;
  const double two_pi = 6.283185307179586476925286766559;
  for (size_t i = 0; i < batch.size(); ++i) {
    Job *j = batch[i];
    SmallJob<float> J;
    memset(&J, 0, sizeof(J));
    J.psi = reinterpret_cast<float2 *>(S->d_arena + o_states + scur);
    J.lam = reinterpret_cast<float2 *>(S->d_arena + o_states + scur + up(state_bytes(j->n)));
    scur += 2 * up(state_bytes(j->n));
    J.cost = S->d_arena + ce[i]->off;
    J.cost_kind = (int)ce[i]->ct;
    J.n = j->n;
    J.nl = j->p;
    J.mode = j->want_grad ? 1 : 0;
    J.init_plus = 1;
    J.reduce = 1;
    J.amp = (float)(1.0 / std::sqrt(std::ldexp(1.0, j->n)));
    J.fmin_d = ce[i]->stats.f_min;
    double *d_o = reinterpret_cast<double *>(S->d_arena + o_out) + ocur;
    J.out = d_o;
    J.out_dg = d_o + 2;
    J.out_db = d_o + 2 + j->p;
    ocur += 2 + 2 * (size_t)j->p;
    J.L = reinterpret_cast<const SmallLayer<float> *>(S->d_arena + o_stage + layers_off) + lcur;
    for (int l = 0; l < j->p; ++l) {
      SmallLayer<float> L;
      L.cb = (float)std::cos(j->b[l]);
      L.sb = (float)std::sin(j->b[l]);
      const double g2 = j->g[l] / two_pi;
      L.g2pi = g2;
      L.g_hi = (float)g2;
      L.g_lo = (float)(g2 - (double)L.g_hi);
      hl[lcur + l] = L;
    }
    lcur += j->p;
    hj[i] = J;
    j->holds_cost = true;
    j->ckey = CostKey{j->problem, j->n, j->key};
    j->t_admit = now_s();
    j->state = kRunning;
    j->unit = u;
  }
  cudaError_t e = cudaMemcpyAsync(S->d_arena + o_stage, U.h_stage, stage, cudaMemcpyHostToDevice, U.stream);
  if (e == cudaSuccess)
    e = launch_small_batch(reinterpret_cast<const SmallJob<float> *>(S->d_arena + o_stage), (int)batch.size(),
                           max_n, U.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(U.h_out, S->d_arena + o_out, outs * sizeof(double), cudaMemcpyDeviceToHost, U.stream);
  if (e == cudaSuccess) e = cudaEventRecord(U.done, U.stream);
  U.allocs = got;
  U.jobs = batch;
  U.busy = true;
  if (e != cudaSuccess) {
    // the unit is reaped at once; its jobs report the error
    for (Job *j : batch) j->status = QAOA_ERR_CUDA;
  }
  for (Job *j : batch) {
    auto it = std::find(S->pending.begin(), S->pending.end(), j);
    if (it != S->pending.end()) S->pending.erase(it);
  }
  return true;
}

void reap(qaoa_server *S) {
  for (size_t u = 0; u < S->units.size(); ++u) {
    Unit &U = S->units[u];
    if (!U.busy) continue;
    const cudaError_t q = cudaEventQuery(U.done);
    if (q == cudaErrorNotReady) continue;
    size_t ocur = 0;
    for (Job *j : U.jobs) {
      const size_t nd = 2 + 2 * (size_t)j->p;
      const size_t len = (U.jobs.size() == 1 && !j->want_grad) ? 2 : nd;
      qaoa_status st = (q == cudaSuccess && j->status == QAOA_OK) ? QAOA_OK : QAOA_ERR_CUDA;
      if (j->cancelled) st = QAOA_ERR_CANCELLED;
      j->result.assign(U.h_out + ocur, U.h_out + ocur + len);
      ocur += (U.jobs.size() == 1) ? len : nd;
      finish_job(S, j, st);
      if (j->cancelled) S->n_cancelled += 1;
    }
    for (auto &a : U.allocs) S->arena.release(a.first, a.second);
    U.allocs.clear();
    U.jobs.clear();
    U.busy = false;
  }
}

constexpr int kMaxBypass = 8;

void worker_main(qaoa_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    reap(S);
    bool progressed = false;
    // small jobs: one batched launch per free unit
    std::vector<Job *> small;
    for (Job *j : S->pending)
      if (j->n <= kSmallMaxN && j->p <= kSmallMaxLayers) small.push_back(j);
    if (!small.empty()) {
      const int u = free_unit(S);
      if (u >= 0 && start_small_batch(S, small, u)) progressed = true;
    }
    // large jobs in arrival order; later ones may pass an earlier one that
    // does not fit yet (bounded look-ahead), but each waiting job lets at
    // most kMaxBypass pass it: after that nothing more is admitted behind it
    // until the running work has freed enough memory for it (no starvation
    // of the largest requests)
    int looked = 0;
    std::vector<Job *> skipped;
    for (auto it = S->pending.begin(); it != S->pending.end() && looked < 64;) {
      Job *j = *it;
      if (j->n <= kSmallMaxN && j->p <= kSmallMaxLayers) {
        ++it;
        continue;
      }
      ++looked;
      const int u = free_unit(S);
      if (u < 0) break;
      if (start_large(S, j, u)) {
        for (Job *k : skipped) ++k->bypassed;
        it = S->pending.erase(it);
        progressed = true;
      } else {
        if (j->bypassed >= kMaxBypass) break;
        skipped.push_back(j);
        ++it;
      }
    }
    S->cv_done.notify_all();
    if (!progressed) S->cv_work.wait_for(lk, std::chrono::microseconds(50));
  }
}

qaoa_status fail(qaoa_status st, const char *msg) {
  qaoa::set_last_error(msg);
  return st;
}

}  // namespace

extern "C" {

qaoa_status qaoa_server_create(const qaoa_server_config *cfg, void *d_arena, size_t arena_bytes,
                               qaoa_server **out) {
  if (!cfg || !d_arena || !out || ((uintptr_t)d_arena & (kAlign - 1)) || arena_bytes < (1u << 20))
    return fail(QAOA_ERR_INVALID_ARG, "server_create: bad config, arena (256-byte aligned, >= 1 MiB) or out");
  if (cfg->max_inflight < 1 || cfg->max_inflight > 64 || cfg->max_queue < 1 || cfg->small_batch < 1 ||
      cfg->small_batch > 4096)
    return fail(QAOA_ERR_INVALID_ARG, "server_create: max_inflight in [1, 64], max_queue >= 1, small_batch in [1, 4096]");
  qaoa_server *S = new qaoa_server();
  S->cfg = *cfg;
  S->d_arena = reinterpret_cast<unsigned char *>(d_arena);
  S->arena.init(arena_bytes);
  cudaGetDevice(&S->device);
  S->units.resize(cfg->max_inflight);
  for (Unit &U : S->units) {
    if (cudaStreamCreateWithFlags(&U.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&U.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&U.h_out, kOutDoubles * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&U.h_stage, kStageBytes) != cudaSuccess) {
      qaoa_server_destroy(S);
      return fail(QAOA_ERR_CUDA, "server_create: stream, event or pinned host buffer");
    }
    U.h_out_cap = kOutDoubles;
    U.h_stage_cap = kStageBytes;
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return QAOA_OK;
}

qaoa_status qaoa_server_submit(qaoa_server *S, const qaoa_request *req, uint64_t *ticket) {
  if (!S || !req || !ticket) return fail(QAOA_ERR_INVALID_ARG, "server_submit: NULL argument");
  if ((req->problem != QAOA_PROBLEM_LABS && req->problem != QAOA_PROBLEM_MAXCUT) || req->n < 2 ||
      req->n > 32 || req->p < 1 || req->p > 100000 || !req->gammas || !req->betas)
    return fail(QAOA_ERR_INVALID_ARG, "server_submit: bad problem, n (2..32), p or angles");
  for (int l = 0; l < req->p; ++l)
    if (!std::isfinite(req->gammas[l]) || !std::isfinite(req->betas[l]))
      return fail(QAOA_ERR_INVALID_ARG, "server_submit: non-finite angle");
  if (req->problem == QAOA_PROBLEM_MAXCUT) {
    if (req->m > 1536 || (req->m && !req->edges)) return fail(QAOA_ERR_INVALID_ARG, "server_submit: edges");
    for (size_t e = 0; e < req->m; ++e) {
      const int i = req->edges[2 * e], k = req->edges[2 * e + 1];
      if (i < 0 || k < 0 || i >= req->n || k >= req->n || i == k)
        return fail(QAOA_ERR_INVALID_ARG, "server_submit: bad edge");
      if (req->weights && !std::isfinite(req->weights[e])) return fail(QAOA_ERR_INVALID_ARG, "server_submit: weight");
    }
  }
  Job *j = new Job();
  j->problem = req->problem;
  j->n = req->n;
  j->p = req->p;
  j->want_grad = req->want_grad ? 1 : 0;
  j->key = req->problem_key;
  j->g.assign(req->gammas, req->gammas + req->p);
  j->b.assign(req->betas, req->betas + req->p);
  if (req->problem == QAOA_PROBLEM_MAXCUT) {
    j->edges.assign(req->edges, req->edges + 2 * req->m);
    j->weights.resize(req->m);
    for (size_t e = 0; e < req->m; ++e) j->weights[e] = req->weights ? req->weights[e] : 1.0;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  // can it ever fit?  (footprint + its cost vector must fit the empty arena)
  const bool small = j->n <= kSmallMaxN && j->p <= kSmallMaxLayers;
  const size_t need = small ? (2 * up(state_bytes(j->n)) + up(cost_bytes_of(j->n)) + (1u << 20))
                            : large_footprint(*j) + up(cost_bytes_of(j->n));
  j->t_submit = now_s();
  j->ticket = S->next_ticket++;
  *ticket = j->ticket;
  S->jobs[j->ticket] = j;
  S->n_submitted += 1;
  if (S->first_submit < 0) S->first_submit = j->t_submit;
  if (need > S->arena.size) {
    j->state = kDone;
    j->status = QAOA_ERR_REJECTED;
    j->t_finish = j->t_submit;
    S->n_rejected += 1;
    S->cv_done.notify_all();
    return QAOA_OK;  // the ticket reports the rejection
  }
  if ((int)S->pending.size() >= S->cfg.max_queue) {
    S->jobs.erase(j->ticket);
    S->n_submitted -= 1;
    delete j;
    return fail(QAOA_ERR_BUSY, "server_submit: queue full");
  }
  S->pending.push_back(j);
  S->cv_work.notify_one();
  return QAOA_OK;
}

qaoa_status qaoa_server_wait(qaoa_server *S, uint64_t ticket, qaoa_result *out, double *h_dgamma,
                             double *h_dbeta, int timeout_ms) {
  if (!S || !out) return fail(QAOA_ERR_INVALID_ARG, "server_wait: NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return fail(QAOA_ERR_NOT_FOUND, "server_wait: unknown ticket");
  Job *j = it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (j->state != kDone) {
    if (timeout_ms >= 0) {
      if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && j->state != kDone)
        return fail(QAOA_ERR_TIMEOUT, "server_wait: timed out");
    } else {
      S->cv_done.wait(lk);
    }
  }
  out->status = j->status;
  out->energy = j->result.size() >= 1 ? j->result[0] : NAN;
  out->overlap = j->result.size() >= 2 ? j->result[1] : NAN;
  out->submit_s = j->t_submit;
  out->admit_s = j->t_admit;
  out->finish_s = j->t_finish;
  if (j->status == QAOA_OK && j->want_grad && j->result.size() >= 2 + 2 * (size_t)j->p) {
    if (h_dgamma) memcpy(h_dgamma, j->result.data() + 2, sizeof(double) * j->p);
    if (h_dbeta) memcpy(h_dbeta, j->result.data() + 2 + j->p, sizeof(double) * j->p);
  }
  S->jobs.erase(it);
  delete j;
  return QAOA_OK;
}

qaoa_status qaoa_server_cancel(qaoa_server *S, uint64_t ticket) {
  if (!S) return fail(QAOA_ERR_INVALID_ARG, "server_cancel: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return fail(QAOA_ERR_NOT_FOUND, "server_cancel: unknown ticket");
  Job *j = it->second;
  if (j->state == kPending) {
    S->pending.erase(std::find(S->pending.begin(), S->pending.end(), j));
    j->state = kDone;
    j->status = QAOA_ERR_CANCELLED;
    j->t_finish = now_s();
    S->n_cancelled += 1;
    S->cv_done.notify_all();
  } else if (j->state == kRunning) {
    j->cancelled = true;  // the GPU work finishes; its result is dropped
  }
  return QAOA_OK;
}

qaoa_status qaoa_server_stats(qaoa_server *S, qaoa_server_stats_t *out) {
  if (!S || !out) return fail(QAOA_ERR_INVALID_ARG, "server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = S->n_submitted;
  out->completed = S->n_completed;
  out->rejected = S->n_rejected;
  out->cancelled = S->n_cancelled;
  std::vector<double> lat = S->latencies;
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
      const size_t i = (size_t)std::min<double>(lat.size() - 1, std::floor(q * (lat.size() - 1) + 0.5));
      return lat[i] * 1000.0;
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    const double span = S->last_finish - S->first_submit;
    out->evals_per_s = span > 0 ? (double)S->n_completed / span : 0.0;
  }
  out->arena_bytes = S->arena.size;
  out->arena_peak_bytes = S->arena.peak;
  out->cached_cost_vectors = S->costs.size();
  return QAOA_OK;
}

qaoa_status qaoa_server_destroy(qaoa_server *S) {
  if (!S) return QAOA_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  for (Unit &U : S->units) {
    if (U.stream) cudaStreamSynchronize(U.stream);
    if (U.done) cudaEventDestroy(U.done);
    if (U.stream) cudaStreamDestroy(U.stream);
    if (U.h_out) cudaFreeHost(U.h_out);
    if (U.h_stage) cudaFreeHost(U.h_stage);
  }
  for (auto &kv : S->jobs) delete kv.second;
  delete S;
  return QAOA_OK;
}

}  // extern "C"
