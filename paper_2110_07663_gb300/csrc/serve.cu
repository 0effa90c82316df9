// Solve server with continuous batching.
//
// Requests (a mesh description with a client-chosen key, a preconditioner description and a
// right-hand side) are queued at submission.  A scheduler thread admits them as slots and device
// memory free up: a request whose mesh is resident reuses it (geometry, FDM factors, Krylov work
// space and its captured solve graph stay on the device); otherwise the mesh is handed to a pool
// of builder threads if its estimated footprint fits the HBM budget (reserved while it is built),
// evicting idle resident meshes least recently used first.  The scheduler keeps admitting and
// completing while meshes are built, and a request for a key that is being built waits for it.
// Each admitted request launches its device-driven solve graph on its mesh's own non-blocking
// stream, so solves and set-ups of different requests overlap on the GPU; device memory is
// allocated and freed in stream order, so neither set-up nor eviction waits for other requests'
// work.  Completions are detected with events.  Latency = completion time - submission time.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pmg_internal.h"

namespace se {

using Clock = std::chrono::steady_clock;

static double now_ms() {
  return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count();
}

// Device bytes of a mesh + preconditioner + solve work space, from the allocation sizes of the
// code (per local point of each level, plus per-element FDM data and the coarse operator).
size_t footprint_bytes(const se_mesh_desc& d, const se_pmg_desc& pd) {
  const double E = (double)d.nel[0] * d.nel[1] * d.nel[2];
  const bool fp32 = pd.precision == SE_FP32;
  const double vec = fp32 ? 4.0 : 8.0;
  double total = 0.0, arnoldi_peak = 0.0;
  for (int l = 0; l < pd.nlev; ++l) {
    const int p = pd.schedule[l];
    const double N3 = (double)(p + 1) * (p + 1) * (p + 1), pb = p + 3.0;
    const double L = E * N3;
    // X 24, G 48, B 8, dinv 8 + 4, flags 1, QQ^T ids ~4, vectors 7 in the V-cycle precision
    double per_pt = 24 + 48 + 8 + 12 + 1 + 4 + 7 * vec;
    if (fp32 && l + 1 < pd.nlev) per_pt += 24;                  // FP32 geometric factors
    if (l == 0) per_pt += 5 * 8 + 8 + 8;                         // Krylov vectors, temporaries
    total += L * per_pt;
    if (l + 1 < pd.nlev && pd.smoother != SE_SMOOTH_JACOBI) {
      const double fdm = 3 * pb * pb * 8 + 3 * pb * 8 + pb * pb * pb * 8 +
                         (fp32 ? 3 * pb * pb * 4 + 3 * pb * 4 : 0) +
                         (pd.smoother == SE_SMOOTH_ASM ? pb * pb * pb * (8 + (fp32 ? 4 : 0)) : 0);
      total += E * fdm;
      arnoldi_peak = std::max(arnoldi_peak, (pd.arnoldi_steps + 3) * L * 8.0);
    }
    if (l + 1 == pd.nlev) {
      const double n = (d.nel[0] + 1.0) * (d.nel[1] + 1.0) * (d.nel[2] + 1.0);
      total += n * (27 * 8 + 8 + 4 + 9 * 8) + L * 4;
    }
  }
  total += E * 27 * 4 + 1024 * 1024;                               // neighbours, small buffers
  return (size_t)(total + arnoldi_peak);
}

struct Resident {
  uint64_t key = 0;
  se_mesh_t m = nullptr;
  se_pmg_t P = nullptr;
  se_proj_t proj = nullptr;    // prior solutions (server option)
  bool has_solution = false;   // x holds the last completed solve, not yet in proj
  double* b = nullptr;
  double* x = nullptr;
  size_t bytes = 0;
  bool busy = false;
  double last_used = 0.0;
  int64_t L = 0;
  int op_df = 0;               // outer operator in df64 (server option)
};

struct Ticket {
  uint64_t id = 0;
  se_request req{};
  std::vector<double> b_host;
  double t_submit = 0, t_start = 0, t_done = 0, setup_ms = 0;
  bool done = false, is_new_mesh = false;
  int status = SE_OK;
  int iterations = 0;
  double rel = 0.0;
  Resident* res = nullptr;
  cudaEvent_t ev = nullptr;
  int proj_size = 0;           // vectors in the mesh's projection space when the solve started
};

}  // namespace se

struct se_server_s {
  se_serve_cfg cfg{};
  std::mutex mu;
  std::condition_variable cv;
  std::thread thr;
  std::vector<std::thread> builders;
  std::deque<se::Ticket*> build_q;      // new meshes waiting for a builder
  std::vector<uint64_t> building_keys;  // keys being built (queued or in progress)
  int building = 0;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<se::Ticket*> queue;
  std::vector<se::Ticket*> running;
  std::unordered_map<uint64_t, se::Ticket*> tickets;
  std::vector<se::Resident*> residents;
  size_t used = 0;
  int64_t submitted = 0, completed = 0, refused = 0, failed = 0, created = 0, reused = 0,
          evicted = 0, projected = 0, cancelled = 0;
  int max_running = 0;
  double t_first = 0, t_last = 0;
  std::vector<double> latencies;
};

namespace se {

static void destroy_resident(Resident* r) {
  if (r->proj) se_proj_destroy(r->proj);
  if (r->P) se_pmg_destroy(r->P);
  if (r->m) {
    if (r->b) cudaFreeAsync(r->b, r->m->stream);
    if (r->x) cudaFreeAsync(r->x, r->m->stream);
    se_mesh_destroy(r->m);
  }
  delete r;
}

// Frees idle residents (least recently used first) until `need` more bytes fit the budget.
static bool make_room(se_server_s* S, size_t need) {
  while (S->used + need > S->cfg.hbm_budget) {
    Resident* victim = nullptr;
    for (Resident* r : S->residents)
      if (!r->busy && (!victim || r->last_used < victim->last_used)) victim = r;
    if (!victim) return false;
    S->residents.erase(std::find(S->residents.begin(), S->residents.end(), victim));
    S->used -= victim->bytes;
    destroy_resident(victim);
    ++S->evicted;
  }
  return true;
}

// Device bytes of a request's mesh as this server keeps it (with its projection space).
static size_t need_bytes(const se_server_s* S, const se_request& q) {
  const double L = (double)q.mesh.nel[0] * q.mesh.nel[1] * q.mesh.nel[2] * (q.mesh.p + 1) *
                   (q.mesh.p + 1) * (q.mesh.p + 1);
  const bool df = S->cfg.operator_df64 != 0;
  return footprint_bytes(q.mesh, q.pmg) + (size_t)(2.0 * S->cfg.proj_vectors * L * sizeof(double)) +
         (size_t)(df ? 6.0 * L * sizeof(df64) : 0.0);
}

static int build_resident(const se_request& q, int proj_vectors, int op_df, Resident** out) {
  se_mesh_desc d = q.mesh;
  d.flags |= SE_MESH_NONBLOCKING_STREAM;
  auto* r = new Resident();
  r->key = q.mesh_key;
  int rc = se_mesh_create(&d, &r->m);
  if (rc == SE_OK) rc = se_pmg_setup(r->m, &q.pmg, &r->P);
  if (rc == SE_OK) {
    r->L = r->m->fine.L;
    if (dmalloc_transient(reinterpret_cast<void**>(&r->b), r->L * sizeof(double), r->m->stream) != SE_OK ||
        dmalloc_transient(reinterpret_cast<void**>(&r->x), r->L * sizeof(double), r->m->stream) != SE_OK) {
      set_error("server: out of device memory for a request's vectors");
      rc = SE_ENOMEM;
    }
  }
  if (rc == SE_OK && proj_vectors > 0) rc = se_proj_create(r->m, proj_vectors, &r->proj);
  if (rc == SE_OK && op_df) {
    rc = make_df_geometry(r->m->fine, r->m->allocs, r->m->stream);
    r->op_df = 1;
  }
  if (rc != SE_OK) {
    destroy_resident(r);
    return rc;
  }
  r->bytes = r->m->allocs.bytes + r->P->allocs.bytes + 2 * r->L * sizeof(double) +
             (size_t)(r->proj ? 2.0 * proj_vectors * r->L * sizeof(double) : 0.0);
  *out = r;
  return SE_OK;
}

static int start_ticket(Ticket* t) {
  Resident* r = t->res;
  cudaStream_t s = r->m->stream;
  if (r->proj && r->has_solution) {  // the previous request's solution joins the space
    SE_TRY(se_proj_update(r->proj, r->x, &t->proj_size, s));
    r->has_solution = false;
  }
  if (t->req.rhs_kind == SE_RHS_HOST) {
    SE_CUDA(cudaMemcpyAsync(r->b, t->b_host.data(), r->L * sizeof(double), cudaMemcpyHostToDevice, s));
  } else {
    SE_TRY(rhs_modes(r->m, t->req.modes, t->req.amplitude, r->b, s));
  }
  if (r->proj) {
    SE_TRY(se_proj_guess(r->proj, r->b, r->x, s));
  } else {
    SE_CUDA(cudaMemsetAsync(r->x, 0, r->L * sizeof(double), s));
  }
  SE_TRY(graph_solve_launch(r->m, r->P, r->b, r->x, t->req.tol, t->req.maxit, s,
                            r->proj ? SE_TOL_B : SE_TOL_R0, r->op_df));
  if (!t->ev) SE_CUDA(cudaEventCreateWithFlags(&t->ev, cudaEventDisableTiming));
  SE_CUDA(cudaEventRecord(t->ev, s));
  return SE_OK;
}

static void finish_ticket(se_server_s* S, Ticket* t) {
  Resident* r = t->res;
  se_solve_stats st{};
  int rc = graph_solve_result(r->m, r->m->stream, t->req.tol, t->req.maxit, &st);
  if (level_pipeline_take(r->m->fine, r->m->stream) != SE_OK) rc = SE_ETIMEOUT;
  if (pmg_faults_take(r->P, r->m->stream) != SE_OK) rc = SE_ETIMEOUT;
  if (t->req.x_host && rc != SE_ECUDA)
    if (cudaMemcpy(t->req.x_host, r->x, r->L * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = SE_ECUDA;
  t->status = rc;
  t->iterations = st.iterations;
  t->rel = st.rel_residual;
  t->t_done = now_ms();
  t->done = true;
  r->busy = false;
  r->has_solution = r->proj && rc == SE_OK;
  if (t->proj_size > 0) ++S->projected;
  r->last_used = t->t_done;
  if (rc == SE_OK) {
    ++S->completed;
    S->latencies.push_back(t->t_done - t->t_submit);
  } else {
    ++S->failed;
  }
  S->t_last = t->t_done;
  if (t->ev) {
    cudaEventDestroy(t->ev);
    t->ev = nullptr;
  }
}

static void scheduler(se_server_s* S) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    bool progress = false;
    // completions
    for (size_t i = 0; i < S->running.size();) {
      Ticket* t = S->running[i];
      if (cudaEventQuery(t->ev) == cudaSuccess) {
        finish_ticket(S, t);
        S->running.erase(S->running.begin() + i);
        progress = true;
      } else {
        ++i;
      }
    }
    if (progress) S->cv.notify_all();
    // admissions (in arrival order; a request whose mesh is busy or being built waits without
    // blocking others)
    size_t qi = 0;
    while (qi < S->queue.size() && (int)S->running.size() + S->building < S->cfg.max_slots) {
      Ticket* t = S->queue[qi];
      Resident* r = nullptr;
      for (Resident* x : S->residents)
        if (x->key == t->req.mesh_key) r = x;
      const bool key_building = std::find(S->building_keys.begin(), S->building_keys.end(),
                                          t->req.mesh_key) != S->building_keys.end();
      if ((r && r->busy) || key_building) {
        ++qi;
        continue;
      }
      if (!r) {
        const size_t need = need_bytes(S, t->req);
        if (!make_room(S, need)) break;  // wait for memory to free up
        S->queue.erase(S->queue.begin() + qi);
        S->used += need;                 // reserved while the mesh is built
        ++S->building;
        S->building_keys.push_back(t->req.mesh_key);
        S->build_q.push_back(t);
        S->cv.notify_all();
        progress = true;
        continue;
      }
      S->queue.erase(S->queue.begin() + qi);
      ++S->reused;
      r->busy = true;
      t->res = r;
      t->t_start = now_ms();
      int rc = start_ticket(t);
      if (rc != SE_OK) {
        t->status = rc;
        t->done = true;
        t->t_done = now_ms();
        r->busy = false;
        ++S->failed;
        S->cv.notify_all();
        progress = true;
        continue;
      }
      S->running.push_back(t);
      S->max_running = std::max(S->max_running, (int)S->running.size());
      progress = true;
    }
    if (!progress) {
      // nothing to do now: wait for a submission, or poll the running solves shortly
      S->cv.wait_for(lk, std::chrono::microseconds(S->running.empty() ? 2000 : 50));
    }
  }
  (void)dev;
}

// Builds the meshes of queued requests (set-up kernels on the new mesh's own stream), starts
// their solves, and hands them to the scheduler's running list.
static void builder(se_server_s* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv.wait(lk, [S] { return S->stop || !S->build_q.empty(); });
    if (S->build_q.empty()) break;  // stopping, nothing left to build
    Ticket* t = S->build_q.front();
    S->build_q.pop_front();
    const size_t need = need_bytes(S, t->req);
    lk.unlock();
    const double tb = now_ms();
    Resident* r = nullptr;
    int rc = build_resident(t->req, S->cfg.proj_vectors, S->cfg.operator_df64, &r);
    t->setup_ms = now_ms() - tb;
    if (rc == SE_OK) {
      // not yet visible to the scheduler: its first solve starts outside the lock
      r->busy = true;
      t->res = r;
      t->t_start = now_ms();
      rc = start_ticket(t);
      if (rc != SE_OK) r->busy = false;
    }
    lk.lock();
    S->used -= need;
    --S->building;
    auto it = std::find(S->building_keys.begin(), S->building_keys.end(), t->req.mesh_key);
    if (it != S->building_keys.end()) S->building_keys.erase(it);
    if (r) {
      S->residents.push_back(r);
      S->used += r->bytes;
      ++S->created;
      t->is_new_mesh = true;
    }
    if (rc != SE_OK) {
      t->status = rc;
      t->done = true;
      t->t_done = now_ms();
      ++S->failed;
    } else {
      S->running.push_back(t);
      S->max_running = std::max(S->max_running, (int)S->running.size());
    }
    S->cv.notify_all();
  }
}

}  // namespace se

using namespace se;

extern "C" {

int se_mesh_footprint_bytes(const se_mesh_desc* desc, const se_pmg_desc* pmg, size_t* out) {
  SE_CHECK(desc && pmg && out, SE_EINVAL, "se_mesh_footprint_bytes: null argument");
  *out = footprint_bytes(*desc, *pmg);
  return SE_OK;
}

int se_serve_create(const se_serve_cfg* cfg, se_server_t* out) {
  SE_CHECK(cfg && out, SE_EINVAL, "se_serve_create: null argument");
  SE_CHECK(cfg->max_slots >= 1 && cfg->max_slots <= 256, SE_EINVAL, "se_serve_create: max_slots");
  SE_CHECK(cfg->builders >= 0 && cfg->builders <= 64, SE_EINVAL, "se_serve_create: builders");
  SE_CHECK(cfg->proj_vectors >= 0 && cfg->proj_vectors <= 16, SE_EINVAL,
           "se_serve_create: proj_vectors");
  SE_CHECK(cfg->operator_df64 == 0 || cfg->operator_df64 == 1, SE_EINVAL,
           "se_serve_create: operator_df64");
  SE_CHECK(cfg->hbm_budget > 0, SE_EINVAL, "se_serve_create: hbm_budget");
  auto* S = new se_server_s();
  S->cfg = *cfg;
  int dev = 0;
  cudaGetDevice(&dev);
  const int nb = cfg->builders > 0 ? cfg->builders : std::min(4, cfg->max_slots);
  S->thr = std::thread([S, dev] {
    cudaSetDevice(dev);
    scheduler(S);
  });
  for (int i = 0; i < nb; ++i)
    S->builders.emplace_back([S, dev] {
      cudaSetDevice(dev);
      builder(S);
    });
  *out = S;
  return SE_OK;
}

int se_serve_submit(se_server_t S, const se_request* req, uint64_t* ticket) {
  SE_CHECK(S && req && ticket, SE_EINVAL, "se_serve_submit: null argument");
  const se_request& q = *req;
  bool ok = q.mesh.p >= 1 && q.mesh.p <= SE_MAX_ORDER && q.mesh.nel[0] >= 1 && q.mesh.nel[1] >= 1 &&
            q.mesh.nel[2] >= 1 && q.tol > 0 && q.maxit >= 1 && q.pmg.nlev >= 2 &&
            q.pmg.schedule[0] == q.mesh.p && (q.rhs_kind == SE_RHS_MODES || q.rhs_kind == SE_RHS_HOST);
  if (ok && q.rhs_kind == SE_RHS_HOST) ok = q.b_host != nullptr;
  SE_CHECK(ok, SE_EINVAL, "se_serve_submit: malformed request");
  const double t_arrival = now_ms();
  const size_t need = need_bytes(S, q);
  std::lock_guard<std::mutex> g(S->mu);
  ++S->submitted;
  if (need > S->cfg.hbm_budget) {
    ++S->refused;
    set_error("se_serve_submit: request needs about %zu bytes, above the budget of %zu", need,
              S->cfg.hbm_budget);
    return SE_EREFUSED;
  }
  auto* t = new Ticket();
  t->id = S->next_id++;
  t->req = q;
  if (q.rhs_kind == SE_RHS_HOST) {
    const int64_t L = (int64_t)q.mesh.nel[0] * q.mesh.nel[1] * q.mesh.nel[2] * (q.mesh.p + 1) *
                      (q.mesh.p + 1) * (q.mesh.p + 1);
    t->b_host.assign(q.b_host, q.b_host + L);
    t->req.b_host = nullptr;
  }
  t->t_submit = t_arrival;
  if (S->t_first == 0) S->t_first = t->t_submit;
  S->tickets[t->id] = t;
  S->queue.push_back(t);
  S->cv.notify_all();
  *ticket = t->id;
  return SE_OK;
}

static void fill_result(const Ticket* t, se_result* r) {
  r->status = t->status;
  r->iterations = t->iterations;
  r->rel_residual = t->rel;
  r->latency_ms = t->t_done - t->t_submit;
  r->queue_ms = (t->t_start > 0 ? t->t_start : t->t_done) - t->t_submit;
  r->new_mesh = t->is_new_mesh ? 1 : 0;
  r->setup_ms = t->setup_ms;
  r->solve_ms = t->t_start > 0 ? t->t_done - t->t_start : 0.0;
}

int se_serve_poll(se_server_t S, uint64_t ticket, se_result* res) {
  SE_CHECK(S && res, SE_EINVAL, "se_serve_poll: null argument");
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->tickets.find(ticket);
  SE_CHECK(it != S->tickets.end(), SE_EINVAL, "se_serve_poll: unknown ticket %llu",
           (unsigned long long)ticket);
  if (!it->second->done) return SE_EBUSY;
  fill_result(it->second, res);
  return it->second->status;
}

int se_serve_wait(se_server_t S, uint64_t ticket, double timeout_ms, se_result* res) {
  SE_CHECK(S && res, SE_EINVAL, "se_serve_wait: null argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  SE_CHECK(it != S->tickets.end(), SE_EINVAL, "se_serve_wait: unknown ticket %llu",
           (unsigned long long)ticket);
  Ticket* t = it->second;
  const auto deadline = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1000));
  while (!t->done) {
    if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout && !t->done) {
      set_error("se_serve_wait: ticket %llu still pending after %.1f ms",
                (unsigned long long)ticket, timeout_ms);
      return SE_ETIMEOUT;
    }
  }
  fill_result(t, res);
  return t->status;
}

int se_serve_cancel(se_server_t S, uint64_t ticket) {
  SE_CHECK(S, SE_EINVAL, "se_serve_cancel: null server");
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->tickets.find(ticket);
  SE_CHECK(it != S->tickets.end(), SE_EINVAL, "se_serve_cancel: unknown ticket %llu",
           (unsigned long long)ticket);
  Ticket* t = it->second;
  SE_CHECK(!t->done, SE_EINVAL, "se_serve_cancel: ticket %llu has finished", (unsigned long long)ticket);
  auto q = std::find(S->queue.begin(), S->queue.end(), t);
  if (q == S->queue.end()) {
    set_error("se_serve_cancel: ticket %llu has started", (unsigned long long)ticket);
    return SE_EBUSY;  // being built or solved: it completes normally
  }
  S->queue.erase(q);
  t->status = SE_ECANCELED;
  t->t_done = now_ms();
  t->done = true;
  ++S->cancelled;
  S->cv.notify_all();
  return SE_OK;
}

int se_serve_stats(se_server_t S, se_serve_summary* out) {
  SE_CHECK(S && out, SE_EINVAL, "se_serve_stats: null argument");
  std::lock_guard<std::mutex> g(S->mu);
  std::vector<double> lat = S->latencies;
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double q) {
    if (lat.empty()) return 0.0;
    size_t i = (size_t)std::ceil(q * lat.size()) - 1;
    return lat[std::min(i, lat.size() - 1)];
  };
  double mean = 0.0;
  for (double v : lat) mean += v;
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->refused = S->refused;
  out->failed = S->failed;
  out->pending = (int64_t)S->queue.size() + (int64_t)S->running.size() + S->building;
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  out->mean_ms = lat.empty() ? 0.0 : mean / lat.size();
  const double span = S->t_last - S->t_first;
  out->solves_per_s = span > 0 ? S->completed / (span * 1e-3) : 0.0;
  out->max_concurrent = S->max_running;
  out->meshes_created = S->created;
  out->mesh_reuses = S->reused;
  out->evictions = S->evicted;
  out->resident_bytes = S->used;
  out->projected = S->projected;
  out->cancelled = S->cancelled;
  return SE_OK;
}

int se_serve_destroy(se_server_t S) {
  if (!S) return SE_OK;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  for (auto& b : S->builders) b.join();  // builders finish the meshes already handed to them
  S->thr.join();
  for (Ticket* t : S->running) cudaEventSynchronize(t->ev);
  for (auto& kv : S->tickets) {
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    delete kv.second;
  }
  for (Resident* r : S->residents) destroy_resident(r);
  delete S;
  return SE_OK;
}

}  // extern "C"
