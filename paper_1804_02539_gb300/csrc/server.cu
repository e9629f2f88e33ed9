// Serving layer: many requests (a model = one multi-patch problem, a request = one
// right-hand side of a model) answered by a pool of worker threads with a CUDA stream
// each.  Hierarchies stay resident between requests of the same model, under a device
// memory budget: a model without a resident hierarchy is admitted (set up) only when its
// estimated footprint fits, after evicting least-recently-used idle hierarchies; requests
// wait in arrival order, and a worker takes the oldest request whose model is not in use by
// another worker (continuous batching: a freed worker starts the next request at once, so
// requests of different models run concurrently on the device).  For a model the lockstep
// engine covers, the worker also takes that model's other waiting requests of the same
// tolerance (up to kMaxGroup in all) and solves them together with igamg_solve_multi: one
// launch per step of the cycle for the whole group, the hierarchy's constant arrays shared.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/igamg.h"
#include "host_math.h"
#include "topology.h"

namespace igamg {
void set_context_free_error(const std::string& msg);
void ctx_set_stream(igamg_ctx* c, cudaStream_t s);
size_t ctx_device_bytes(const igamg_ctx* c);
bool ctx_multi_ok(const igamg_ctx* c);
bool rect_metric(const double* X, double* c0, double* c1);
}  // namespace igamg

namespace {

constexpr size_t kMaxGroup = 16;  // requests of one model solved together at most

struct ProblemCopy {  // owns the arrays an igamg_problem points to
  std::vector<int> degree, num_knots, geo_degree, geo_num_ctrl, side_bc;
  std::vector<double> knots, geo_ctrl;
  igamg_problem view{};
  void take(const igamg_problem& p) {
    const int Kd = p.num_patches * p.dim;
    degree.assign(p.degree, p.degree + Kd);
    num_knots.assign(p.num_knots, p.num_knots + Kd);
    geo_degree.assign(p.geo_degree, p.geo_degree + Kd);
    geo_num_ctrl.assign(p.geo_num_ctrl, p.geo_num_ctrl + Kd);
    side_bc.assign(p.side_bc, p.side_bc + 2 * Kd);
    size_t nk = 0, nc = 0;
    for (int i = 0; i < p.num_patches; ++i) {
      size_t ctrl = 1;
      for (int j = 0; j < p.dim; ++j) {
        nk += size_t(p.num_knots[i * p.dim + j]);
        ctrl *= size_t(p.geo_num_ctrl[i * p.dim + j]);
      }
      nc += ctrl * p.dim;
    }
    knots.assign(p.knots, p.knots + nk);
    geo_ctrl.assign(p.geo_ctrl, p.geo_ctrl + nc);
    view = p;
    view.degree = degree.data();
    view.num_knots = num_knots.data();
    view.knots = knots.data();
    view.geo_degree = geo_degree.data();
    view.geo_num_ctrl = geo_num_ctrl.data();
    view.geo_ctrl = geo_ctrl.data();
    view.side_bc = side_bc.data();
  }
};

struct Model {
  ProblemCopy prob;
  int64_t ndofs = 0;
  size_t est_bytes = 0;  // admission estimate before the first setup, then the measured size
  igamg_ctx* ctx = nullptr;
  bool busy = false, building = false;
  bool multi = false;  // igamg_solve_multi runs its requests in lockstep
  uint64_t last_use = 0;
};

struct Request {
  int model;
  const double* b;
  double* x;
  double tol;
  igamg_request_info info{};
  bool done = false;
};

struct Worker {
  cudaStream_t stream = nullptr;
  double *hb = nullptr, *hx = nullptr, *db = nullptr, *dx = nullptr;  // pinned / device staging
  int64_t cap = 0;
};

}  // namespace

struct igamg_server {
  igamg_options opt{};
  int64_t budget = 0, used = 0;
  std::vector<std::unique_ptr<Model>> models;
  std::unordered_map<int64_t, Request> reqs;
  std::deque<int64_t> queue;  // waiting requests, arrival order
  int64_t next_id = 0;
  uint64_t tick = 0;
  int64_t setups = 0, evictions = 0, completed = 0, groups = 0, grouped = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int dev = 0;
  std::vector<Worker> workers;
  std::vector<std::thread> threads;
  std::chrono::steady_clock::time_point t0;
  double now() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Device bytes of a hierarchy, estimated from the level topologies: vectors, maps, FD and
// transfer work arrays (~80 B per tile node, 40 B more on the finest level for the PCG
// vectors), band coefficients ((2p+1)^d doubles per node; none above the coarsest level
// when every 2D patch is a rectangle), the dense coarse inverse, and ~1.6x that for the
// precision variant's twins.
int64_t estimate_bytes(const igamg_problem& p, const igamg_options& opt, int64_t* ndofs, std::string* err) {
  igamg::ProblemDesc pd;
  int code = 0;
  std::string e = igamg::parse_problem(p.dim, p.num_patches, p.degree, p.num_knots, p.knots, p.geo_degree,
                                       p.geo_num_ctrl, p.geo_ctrl, p.side_bc, p.num_levels, pd, &code);
  if (!e.empty()) {
    *err = e;
    return -1;
  }
  bool kron = pd.dim == 2 && opt.apply_engine == 0;
  for (int k = 0; k < pd.K && kron; ++k) {
    double c0, c1;
    kron = igamg::rect_metric(pd.corners.data() + size_t(k) * 8, &c0, &c1);
  }
  int pmax = 1;
  for (int q : pd.p) pmax = std::max(pmax, q);
  const double band = 8.0 * std::pow(2.0 * pmax + 1.0, pd.dim);
  double total = 1 << 20;
  for (int l = 0; l < pd.levels; ++l) {
    igamg::LevelTopo T;
    e = igamg::build_level(pd, l, T, &code);
    if (!e.empty()) {
      *err = e;
      return -1;
    }
    double per_node = 80.0 + ((kron && l > 0) ? 1.0 : band) + (l == pd.levels - 1 ? 40.0 : 0.0);
    total += double(T.T) * per_node;
    if (l == 0) total += 8.0 * double(T.N) * double(T.N);
    if (l == pd.levels - 1) *ndofs = T.N;
  }
  if (opt.precision != IGAMG_FP64) total *= 1.6;
  return int64_t(total);
}

void ensure_staging(Worker& w, int64_t n) {
  if (n <= w.cap) return;
  if (w.hb) cudaFreeHost(w.hb);
  if (w.hx) cudaFreeHost(w.hx);
  if (w.db) cudaFree(w.db);
  if (w.dx) cudaFree(w.dx);
  w.hb = w.hx = w.db = w.dx = nullptr;
  w.cap = 0;
  if (cudaMallocHost(&w.hb, n * sizeof(double)) != cudaSuccess || cudaMallocHost(&w.hx, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&w.db, n * sizeof(double)) != cudaSuccess || cudaMalloc(&w.dx, n * sizeof(double)) != cudaSuccess)
    return;
  w.cap = n;
}

// Solve of a group of requests of one model (one request: igamg_solve; more: together by
// igamg_solve_multi) on worker w (model hierarchy resident and reserved for it).
void run_group(Worker& w, Model& m, const std::vector<Request*>& rs) {
  const int64_t n = m.ndofs;
  const int g = int(rs.size());
  ensure_staging(w, n * g);
  if (g > 1 && w.cap < n * g) {  // no staging for the whole group: one request at a time
    for (Request* r : rs) run_group(w, m, std::vector<Request*>{r});
    return;
  }
  std::vector<igamg_result> res(static_cast<size_t>(g), igamg_result{});
  std::vector<igamg_status> sts(static_cast<size_t>(g), IGAMG_ERR_OOM);
  if (w.cap >= n * g) {
    std::vector<const double*> bp(static_cast<size_t>(g), nullptr);
    std::vector<double*> xp(static_cast<size_t>(g), nullptr);
    for (int i = 0; i < g; ++i) {
      std::memcpy(w.hb + i * n, rs[i]->b, n * sizeof(double));
      bp[i] = w.db + i * n;
      xp[i] = w.dx + i * n;
    }
    cudaMemcpyAsync(w.db, w.hb, g * n * sizeof(double), cudaMemcpyHostToDevice, w.stream);
    cudaMemsetAsync(w.dx, 0, g * n * sizeof(double), w.stream);
    igamg::ctx_set_stream(m.ctx, w.stream);
    igamg_status st;
    if (g == 1) st = sts[0] = igamg_solve(m.ctx, bp[0], xp[0], rs[0]->tol, &res[0]);
    else st = igamg_solve_multi(m.ctx, g, bp.data(), xp.data(), rs[0]->tol, res.data(), sts.data());
    cudaMemcpyAsync(w.hx, w.dx, g * n * sizeof(double), cudaMemcpyDeviceToHost, w.stream);
    if (cudaStreamSynchronize(w.stream) != cudaSuccess && st == IGAMG_OK)
      for (auto& x : sts) x = IGAMG_ERR_CUDA;
    for (int i = 0; i < g; ++i) std::memcpy(rs[i]->x, w.hx + i * n, n * sizeof(double));
  }
  for (int i = 0; i < g; ++i) {
    rs[i]->info.status = sts[i];
    rs[i]->info.iters = res[i].iters;
    rs[i]->info.relres = res[i].relres;
    rs[i]->info.group = g;
  }
}

// Frees least-recently-used idle hierarchies until `need` more bytes fit the budget.
bool make_room(igamg_server* S, int64_t need) {
  while (S->used + need > S->budget) {
    Model* victim = nullptr;
    for (auto& m : S->models)
      if (m->ctx && !m->busy && !m->building && (!victim || m->last_use < victim->last_use)) victim = m.get();
    if (!victim) return false;
    igamg_free(victim->ctx);
    victim->ctx = nullptr;
    S->used -= int64_t(victim->est_bytes);
    ++S->evictions;
  }
  return true;
}

void worker_main(igamg_server* S, int wi) {
  cudaSetDevice(S->dev);
  igamg::set_host_threads(1);
  Worker& w = S->workers[wi];
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    if (S->stop) return;
    // requests of a model that can never fit the budget fail at once
    for (auto it = S->queue.begin(); it != S->queue.end();) {
      Request& r = S->reqs[*it];
      const Model& m = *S->models[r.model];
      if (!m.ctx && !m.building && int64_t(m.est_bytes) > S->budget) {
        r.info.status = IGAMG_ERR_OOM;
        r.info.t_start_ms = r.info.t_done_ms = S->now();
        r.done = true;
        ++S->completed;
        it = S->queue.erase(it);
        S->cv_done.notify_all();
      } else {
        ++it;
      }
    }
    // the oldest request whose model is idle and resident, or admissible after evictions
    auto pick = S->queue.end();
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
      const Model& m = *S->models[S->reqs[*it].model];
      if (m.busy || m.building) continue;
      if (m.ctx || make_room(S, int64_t(m.est_bytes))) {
        pick = it;
        break;
      }
    }
    if (pick == S->queue.end()) {
      S->cv_work.wait(lk);
      continue;
    }
    const int64_t id = *pick;
    S->queue.erase(pick);
    Request& r = S->reqs[id];
    Model& m = *S->models[r.model];
    r.info.t_start_ms = S->now();
    if (!m.ctx) {  // admit: reserve the estimate, build outside the lock
      m.building = true;
      S->used += int64_t(m.est_bytes);
      lk.unlock();
      double t0 = S->now();
      igamg_ctx* ctx = nullptr;
      igamg_status st = igamg_setup(&m.prob.view, &S->opt, w.stream, &ctx);
      double t1 = S->now();
      lk.lock();
      m.building = false;
      r.info.setup_ms = t1 - t0;
      if (st != IGAMG_OK) {
        S->used -= int64_t(m.est_bytes);
        r.info.status = st;
        r.info.t_done_ms = S->now();
        r.done = true;
        ++S->completed;
        S->cv_done.notify_all();
        S->cv_work.notify_all();
        continue;
      }
      ++S->setups;
      const int64_t actual = int64_t(igamg::ctx_device_bytes(ctx));
      S->used += actual - int64_t(m.est_bytes);
      m.est_bytes = size_t(actual);
      m.ctx = ctx;
      m.multi = igamg::ctx_multi_ok(ctx);
    }
    std::vector<Request*> grp{&r};
    if (m.multi) {  // the model's other waiting requests of the same tolerance, oldest first
      const double t_take = S->now();
      for (auto it = S->queue.begin(); it != S->queue.end() && grp.size() < kMaxGroup;) {
        Request& q = S->reqs[*it];
        if (q.model == r.model && q.tol == r.tol) {
          q.info.t_start_ms = t_take;
          grp.push_back(&q);
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    m.busy = true;
    lk.unlock();
    run_group(w, m, grp);
    lk.lock();
    m.busy = false;
    m.last_use = ++S->tick;
    const int64_t now_bytes = int64_t(igamg::ctx_device_bytes(m.ctx));  // work copies made for the group
    S->used += now_bytes - int64_t(m.est_bytes);
    m.est_bytes = size_t(now_bytes);
    const double t_done = S->now();
    for (Request* q : grp) {
      q->info.t_done_ms = t_done;
      q->done = true;
      ++S->completed;
    }
    if (grp.size() > 1) {
      ++S->groups;
      S->grouped += int64_t(grp.size());
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

igamg_status igamg_server_create(const igamg_options* opt, int workers, int64_t hbm_budget_bytes,
                                 igamg_server** out) {
  if (!out || workers < 1 || hbm_budget_bytes <= 0) {
    igamg::set_context_free_error("igamg_server_create: need out != NULL, workers >= 1, budget > 0");
    return IGAMG_ERR_ARG;
  }
  igamg_server* S = new igamg_server();
  if (opt) S->opt = *opt;
  else igamg_default_options(&S->opt);
  S->budget = hbm_budget_bytes;
  S->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&S->dev);
  S->workers.resize(workers);
  for (auto& w : S->workers)
    if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& v : S->workers)
        if (v.stream) cudaStreamDestroy(v.stream);
      delete S;
      igamg::set_context_free_error("igamg_server_create: cannot create worker streams");
      return IGAMG_ERR_CUDA;
    }
  for (int i = 0; i < workers; ++i) S->threads.emplace_back(worker_main, S, i);
  *out = S;
  return IGAMG_OK;
}

igamg_status igamg_server_add_model(igamg_server* S, const igamg_problem* prob, int* model, int64_t* num_dofs,
                                    int64_t* est_bytes) {
  if (!S || !prob || !model) return IGAMG_ERR_ARG;
  auto m = std::make_unique<Model>();
  m->prob.take(*prob);
  std::string err;
  int64_t est = estimate_bytes(m->prob.view, S->opt, &m->ndofs, &err);
  if (est < 0) {
    igamg::set_context_free_error("igamg_server_add_model: " + err);
    return IGAMG_ERR_ARG;
  }
  m->est_bytes = size_t(est);
  std::lock_guard<std::mutex> lk(S->mu);
  *model = int(S->models.size());
  if (num_dofs) *num_dofs = m->ndofs;
  if (est_bytes) *est_bytes = int64_t(m->est_bytes);
  S->models.push_back(std::move(m));
  return IGAMG_OK;
}

igamg_status igamg_server_submit(igamg_server* S, int model, const double* rhs, double* x, double tol,
                                 int64_t* request) {
  if (!S || !rhs || !x || !request || !(tol >= 0)) return IGAMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (model < 0 || model >= int(S->models.size())) return IGAMG_ERR_ARG;
  const int64_t id = S->next_id++;
  Request& r = S->reqs[id];
  r.model = model;
  r.b = rhs;
  r.x = x;
  r.tol = tol;
  r.info.t_submit_ms = S->now();
  r.info.group = 1;
  S->queue.push_back(id);
  S->cv_work.notify_one();
  *request = id;
  return IGAMG_OK;
}

igamg_status igamg_server_wait(igamg_server* S, int64_t request, igamg_request_info* info) {
  if (!S) return IGAMG_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(request);
  if (it == S->reqs.end()) return IGAMG_ERR_ARG;
  S->cv_done.wait(lk, [&] { return it->second.done; });
  if (info) *info = it->second.info;
  S->reqs.erase(it);
  return IGAMG_OK;
}

igamg_status igamg_server_stats(igamg_server* S, igamg_server_counters* st) {
  if (!S || !st) return IGAMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  st->models = int(S->models.size());
  st->resident = 0;
  for (auto& m : S->models) st->resident += m->ctx ? 1 : 0;
  st->device_bytes = S->used;
  st->setups = S->setups;
  st->evictions = S->evictions;
  st->completed = S->completed;
  st->waiting = int64_t(S->queue.size());
  st->groups = S->groups;
  st->grouped = S->grouped;
  return IGAMG_OK;
}

igamg_status igamg_server_free(igamg_server* S) {
  if (!S) return IGAMG_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->threads) t.join();
  for (auto& m : S->models)
    if (m->ctx) igamg_free(m->ctx);
  for (auto& w : S->workers) {
    if (w.stream) cudaStreamSynchronize(w.stream);
    if (w.hb) cudaFreeHost(w.hb);
    if (w.hx) cudaFreeHost(w.hx);
    if (w.db) cudaFree(w.db);
    if (w.dx) cudaFree(w.dx);
    if (w.stream) cudaStreamDestroy(w.stream);
  }
  delete S;
  return IGAMG_OK;
}

}  // extern "C"
