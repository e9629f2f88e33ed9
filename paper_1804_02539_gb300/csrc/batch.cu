// Batched solves of independent problems: one context per problem (its own hierarchy, kept
// resident).  When every problem is in its scope the lockstep engine (igamg.cu) solves them
// all at once, each step of the cycle one launch over every problem.  Otherwise a pool of
// host worker threads that each own a CUDA stream takes the problems in largest-first order
// (longest-processing-time list scheduling), lends each context its stream for the solve and
// returns it; those solves are the single-problem path (PCG iterations replayed as CUDA
// graphs), so their results are bit-identical to solving each problem alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/igamg.h"
#include "host_math.h"

namespace igamg {
void set_context_free_error(const std::string& msg);
cudaStream_t ctx_stream(const igamg_ctx* c);
void ctx_set_stream(igamg_ctx* c, cudaStream_t s);
double ctx_work_estimate(const igamg_ctx* c);
struct Lockstep;
Lockstep* lockstep_build(const std::vector<igamg_ctx*>& ctx, std::string* why);
igamg_status lockstep_solve(Lockstep* k, cudaStream_t s, const double* const* b, double* const* x, double tol,
                            igamg_result* res, igamg_status* status);
void lockstep_free(Lockstep* k);
void lockstep_stats(const Lockstep* k, int64_t* launches, double* flops, double* mma_flops);
}  // namespace igamg

struct igamg_batch {
  igamg::Lockstep* lock = nullptr;  // the lockstep engine, when every problem is in its scope
  std::vector<igamg_ctx*> ctx;
  std::vector<cudaStream_t> streams;  // one per worker
  std::vector<cudaEvent_t> done;      // one per worker
  cudaEvent_t start = nullptr;
  cudaStream_t user = nullptr;
  std::vector<int> order;  // largest estimated work first
};

namespace {

constexpr int kDefaultWorkers = 16;

void destroy(igamg_batch* b) {
  if (!b) return;
  if (b->user) cudaStreamSynchronize(b->user);
  igamg::lockstep_free(b->lock);
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  for (igamg_ctx* c : b->ctx)
    if (c) {
      igamg::ctx_set_stream(c, b->user);
      igamg_free(c);
    }
  for (cudaEvent_t e : b->done) cudaEventDestroy(e);
  if (b->start) cudaEventDestroy(b->start);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  delete b;
}

// Runs fn(worker, item) over items [0, n) on `workers` threads pulling from one counter.
template <class F>
void run_pool(int workers, int n, F&& fn) {
  std::atomic<int> next{0};
  std::vector<std::thread> th;
  th.reserve(workers);
  for (int w = 0; w < workers; ++w)
    th.emplace_back([&, w] {
      igamg::set_host_threads(1);  // the pool already keeps the cores busy
      for (int i = next++; i < n; i = next++) fn(w, i);
    });
  for (auto& t : th) t.join();
}

}  // namespace

extern "C" {

igamg_status igamg_setup_batch(const igamg_problem* problems, int count, const igamg_options* opt, int workers,
                               void* cuda_stream, igamg_batch** out) {
  if (!out) return IGAMG_ERR_ARG;
  *out = nullptr;
  if (!problems || count < 1) {
    igamg::set_context_free_error("igamg_setup_batch: need at least one problem");
    return IGAMG_ERR_ARG;
  }
  igamg_batch* b = new igamg_batch();
  b->user = static_cast<cudaStream_t>(cuda_stream);
  const int W = std::min(count, workers > 0 ? workers : kDefaultWorkers);
  b->ctx.assign(count, nullptr);
  for (int w = 0; w < W; ++w) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      destroy(b);
      igamg::set_context_free_error("igamg_setup_batch: cannot create worker streams");
      return IGAMG_ERR_CUDA;
    }
    b->streams.push_back(s);
    b->done.push_back(e);
  }
  if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
    destroy(b);
    igamg::set_context_free_error("igamg_setup_batch: cannot create events");
    return IGAMG_ERR_CUDA;
  }
  std::vector<igamg_status> st(count, IGAMG_OK);
  std::vector<std::string> msg(count);
  int dev = 0;
  cudaGetDevice(&dev);
  // Phase 1, one thread: the first problem of every (dim, patches, degree, knots, levels)
  // class, so that the FD autotuner times its candidates on an otherwise idle device and
  // caches the choices.  Phase 2, the pool: the rest, which find their choices cached.
  std::vector<int> first, rest;
  {
    std::map<std::vector<int>, int> seen;
    for (int i = 0; i < count; ++i) {
      const igamg_problem& p = problems[i];
      std::vector<int> key{p.dim, p.num_patches, p.num_levels, p.degree ? p.degree[0] : 0,
                           p.num_knots ? p.num_knots[0] : 0};
      if (seen.emplace(key, i).second) first.push_back(i);
      else rest.push_back(i);
    }
  }
  igamg::set_host_threads(0);
  for (int i : first) {
    st[i] = igamg_setup(&problems[i], opt, b->streams[0], &b->ctx[i]);
    if (st[i] != IGAMG_OK) msg[i] = igamg_last_error(nullptr);
  }
  run_pool(W, int(rest.size()), [&](int w, int k) {
    cudaSetDevice(dev);
    const int i = rest[k];
    st[i] = igamg_setup(&problems[i], opt, b->streams[w], &b->ctx[i]);
    if (st[i] != IGAMG_OK) msg[i] = igamg_last_error(nullptr);
  });
  for (int i = 0; i < count; ++i)
    if (st[i] != IGAMG_OK) {
      destroy(b);
      igamg::set_context_free_error("problem " + std::to_string(i) + ": " + msg[i]);
      return st[i];
    }
  for (igamg_ctx* c : b->ctx) igamg::ctx_set_stream(c, b->user);
  std::vector<double> work(count);
  for (int i = 0; i < count; ++i) work[i] = igamg::ctx_work_estimate(b->ctx[i]);
  b->order.resize(count);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return work[a] > work[c]; });
  if (!opt || opt->batch_engine == 0) {
    std::string why;
    b->lock = igamg::lockstep_build(b->ctx, &why);  // NULL: outside the lockstep scope
  }
  *out = b;
  return IGAMG_OK;
}

igamg_status igamg_batch_engine(igamg_batch* b, int* engine, int64_t* launches, double* flops, double* mma_flops) {
  if (!b || !engine) return IGAMG_ERR_ARG;
  *engine = b->lock ? 0 : 1;
  int64_t l = -1;
  double f = -1.0, m = -1.0;
  if (b->lock) igamg::lockstep_stats(b->lock, &l, &f, &m);
  if (launches) *launches = l;
  if (flops) *flops = f;
  if (mma_flops) *mma_flops = m;
  return IGAMG_OK;
}

igamg_status igamg_batch_context(igamg_batch* b, int i, igamg_ctx** ctx) {
  if (!b || !ctx || i < 0 || i >= int(b->ctx.size())) return IGAMG_ERR_ARG;
  *ctx = b->ctx[i];
  return IGAMG_OK;
}

igamg_status igamg_solve_batch(igamg_batch* b, const double* const* rhs, double* const* x, double tol,
                               igamg_result* res, igamg_status* status) {
  if (!b || !rhs || !x || !(tol >= 0)) return IGAMG_ERR_ARG;
  const int n = int(b->ctx.size()), W = int(b->streams.size());
  for (int i = 0; i < n; ++i)
    if (!rhs[i] || !x[i]) return IGAMG_ERR_ARG;
  if (b->lock) return igamg::lockstep_solve(b->lock, b->user, rhs, x, tol, res, status);
  // the solves start after the work already queued on the caller's stream
  if (cudaEventRecord(b->start, b->user) != cudaSuccess) return IGAMG_ERR_CUDA;
  for (cudaStream_t s : b->streams)
    if (cudaStreamWaitEvent(s, b->start, 0) != cudaSuccess) return IGAMG_ERR_CUDA;
  std::vector<igamg_status> st(n, IGAMG_OK);
  int dev = 0;
  cudaGetDevice(&dev);
  run_pool(W, n, [&](int w, int k) {
    cudaSetDevice(dev);
    const int i = b->order[k];
    igamg_ctx* c = b->ctx[i];
    igamg::ctx_set_stream(c, b->streams[w]);
    st[i] = igamg_solve(c, rhs[i], x[i], tol, res ? &res[i] : nullptr);
    igamg::ctx_set_stream(c, b->user);
  });
  // and the caller's stream continues after every solve
  for (int w = 0; w < W; ++w) {
    if (cudaEventRecord(b->done[w], b->streams[w]) != cudaSuccess) return IGAMG_ERR_CUDA;
    if (cudaStreamWaitEvent(b->user, b->done[w], 0) != cudaSuccess) return IGAMG_ERR_CUDA;
  }
  igamg_status worst = IGAMG_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = st[i];
    if (st[i] != IGAMG_OK && (worst == IGAMG_OK || worst == IGAMG_ERR_NOT_CONVERGED)) worst = st[i];
  }
  return worst;
}

igamg_status igamg_free_batch(igamg_batch* b) {
  destroy(b);
  return IGAMG_OK;
}

}  // extern "C"
