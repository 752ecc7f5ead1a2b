// Continuous-batching solver server.
//
// Grids are registered once and stay resident (A, Z, D^-1 and the work planes,
// including the last solution used for warm starts). A scheduler thread keeps
// up to max_slots requests on the device. Every round it
//   1. admits queued requests, in arrival order, whose grid has no request in
//      flight (per-grid FIFO: a timestep depends on the previous solution),
//      and runs their init kernels (r0 = b - A x0, s0, rho0);
//   2. advances every admitted request together by at most chunk_iters PCG
//      iterations: one launch of each kernel covers the work units of all of
//      them, through a conditional CUDA graph that stops early once all are
//      done;
//   3. reads the per-grid states back; each finished request gets its final
//      x update and true-residual check, is restarted from the true residual
//      if that fails, or retires (solution copied out, latency recorded,
//      callback fired).
// Requests that arrive while others iterate join at the next round, so their
// work overlaps on the device with the requests already in flight. Every
// kernel computes each grid's reductions from that grid's own partial sums in
// a fixed order, so a request's result does not depend on what else is in the
// batch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "handle.cuh"

using namespace pcg;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t id = 0;
  int grid = 0;
  std::vector<double> b;           // copy of the right-hand side (host)
  double *x_out = nullptr;
  bool warm = false;
  void (*done)(void *, const pcg_stats *) = nullptr;
  void *user = nullptr;
  Clock::time_point t_submit, t_done;
  pcg_stats stats{};
  int status = -1;
  bool finished = false;
};

struct GridEntry {
  pcg_handle *h = nullptr;
  bool busy = false;
  bool has_solution = false;
};

}  // namespace

struct pcg_server {
  pcg_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread th;
  bool stop = false;
  std::vector<GridEntry> grids;
  size_t hbm_used = 0;
  std::map<uint64_t, std::shared_ptr<Request>> reqs;
  std::deque<uint64_t> queue;
  uint64_t next_id = 1;
  uint64_t submitted = 0, completed = 0, failed = 0, rejected = 0;
  std::vector<double> lat_ms;
  Clock::time_point t_first, t_last;
  bool any_submit = false;
  int in_flight = 0;
  cudaStream_t stream = nullptr;
  LaunchState *ls_dev = nullptr, *ls_host = nullptr;

  void run();
};

void pcg_server::run() {
  struct Active {
    std::shared_ptr<Request> r;
    Member m;
    SolveState *st_host = nullptr;
  };
  std::vector<Active> active;
  std::unique_ptr<LoopPlan> plan;
  bool plan_dirty = true;
  pcg_opts o;
  fill_opts(&opts.solve, o);
  const int chunk = std::max(1, opts.chunk_iters);
  auto finish = [&](Active &a, int status) {
    a.m.final_status = status;
    member_stats(a.m);
    a.r->stats = a.m.stats ? *a.m.stats : pcg_stats{};
    a.r->stats.status = status;
    a.r->t_done = Clock::now();
    a.r->stats.seconds = std::chrono::duration<double>(a.r->t_done - a.r->t_submit).count();
    if (a.r->done) a.r->done(a.r->user, &a.r->stats);
    std::lock_guard<std::mutex> lk(mu);
    a.r->status = status;
    a.r->finished = true;
    grids[a.r->grid].busy = false;
    if (status == PCG_OK) grids[a.r->grid].has_solution = true;
    if (status == PCG_OK) ++completed; else ++failed;
    lat_ms.push_back(a.r->stats.seconds * 1e3);
    t_last = a.r->t_done;
    --in_flight;
    cv_done.notify_all();
  };

  for (;;) {
    std::vector<std::shared_ptr<Request>> admitted;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !active.empty() || !queue.empty(); });
      if (stop) break;
      for (auto it = queue.begin(); it != queue.end() && (int)(active.size() + admitted.size()) < opts.max_slots;) {
        auto r = reqs[*it];
        if (grids[r->grid].busy) { ++it; continue; }
        grids[r->grid].busy = true;
        admitted.push_back(r);
        ++in_flight;
        it = queue.erase(it);
      }
    }
    // 1. admission: load inputs and run the init kernels of each new request
    for (auto &r : admitted) {
      Active a;
      a.r = r;
      a.m.h = grids[r->grid].h;
      a.m.b = r->b.data();
      a.m.x = r->x_out;
      a.m.stats = &r->stats;
      a.m.st_host = a.m.h->st_host;
      pcg_opts ro = o;
      ro.use_x0 = (r->warm && grids[r->grid].has_solution) ? 1 : 0;
      int rc = member_load(a.m, ro, false, stream);
      LoopPlan *single = nullptr;
      if (!rc) rc = plan_single(a.m.h);
      if (!rc) {
        single = a.m.h->plan64.get();
        rc = members_arm(*single, a.m.h->ls_host, 1, 1, stream);
      }
      if (!rc) rc = members_init(*single, stream);
      if (rc) { finish(a, rc); continue; }
      active.push_back(std::move(a));
      plan_dirty = true;
    }
    if (active.empty()) continue;
    // states after init (some may already be done)
    for (auto &a : active) cudaMemcpyAsync(a.m.st_host, a.m.h->p64.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess) {
      for (auto &a : active) finish(a, PCG_ECUDA);
      active.clear();
      continue;
    }
    int n_iter = 0;
    for (auto &a : active) n_iter += (!a.m.st_host->done && a.m.st_host->status == PCG_OK) ? 1 : 0;
    // 2. advance all together by up to `chunk` iterations
    if (n_iter > 0) {
      if (plan_dirty) {
        plan = std::make_unique<LoopPlan>();
        std::vector<pcg_handle *> hs;
        for (auto &a : active) hs.push_back(a.m.h);
        int rc = plan_build(*plan, hs.data(), (int)hs.size(), true, ls_dev, stream);
        if (rc) { for (auto &a : active) finish(a, rc); active.clear(); continue; }
        plan_dirty = false;
      }
      int rc = members_arm(*plan, ls_host, n_iter, chunk, stream);
      if (!rc) rc = members_loop(*plan, ls_host, chunk, stream);
      for (auto &a : active) cudaMemcpyAsync(a.m.st_host, a.m.h->p64.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream);
      if (rc || cudaStreamSynchronize(stream) != cudaSuccess) {
        for (auto &a : active) finish(a, PCG_ECUDA);
        active.clear();
        continue;
      }
    }
    // 3. close finished requests: x update, true residual, restart or retire
    std::vector<Active> still;
    for (auto &a : active) {
      const SolveState &st = *a.m.st_host;
      if (!st.done && st.status == PCG_OK) { still.push_back(std::move(a)); continue; }
      LoopPlan *single = a.m.h->plan64.get();
      int rc = members_close(*single, stream);
      if (!rc && cudaMemcpyAsync(a.m.st_host, a.m.h->p64.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream) != cudaSuccess) rc = PCG_ECUDA;
      if (!rc && cudaStreamSynchronize(stream) != cudaSuccess) rc = PCG_ECUDA;
      if (rc) { finish(a, rc); plan_dirty = true; continue; }
      int err = PCG_OK;
      const bool again = member_decide(a.m, o, false, stream, &err);
      if (err) { finish(a, err); plan_dirty = true; continue; }
      if (again) {
        rc = members_arm(*single, a.m.h->ls_host, 1, 1, stream);
        if (!rc) rc = members_init(*single, stream);
        if (rc) { finish(a, rc); plan_dirty = true; continue; }
        still.push_back(std::move(a));
        continue;
      }
      rc = member_store(a.m, stream);
      if (!rc && cudaStreamSynchronize(stream) != cudaSuccess) rc = PCG_ECUDA;
      finish(a, rc ? rc : a.m.final_status);
      plan_dirty = true;
    }
    active.swap(still);
  }
  // shutting down: whatever is still active is abandoned
  for (auto &a : active) finish(a, PCG_ECANCELLED);
}

extern "C" {

int solver_server_create(const pcg_server_opts *opts, pcg_server **out) {
  if (!opts || !out) { set_error("NULL argument"); return PCG_EINVAL; }
  if (opts->max_slots < 1 || opts->max_slots > 256) { set_error("max_slots must be 1..256"); return PCG_EINVAL; }
  *out = nullptr;
  auto s = std::make_unique<pcg_server>();
  s->opts = *opts;
  if (s->opts.chunk_iters <= 0) s->opts.chunk_iters = 16;
  CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  CK(cudaMalloc(&s->ls_dev, sizeof(LaunchState)));
  CK(cudaMallocHost(&s->ls_host, sizeof(LaunchState)));
  pcg_server *raw = s.release();
  raw->th = std::thread([raw] { raw->run(); });
  *out = raw;
  return PCG_OK;
}

int solver_server_register(pcg_server *s, pcg_handle *h, int32_t *grid_id) {
  if (!s || !h || !grid_id) { set_error("NULL argument"); return PCG_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto &g : s->grids)
    if (g.h == h) { set_error("grid already registered"); return PCG_EINVAL; }
  const size_t need = pcg_resident_bytes(h);
  if (s->hbm_used + need > s->opts.hbm_budget_bytes) {
    set_error("registering this grid would exceed the HBM budget");
    return PCG_EBUDGET;
  }
  s->hbm_used += need;
  GridEntry e;
  e.h = h;
  s->grids.push_back(e);
  *grid_id = (int32_t)s->grids.size() - 1;
  return PCG_OK;
}

int solver_server_submit(pcg_server *s, int32_t grid_id, const double *b, double *x_out, int32_t warm_start,
                         void (*done)(void *, const pcg_stats *), void *user, uint64_t *req_id) {
  if (!s || !b || !x_out) { set_error("NULL argument"); return PCG_EINVAL; }
  pcg_handle *h;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (grid_id < 0 || grid_id >= (int)s->grids.size()) { set_error("unknown grid id"); ++s->rejected; return PCG_EINVAL; }
    h = s->grids[grid_id].h;
  }
  auto r = std::make_shared<Request>();
  r->grid = grid_id;
  r->x_out = x_out;
  r->warm = warm_start != 0;
  r->done = done;
  r->user = user;
  const size_t n = (size_t)h->G.nx * h->G.ny;
  r->b.resize(n);
  if (is_device_ptr(b)) {
    CK(cudaMemcpy(r->b.data(), b, n * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(r->b.data(), b, n * sizeof(double));
  }
  std::lock_guard<std::mutex> lk(s->mu);
  r->t_submit = Clock::now();
  r->id = s->next_id++;
  if (!s->any_submit) { s->t_first = r->t_submit; s->any_submit = true; }
  s->reqs[r->id] = r;
  s->queue.push_back(r->id);
  ++s->submitted;
  if (req_id) *req_id = r->id;
  s->cv_work.notify_all();
  return PCG_OK;
}

int solver_server_wait(pcg_server *s, uint64_t req_id, int32_t timeout_ms, pcg_stats *stats) {
  if (!s) { set_error("NULL server"); return PCG_EINVAL; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) { set_error("unknown request id"); return PCG_EINVAL; }
  auto r = it->second;
  auto ready = [&] { return r->finished; };
  if (timeout_ms < 0) s->cv_done.wait(lk, ready);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    set_error("request not finished before the timeout");
    return PCG_ETIMEOUT;
  }
  if (stats) *stats = r->stats;
  const int st = r->status;
  s->reqs.erase(req_id);
  return st;
}

int solver_server_cancel(pcg_server *s, uint64_t req_id) {
  if (!s) { set_error("NULL server"); return PCG_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = std::find(s->queue.begin(), s->queue.end(), req_id);
  if (it == s->queue.end()) { set_error("request is not queued (running, finished or unknown)"); return PCG_EINVAL; }
  s->queue.erase(it);
  auto r = s->reqs[req_id];
  r->status = PCG_ECANCELLED;
  r->stats.status = PCG_ECANCELLED;
  r->finished = true;
  ++s->failed;
  s->cv_done.notify_all();
  return PCG_OK;
}

int solver_server_stats(pcg_server *s, pcg_server_stats *out) {
  if (!s || !out) { set_error("NULL argument"); return PCG_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->rejected = s->rejected;
  out->in_flight = s->in_flight;
  out->queued = (int32_t)s->queue.size();
  out->hbm_used_bytes = s->hbm_used;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto rank = [&](double p) {   // nearest rank
      size_t k = (size_t)std::ceil(p * v.size());
      return v[std::min(v.size() - 1, k == 0 ? 0 : k - 1)];
    };
    out->p50_latency_ms = rank(0.50);
    out->p99_latency_ms = rank(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_latency_ms = sum / v.size();
    const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
    out->solves_per_s = span > 0 ? (double)s->completed / span : 0.0;
  }
  return PCG_OK;
}

void solver_server_destroy(pcg_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (uint64_t id : s->queue) {
      auto r = s->reqs[id];
      r->status = PCG_ECANCELLED;
      r->finished = true;
    }
    s->queue.clear();
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  cudaStreamSynchronize(s->stream);
  cudaStreamDestroy(s->stream);
  cudaFree(s->ls_dev);
  cudaFreeHost(s->ls_host);
  delete s;
}

}  // extern "C"
