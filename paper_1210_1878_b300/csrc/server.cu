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
  double *b = nullptr;             // device copy of the right-hand side (from the grid's buffer pool)
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
  std::vector<double *> pool;      // free right-hand-side buffers of this grid's size
  size_t buffers = 0;              // buffers allocated for this grid
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
  // A request moves through phases. binary64: START (init kernels) -> ITER
  // (advanced with the others, chunk by chunk) -> its x update and true
  // residual, then a restart from the true residual or the end. Mixed: START
  // (binary64 residual; the end, or a binary32 inner solve set up) -> ITER
  // (the inner solve, advanced with the others) -> its last x32 update and the
  // binary64 correction -> START again.
  //
  // The chunks run through one batched plan over every registered grid,
  // built again only when a grid is registered: a grid with no request
  // iterating has its device state marked done, and the persistent kernels
  // skip a done grid's units in one step.
  enum { START = 0, ITER = 1 };
  struct Active {
    std::shared_ptr<Request> r;
    Member m;
    int phase = START;
    int outer = 0;
  };
  std::vector<Active> active;
  std::unique_ptr<LoopPlan> plan;
  size_t plan_grids = 0;
  pcg_opts o;
  fill_opts(&opts.solve, o);
  const bool mixed = o.prec == PCG_MIXED;
  const int chunk = std::max(1, opts.chunk_iters);
  static const int32_t kOne = 1;
  auto finish = [&](Active &a, int status) {
    a.m.final_status = status;
    if (mixed) mixed_stats(a.m); else member_stats(a.m);
    a.r->stats.status = status;
    a.r->t_done = Clock::now();
    a.r->stats.seconds = std::chrono::duration<double>(a.r->t_done - a.r->t_submit).count();
    if (a.r->done) a.r->done(a.r->user, &a.r->stats);
    std::lock_guard<std::mutex> lk(mu);
    a.r->status = status;
    a.r->finished = true;
    grids[a.r->grid].busy = false;
    if (a.r->b) { grids[a.r->grid].pool.push_back(a.r->b); a.r->b = nullptr; }
    if (status == PCG_OK) grids[a.r->grid].has_solution = true;
    if (status == PCG_OK) ++completed; else ++failed;
    lat_ms.push_back(a.r->stats.seconds * 1e3);
    t_last = a.r->t_done;
    --in_flight;
    cv_done.notify_all();
  };
  // the final x of each finished request goes to its output buffer, one sync for all
  auto retire_all = [&](std::vector<Active> &done_list) {
    if (done_list.empty()) return;
    std::vector<int> rcs(done_list.size(), PCG_OK);
    for (size_t i = 0; i < done_list.size(); ++i) rcs[i] = member_store(done_list[i].m, stream);
    const bool ok = cudaStreamSynchronize(stream) == cudaSuccess;
    for (size_t i = 0; i < done_list.size(); ++i)
      finish(done_list[i], rcs[i] ? rcs[i] : (ok ? done_list[i].m.final_status : PCG_ECUDA));
    done_list.clear();
  };
  auto state_of = [&](Active &a) -> SolveState & { return mixed ? *a.m.h->st32_host : *a.m.st_host; };
  auto dev_state = [&](Active &a) { return mixed ? a.m.h->p32.st : a.m.h->p64.st; };

  for (;;) {
    std::vector<std::shared_ptr<Request>> admitted;
    std::vector<pcg_handle *> all;
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
      if (grids.size() != plan_grids)
        for (auto &g : grids) all.push_back(g.h);
    }
    // the batched plan over every registered grid (new registrations only);
    // grids without an iterating request are marked done on the device
    if (!all.empty()) {
      int rc = PCG_OK;
      for (pcg_handle *h : all) {
        if (!rc) rc = plan_single(h);
        if (!rc && mixed) rc = ensure_f32(h, stream);
      }
      for (pcg_handle *h : all) {
        bool busy = false;
        for (auto &a : active) busy = busy || a.m.h == h;
        if (busy || rc) continue;
        if (cudaMemcpyAsync(&h->p64.st->done, &kOne, sizeof(int32_t), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            (mixed && cudaMemcpyAsync(&h->p32.st->done, &kOne, sizeof(int32_t), cudaMemcpyHostToDevice, stream) !=
                          cudaSuccess))
          rc = PCG_ECUDA;
      }
      if (!rc) {
        auto np = std::make_unique<LoopPlan>();
        rc = mixed ? plan_build32(*np, all.data(), (int)all.size(), true, ls_dev, stream)
                   : plan_build(*np, all.data(), (int)all.size(), true, ls_dev, stream);
        if (!rc && cudaStreamSynchronize(stream) != cudaSuccess) rc = PCG_ECUDA;
        if (!rc) { plan = std::move(np); plan_grids = all.size(); }
      }
      if (rc) {
        for (auto &a : active) finish(a, rc);
        active.clear();
        for (auto &r : admitted) {
          Active a;
          a.r = r;
          a.m.h = grids[r->grid].h;
          a.m.stats = &r->stats;
          a.m.st_host = a.m.h->st_host;
          finish(a, rc);
        }
        continue;
      }
    }
    // admission: inputs on the device (the warm start keeps the grid's last x)
    for (auto &r : admitted) {
      Active a;
      a.r = r;
      a.m.h = grids[r->grid].h;
      a.m.b = r->b;
      a.m.x = r->x_out;
      a.m.stats = &r->stats;
      a.m.st_host = a.m.h->st_host;
      pcg_opts ro = o;
      ro.use_x0 = (r->warm && grids[r->grid].has_solution) ? 1 : 0;
      int rc = plan_single(a.m.h);
      if (!rc && mixed) rc = ensure_f32(a.m.h, stream);
      if (!rc) rc = member_load(a.m, ro, false, stream);
      if (rc) { finish(a, rc); continue; }
      a.m.inner_iters = 0; a.m.inner_solves = 0; a.m.relres64 = 0.0;
      active.push_back(std::move(a));
    }
    if (active.empty()) continue;
    // START phase. binary64: the init kernels. Mixed: the binary64 residual
    // of every starting request, one sync, then each one's decision and, if
    // it goes on, its binary32 inner solve set up.
    const int budget_cap = o.max_iter;
    std::vector<Active> next, retiring;
    std::vector<int> start_rc(active.size(), PCG_OK);
    bool any_start = false;
    for (size_t i = 0; i < active.size(); ++i) {
      Active &a = active[i];
      if (a.phase != START) continue;
      pcg_handle *h = a.m.h;
      int rc = members_arm(*h->plan64, h->ls_host, 1, 1, stream);
      if (!rc) rc = single_launch(h, false, 1, K1_RESID_INIT, stream);
      if (!mixed) {
        if (!rc) rc = single_launch(h, false, 2, K2_INIT, stream);
      } else if (!rc &&
                 cudaMemcpyAsync(a.m.st_host, h->p64.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream) !=
                     cudaSuccess) {
        rc = PCG_ECUDA;
      }
      start_rc[i] = rc;
      any_start = true;
    }
    if (mixed && any_start && cudaStreamSynchronize(stream) != cudaSuccess)
      for (size_t i = 0; i < active.size(); ++i)
        if (active[i].phase == START && !start_rc[i]) start_rc[i] = PCG_ECUDA;
    for (size_t i = 0; i < active.size(); ++i) {
      Active &a = active[i];
      if (a.phase != START) { next.push_back(std::move(a)); continue; }
      if (start_rc[i]) { finish(a, start_rc[i]); continue; }
      pcg_handle *h = a.m.h;
      if (mixed) {
        const int budget = budget_cap > 0 ? budget_cap : std::max(h->G.n, 1);
        int err = PCG_OK;
        const bool over = mixed_prepare_inner(a.m, o, budget, a.outer, stream, &err);
        if (err) { finish(a, err); continue; }
        if (over) { retiring.push_back(std::move(a)); continue; }
        int rc = members_arm(*h->plan32, h->ls_host, 1, 1, stream);
        if (!rc) rc = single_launch(h, true, 1, K1_RESID_INIT, stream);
        if (!rc) rc = single_launch(h, true, 2, K2_INIT, stream);
        if (rc) { finish(a, rc); continue; }
        a.outer += 1;
      }
      a.phase = ITER;
      next.push_back(std::move(a));
    }
    active.swap(next);
    retire_all(retiring);
    if (active.empty()) continue;
    // states of the iterating requests (some may be done already)
    for (auto &a : active) cudaMemcpyAsync(&state_of(a), dev_state(a), sizeof(SolveState), cudaMemcpyDeviceToHost, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess) {
      for (auto &a : active) finish(a, PCG_ECUDA);
      active.clear();
      continue;
    }
    int n_iter = 0;
    for (auto &a : active) n_iter += (a.phase == ITER && !state_of(a).done) ? 1 : 0;
    // advance every iterating request together by up to `chunk` iterations
    if (n_iter > 0) {
      int rc = members_arm(*plan, ls_host, n_iter, chunk, stream);
      if (!rc) rc = members_loop(*plan, ls_host, chunk, stream);
      for (auto &a : active) cudaMemcpyAsync(&state_of(a), dev_state(a), sizeof(SolveState), cudaMemcpyDeviceToHost, stream);
      if (rc || cudaStreamSynchronize(stream) != cudaSuccess) {
        for (auto &a : active) finish(a, PCG_ECUDA);
        active.clear();
        continue;
      }
    }
    // requests whose iteration ended. binary64: x update and true residual of
    // all of them, one sync, then each one's decision.
    std::vector<Active> still, ended;
    for (auto &a : active) {
      const SolveState &st = state_of(a);
      if (!st.done && st.status == PCG_OK) still.push_back(std::move(a));
      else ended.push_back(std::move(a));
    }
    if (!ended.empty()) {
      std::vector<int> rcs(ended.size(), PCG_OK);
      for (size_t i = 0; i < ended.size(); ++i) {
        Active &a = ended[i];
        pcg_handle *h = a.m.h;
        if (mixed) {
          // last x32 update, then the binary64 correction
          rcs[i] = single_launch(h, true, 0, 0, stream);
          if (!rcs[i]) rcs[i] = mixed_apply_correction(a.m, stream);
        } else {
          rcs[i] = members_close(*h->plan64, stream);
          if (!rcs[i] &&
              cudaMemcpyAsync(a.m.st_host, h->p64.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
            rcs[i] = PCG_ECUDA;
        }
      }
      if (!mixed && cudaStreamSynchronize(stream) != cudaSuccess)
        for (auto &rc : rcs) rc = rc ? rc : PCG_ECUDA;
      for (size_t i = 0; i < ended.size(); ++i) {
        Active &a = ended[i];
        if (rcs[i]) { finish(a, rcs[i]); continue; }
        if (mixed) {
          if (a.m.final_status >= 0) { retiring.push_back(std::move(a)); continue; }
          a.phase = START;
          still.push_back(std::move(a));
          continue;
        }
        int err = PCG_OK;
        const bool again = member_decide(a.m, o, false, stream, &err);
        if (err) { finish(a, err); continue; }
        if (again) { a.phase = START; still.push_back(std::move(a)); continue; }
        retiring.push_back(std::move(a));
      }
    }
    active.swap(still);
    retire_all(retiring);
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
  handle_finish_pending(h);   // a solve enqueued on the handle before it joins the server
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto &g : s->grids)
    if (g.h == h) { set_error("grid already registered"); return PCG_EINVAL; }
  if (s->opts.solve.prec == PCG_MIXED) {
    // the binary32 planes are resident too (and counted)
    int rc = ensure_f32(h, s->stream);
    if (!rc && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = PCG_ECUDA;
    if (rc) return rc;
  }
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
  auto r = std::make_shared<Request>();
  size_t n = 0;
  {
    // a right-hand-side buffer from the grid's pool; a new one only if the
    // HBM budget (registered grids + buffers) allows it
    std::lock_guard<std::mutex> lk(s->mu);
    if (grid_id < 0 || grid_id >= (int)s->grids.size()) { set_error("unknown grid id"); ++s->rejected; return PCG_EINVAL; }
    GridEntry &g = s->grids[grid_id];
    n = (size_t)g.h->G.nx * g.h->G.ny;
    if (!g.pool.empty()) {
      r->b = g.pool.back();
      g.pool.pop_back();
    } else {
      if (s->hbm_used + n * sizeof(double) > s->opts.hbm_budget_bytes) {
        ++s->rejected;
        set_error("no right-hand-side buffer fits in the HBM budget");
        return PCG_EBUDGET;
      }
      if (cudaMalloc(&r->b, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        ++s->rejected;
        set_error("device allocation of a right-hand-side buffer failed");
        return PCG_ENOMEM;
      }
      s->hbm_used += n * sizeof(double);
      g.buffers += 1;
    }
  }
  r->grid = grid_id;
  r->x_out = x_out;
  r->warm = warm_start != 0;
  r->done = done;
  r->user = user;
  // the caller may reuse b as soon as this returns
  if (cudaMemcpy(r->b, b, n * sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(s->mu);
    s->grids[grid_id].pool.push_back(r->b);
    set_error("copy of the right-hand side failed");
    return PCG_ECUDA;
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
  if (r->b) { s->grids[r->grid].pool.push_back(r->b); r->b = nullptr; }
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
  for (auto &g : s->grids)
    for (double *p : g.pool) cudaFree(p);
  for (auto &kv : s->reqs)
    if (kv.second->b) cudaFree(kv.second->b);
  cudaStreamDestroy(s->stream);
  cudaFree(s->ls_dev);
  cudaFreeHost(s->ls_host);
  delete s;
}

}  // extern "C"
