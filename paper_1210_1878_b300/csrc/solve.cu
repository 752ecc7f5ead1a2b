// Whole solves enqueued on a stream (pcg_solve, pcg_solve_batched, pcg_sync).
//
// A solve is Algorithm 1 plus its stopping rule, run entirely on the device:
// one CUDA graph per plan whose outer conditional WHILE loop repeats a "pass"
// and whose inner WHILE loop is the PCG iteration itself.
//
//   binary64 pass:  arm -> r0 = b - A x, s0 = M^-1 r0 (init kernels)
//                   -> WHILE { stencil kernel, preconditioner kernel }
//                   -> final x update, true residual b - A x
//                   -> decide: per grid, stop (result final) or restart from
//                      the true residual; no restart left ends the outer loop
//   mixed pass:     r = b - A x in binary64 -> decide: per grid, stop or set
//                   up a binary32 inner solve (power-of-two scale, inner
//                   tolerance) -> r scaled into binary32, x32 = d32 = 0 ->
//                   arm -> binary32 init kernels -> WHILE { binary32 stencil,
//                   preconditioner } -> last x32 update -> accounting ->
//                   x += x32 / scale in binary64
//
// The decisions that the host made between passes (restart or stop, the
// refinement step's scale and tolerance) are small single-block kernels that
// read and write the grids' device states, so a solve needs no host round
// trip: the call enqueues the packing of b (and x0), the state set-up, one
// graph launch, the unpacking of x and a copy of the final states into pinned
// host memory, and returns. pcg_sync waits for the stream and fills the
// statistics. The graphs are built once per plan (a handle alone, or a batch
// of handles) and kept.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "solve_graph.cuh"

namespace pcg {


static __device__ __forceinline__ int block_or(int v) { return __syncthreads_or(v); }

// Solve set-up, replacing the host-written state: every member starts from
// iteration 0 with the call's options (kernel arguments, so the host keeps no
// buffer the device reads later).
__global__ void __launch_bounds__(CTL_THREADS) k_ctl_begin(SolveState *const *st, const int32_t *n_wet, int n,
                                                           double rtol, int max_iter_opt, int max_replace,
                                                           double inner_rtol, int max_outer, int budget,
                                                           LaunchState *ls) {
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    SolveState *S = st[m];
    const int nw = n_wet[m];
    SolveState z{};
    z.rtol = rtol;
    z.max_iter = max_iter_opt > 0 ? max_iter_opt : max(nw, 1);
    z.status = PCG_OK;
    z.done = nw == 0 ? 1 : 0;
    z.retired = z.done;
    z.final_status = z.done ? PCG_OK : -1;
    z.max_replace = max_replace;
    z.scale = 1.0;
    z.inner_rtol = inner_rtol;
    z.budget = budget;
    z.max_outer = max_outer;
    *S = z;
  }
  if (threadIdx.x == 0) {
    ls->bodies_total = 0;
    ls->passes = 0;
  }
}

// Arm the inner loop of a pass: the members still iterating (done == 0), a cap
// of their largest max_iter + 64 loop bodies, the wall-clock guard, and the
// inner loop's condition set so that its body runs.
__global__ void __launch_bounds__(CTL_THREADS) k_ctl_arm(SolveState *const *st, int n, LaunchState *ls,
                                                         cudaGraphConditionalHandle cond_in, uint64_t budget_ns) {
  __shared__ int s_act, s_mi;
  if (threadIdx.x == 0) { s_act = 0; s_mi = 0; }
  __syncthreads();
  int act = 0, mi = 0;
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    const SolveState *S = st[m];
    if (!S->done) { ++act; mi = max(mi, S->max_iter); }
  }
  if (act) atomicAdd(&s_act, act);
  if (mi) atomicMax(&s_mi, mi);
  __syncthreads();
  if (threadIdx.x == 0) {
    ls->active = s_act;
    ls->launches = 0;
    ls->max_launches = s_mi + 64;
    ls->stop = 0;
    ls->cond = cond_in;
    ls->t0_ns = 0;
    ls->budget_ns = budget_ns;
    ls->timed_out = 0;
    ls->cond_cleared = 0;
    cudaGraphSetConditional(cond_in, 1);
  }
}

// End of a binary64 pass (the stopping rule of Algorithm 1 with the
// true-residual check): per member, the result is final -- the status a
// kernel recorded, the true residual meeting rtol, the iteration cap or the
// restart cap reached, or the loop ended without it -- or it restarts from the
// true residual, which is in its current r plane. No restart ends the outer
// loop.
__global__ void __launch_bounds__(CTL_THREADS) k_ctl_decide64(SolveState *const *st, int n, LaunchState *ls,
                                                              cudaGraphConditionalHandle cond_out) {
  const int pass = ls->passes + 1;
  int again = 0;
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    SolveState *S = st[m];
    if (S->final_status >= 0) continue;
    int fs = -1;
    if (S->status != PCG_OK) fs = S->status;
    else if (!S->done) fs = PCG_ETIMEOUT;           // the loop ended (a runaway guard) without this grid
    else if (S->bzero) fs = PCG_OK;
    else {
      const double tr = sqrt(S->rr_true) / sqrt(S->bb);
      if (tr <= S->rtol) fs = PCG_OK;
      else if (S->iter >= S->max_iter || S->replacements >= S->max_replace) fs = PCG_ENOTCONV;
      else if (pass >= MAX_PASSES) fs = PCG_ETIMEOUT;
    }
    if (fs >= 0) {
      S->final_status = fs;
      S->retired = 1;
    } else {
      S->replacements += 1;
      S->done = 0;
      again = 1;
    }
  }
  again = block_or(again);
  if (threadIdx.x == 0) {
    ls->passes = pass;
    if (!again) cudaGraphSetConditional(cond_out, 0);
  }
}

// Mixed precision, start of a refinement step, after r = b - A x in binary64:
// per member, the result is final (binary64 relative residual at most rtol,
// b = 0, a recorded failure, or a cap reached) or a binary32 inner solve is set
// up: the scale 2^k nearest 1 / RMS(r) (exact), the inner tolerance (inner_rtol
// far from the finish; within a decade of it, half the reduction still needed,
// floor inner_rtol / 10), and the remaining iteration budget. No inner solve
// left ends the outer loop.
__global__ void __launch_bounds__(CTL_THREADS) k_ctl_mixed_prepare(SolveState *const *st64, SolveState *const *st32,
                                                                   const int32_t *n_wet, int n, LaunchState *ls,
                                                                   cudaGraphConditionalHandle cond_out) {
  const int pass = ls->passes + 1;
  int more = 0;
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    SolveState *A = st64[m], *F = st32[m];
    SolveState z{};
    z.status = PCG_OK;
    z.final_status = -1;
    if (A->final_status >= 0) {
      z.done = 1; z.retired = 1;
      *F = z;
      continue;
    }
    int fs = -1;
    if (A->status != PCG_OK) fs = A->status;
    else if (A->bzero) { A->relres64 = 0.0; fs = PCG_OK; }
    else {
      A->relres64 = sqrt(A->rr) / sqrt(A->bb);
      if (!(A->relres64 > A->rtol)) fs = PCG_OK;
      else if (!isfinite(A->relres64)) fs = PCG_EBREAKDOWN;
      else if (A->inner_solves >= A->max_outer || A->inner_iters >= A->budget || pass >= MAX_PASSES) fs = PCG_ENOTCONV;
    }
    if (fs >= 0) {
      A->final_status = fs;
      A->retired = 1;
      A->done = 1;
      z.done = 1; z.retired = 1;
    } else {
      const double rms = sqrt(A->rr / (double)max(n_wet[m], 1));
      A->scale = ldexp(1.0, -ilogb(rms > 0.0 ? rms : 1.0));
      const double need = A->rtol / A->relres64;
      z.rtol = need >= 0.1 * A->inner_rtol ? fmax(0.5 * need, 0.1 * A->inner_rtol) : A->inner_rtol;
      z.max_iter = max(1, A->budget - A->inner_iters);
      more = 1;
    }
    *F = z;
  }
  more = block_or(more);
  if (threadIdx.x == 0) {
    ls->passes = pass;
    if (!more) cudaGraphSetConditional(cond_out, 0);
  }
}

// Mixed precision, end of an inner solve: count its iterations; an inner solve
// that broke down before its first iteration ends the member with that status
// (its correction is then skipped).
__global__ void __launch_bounds__(CTL_THREADS) k_ctl_mixed_after(SolveState *const *st64, SolveState *const *st32,
                                                                 int n) {
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    SolveState *A = st64[m];
    const SolveState *F = st32[m];
    if (A->final_status >= 0 || F->retired) continue;
    A->inner_iters += F->iter;
    A->inner_solves += 1;
    if (F->status == PCG_EBREAKDOWN && F->iter == 0) {
      A->final_status = PCG_EBREAKDOWN;
      A->retired = 1;
      A->done = 1;
    }
  }
}



namespace {

template <typename V>
int upload_array(V **dev, const std::vector<V> &v) {
  CK(cudaMalloc(dev, sizeof(V) * std::max<size_t>(v.size(), 1)));
  CK(cudaMemcpy(*dev, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice));
  return PCG_OK;
}

// Device arrays of the members' states and wet counts, in plan order.
int upload_members(SolveGraph &S, const std::vector<pcg_handle *> &hs, bool mixed) {
  std::vector<SolveState *> s64, s32;
  std::vector<int32_t> nw;
  for (pcg_handle *h : hs) {
    s64.push_back(h->p64.st);
    if (mixed) s32.push_back(h->p32.st);
    nw.push_back(h->G.n);
  }
  S.n = (int)hs.size();
  int rc = upload_array(&S.st64, s64);
  if (!rc && mixed) rc = upload_array(&S.st32, s32);
  if (!rc) rc = upload_array(&S.n_wet, nw);
  return rc;
}

int finish_graph(SolveGraph &S, cudaGraph_t g, Builder &outer, Builder &inner) {
  if (outer.err != cudaSuccess || inner.err != cudaSuccess) {
    const cudaError_t e = outer.err != cudaSuccess ? outer.err : inner.err;
    cudaGetLastError();
    cudaGraphDestroy(g);
    set_error(std::string("solve graph construction failed: ") + cudaGetErrorString(e));
    return PCG_ECUDA;
  }
  const cudaError_t e = cudaGraphInstantiate(&S.exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    S.exec = nullptr;
    set_error(std::string("solve graph instantiation failed: ") + cudaGetErrorString(e));
    return PCG_ECUDA;
  }
  S.outer_kernels = outer.kernels;
  S.inner_kernels = inner.kernels;
  return PCG_OK;
}

// binary64 solve graph over the members (in plan order) of L.
int build_graph64(SolveGraph &S, const LoopPlan &L, const std::vector<pcg_handle *> &hs) {
  int rc = upload_members(S, hs, false);
  if (rc) return rc;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle c_out = 0, c_in = 0;
  Builder top(g);
  top.err = cudaGraphConditionalHandleCreate(&c_out, g, 1, cudaGraphCondAssignDefault);
  cudaGraph_t body = top.while_node(c_out);
  Builder P(body ? body : g);
  P.err = top.err;
  if (P.err == cudaSuccess) P.err = cudaGraphConditionalHandleCreate(&c_in, body, 0, 0);
  SolveState **stp = S.st64;
  int n = S.n;
  LaunchState *ls = L.ls;
  uint64_t bns = loop_budget_ns();
  {
    void *args[] = {&stp, &n, &ls, &c_in, &bns};
    P.kernel((const void *)k_ctl_arm, dim3(1), dim3(CTL_THREADS), 0, args);
  }
  add_groups(P, L, 1, K1_RESID_INIT, 0, false);
  add_groups(P, L, 2, K2_INIT, 0, false);
  cudaGraph_t ib = P.while_node(c_in);
  Builder I(ib ? ib : g);
  I.err = P.err;
  add_groups(I, L, 1, K1_ITER, 1, false);
  add_groups(I, L, 2, K2_ITER, 1, true);
  P.err = I.err;
  add_finalize(P, L);
  add_groups(P, L, 1, K1_RESID_CHECK, 0, false);
  {
    void *args[] = {&stp, &n, &ls, &c_out};
    P.kernel((const void *)k_ctl_decide64, dim3(1), dim3(CTL_THREADS), 0, args);
  }
  return finish_graph(S, g, P, I);
}

// Mixed-precision solve graph: binary64 plan L64 and binary32 plan L32 over the
// same members, in plan order.
int build_graph_mixed(SolveGraph &S, const LoopPlan &L64, const LoopPlan &L32, const std::vector<pcg_handle *> &hs) {
  int rc = upload_members(S, hs, true);
  if (rc) return rc;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle c_out = 0, c_in = 0;
  Builder top(g);
  top.err = cudaGraphConditionalHandleCreate(&c_out, g, 1, cudaGraphCondAssignDefault);
  cudaGraph_t body = top.while_node(c_out);
  Builder P(body ? body : g);
  P.err = top.err;
  if (P.err == cudaSuccess) P.err = cudaGraphConditionalHandleCreate(&c_in, body, 0, 0);
  SolveState **a64 = S.st64, **a32 = S.st32;
  int32_t *nwp = S.n_wet;
  int n = S.n;
  LaunchState *ls = L32.ls;
  uint64_t bns = loop_budget_ns();
  // binary64 residual r = b - A x and ||b|| of every member not finished
  add_groups(P, L64, 1, K1_RESID_INIT, 0, false);
  {
    void *args[] = {&a64, &a32, &nwp, &n, &ls, &c_out};
    P.kernel((const void *)k_ctl_mixed_prepare, dim3(1), dim3(CTL_THREADS), 0, args);
  }
  // r scaled into the binary32 right-hand side, x32 = d32 = 0 (per member: the
  // binary64 and binary32 planes of a member may belong to different groups)
  for (pcg_handle *h : hs) {
    const GridDev<double> *g64 = h->p64.gd_dev;
    const GridDev<float> *g32 = h->p32.gd_dev;
    const Unit *un = h->p64.units_dev;
    double sc = 0.0;
    void *args[] = {(void *)&g64, (void *)&g32, (void *)&un, &sc};
    P.kernel((const void *)k_residual_to_f32, dim3(h->p64.n_units), dim3(h->tx), 0, args);
  }
  {
    void *args[] = {&a32, &n, &ls, &c_in, &bns};
    P.kernel((const void *)k_ctl_arm, dim3(1), dim3(CTL_THREADS), 0, args);
  }
  add_groups(P, L32, 1, K1_RESID_INIT, 0, false);
  add_groups(P, L32, 2, K2_INIT, 0, false);
  cudaGraph_t ib = P.while_node(c_in);
  Builder I(ib ? ib : g);
  I.err = P.err;
  add_groups(I, L32, 1, K1_ITER, 1, false);
  add_groups(I, L32, 2, K2_ITER, 1, true);
  P.err = I.err;
  add_finalize(P, L32);
  {
    void *args[] = {&a64, &a32, &n};
    P.kernel((const void *)k_ctl_mixed_after, dim3(1), dim3(CTL_THREADS), 0, args);
  }
  for (pcg_handle *h : hs) {
    const GridDev<double> *g64 = h->p64.gd_dev;
    const GridDev<float> *g32 = h->p32.gd_dev;
    const Unit *un = h->p64.units_dev;
    double inv = 0.0;
    void *args[] = {(void *)&g64, (void *)&g32, (void *)&un, &inv};
    P.kernel((const void *)k_correct_f64, dim3(h->p64.n_units), dim3(h->tx), 0, args);
  }
  return finish_graph(S, g, P, I);
}

}  // namespace

// ------------------------------------------------------------ batch plans
// A batch's plans and graph, kept for later calls on the same handles (keyed
// by the handles' serial numbers and plane versions, so a freed or rebuilt
// handle never matches).
struct BatchPlan {
  std::vector<std::pair<uint64_t, uint32_t>> key;
  int prec = 0;
  LoopPlan L64, L32;
  std::unique_ptr<SolveGraph> graph;
};

namespace {

std::mutex g_batch_mu;
std::list<std::shared_ptr<BatchPlan>> g_batches;   // most recently used first
constexpr size_t kBatchCache = 4;

std::vector<std::pair<uint64_t, uint32_t>> batch_key(pcg_handle *const *hs, int n) {
  std::vector<std::pair<uint64_t, uint32_t>> k;
  for (int i = 0; i < n; ++i) k.emplace_back(hs[i]->serial, hs[i]->version);
  return k;
}

}  // namespace

// Statistics of member m of a finished whole-solve graph (states read back
// into the handle's pinned mirrors).
static void fill_stats(pcg_handle *h, bool mixed, pcg_stats *out, int *status) {
  const SolveState &st = *h->st_host;
  *status = st.final_status >= 0 ? st.final_status : PCG_ETIMEOUT;
  if (!out) return;
  if (mixed) {
    out->iters = st.inner_iters;
    out->outer_iters = st.inner_solves;
    out->replacements = 0;
    out->relres = st.relres64;
    out->true_relres = st.relres64;
  } else {
    out->iters = st.iter;
    out->outer_iters = 1 + st.replacements;
    out->replacements = st.replacements;
    out->relres = st.bb > 0 ? std::sqrt(st.rr) / std::sqrt(st.bb) : 0.0;
    out->true_relres = st.bb > 0 ? std::sqrt(st.rr_true) / std::sqrt(st.bb) : 0.0;
  }
  out->status = *status;
}

}  // namespace pcg

using namespace pcg;

namespace {

std::atomic<uint64_t> g_serial{1};

// Wait for h's enqueued solve (if any): the call's work on its stream (not
// what was queued there after it) and its members' copies back to host
// buffers. Fill the call's statistics and release what the call kept alive.
// Returns the call's status.
int finish_pending(pcg_handle *h) {
  std::shared_ptr<Pending> p = h->pending;
  if (!p) return h->last_status;
  int rc = PCG_OK;
  cudaError_t e = p->done ? cudaEventSynchronize(p->done) : cudaStreamSynchronize(p->s);
  for (pcg_handle *m : p->hs)
    if (e == cudaSuccess) e = cudaEventSynchronize(m->ev_stage);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("solve failed on the device: ") + cudaGetErrorString(e));
    rc = PCG_ECUDA;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - p->t0).count();
  int first_bad = PCG_OK;
  if (rc == PCG_OK && p->graph) {
    const LaunchState &ls = *p->ls_host;
    note_launches((uint64_t)std::max(ls.passes, 0) * p->outer_kernels +
                  (uint64_t)std::max(ls.bodies_total, 0) * p->inner_kernels);
    for (size_t i = 0; i < p->hs.size(); ++i) {
      int st = PCG_OK;
      fill_stats(p->hs[i], p->mixed, p->stats ? &p->stats[i] : nullptr, &st);
      if (st != PCG_OK && first_bad == PCG_OK) first_bad = st;
    }
  } else if (rc == PCG_OK) {
    first_bad = p->status;          // solved synchronously at the call
  }
  if (p->stats)
    for (size_t i = 0; i < p->hs.size(); ++i) p->stats[i].seconds = secs;
  const int status = rc != PCG_OK ? rc : first_bad;
  if (status != PCG_OK && rc == PCG_OK) set_error("solve finished with status: " + status_name(status));
  for (pcg_handle *m : p->hs) {
    m->pending.reset();
    m->last_status = status;
  }
  return status;
}

}  // namespace

void pcg::handle_init_serial(pcg_handle *h) { h->serial = g_serial.fetch_add(1); }
int pcg::handle_finish_pending(pcg_handle *h) { return finish_pending(h); }

extern "C" {

int pcg_sync(pcg_handle *h) {
  if (!h) { set_error("NULL handle"); return PCG_EINVAL; }
  return finish_pending(h);
}

int pcg_solve(pcg_handle *h, const double *b, double *x, const pcg_opts *opts, pcg_stats *stats, void *cuda_stream) {
  pcg_handle *hs[1] = {h};
  const double *bs[1] = {b};
  double *xs[1] = {x};
  return pcg_solve_batched(hs, 1, bs, xs, opts, stats, cuda_stream);
}

int pcg_solve_batched(pcg_handle *const *hs, int32_t nbatch, const double *const *b, double *const *x,
                      const pcg_opts *opts, pcg_stats *stats, void *cuda_stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!hs || nbatch <= 0 || !b || !x) { set_error("invalid batch arguments"); return PCG_EINVAL; }
  for (int i = 0; i < nbatch; ++i) {
    if (!hs[i] || !b[i] || !x[i]) { set_error("NULL handle or vector in batch"); return PCG_EINVAL; }
    for (int k = 0; k < i; ++k)
      if (hs[k] == hs[i]) { set_error("a handle may appear once per batch"); return PCG_EINVAL; }
  }
  pcg_opts o;
  fill_opts(opts, o);
  if (o.prec != PCG_FP64 && o.prec != PCG_MIXED) { set_error("unknown precision"); return PCG_EINVAL; }
  const bool mixed = o.prec == PCG_MIXED;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // one solve in flight per handle: finish an earlier one first
  for (int i = 0; i < nbatch; ++i) finish_pending(hs[i]);
  int rc;
  if (mixed)
    for (int i = 0; i < nbatch; ++i)
      if ((rc = ensure_f32(hs[i], s))) return rc;
  std::vector<pcg_handle *> members(hs, hs + nbatch);
  auto pend = std::make_shared<Pending>();
  pend->hs = members;
  pend->stats = stats;
  pend->s = s;
  pend->mixed = mixed;
  pend->t0 = t0;
  pend->ls_host = hs[0]->ls_host;

  // plans and the whole-solve graph: a handle alone keeps its own; a batch
  // uses (or builds) a cached batch plan
  SolveGraph *graph = nullptr;
  LoopPlan *L64 = nullptr, *L32 = nullptr;
  if (nbatch == 1) {
    pcg_handle *h = hs[0];
    if ((rc = plan_single(h))) return rc;
    L64 = h->plan64.get();
    L32 = mixed ? h->plan32.get() : nullptr;
    LoopPlan &owner = mixed ? *h->plan32 : *h->plan64;
    if (!owner.solve_tried && L64->graph_ok && (!mixed || L32->graph_ok)) {
      owner.solve_tried = true;
      auto G = std::make_unique<SolveGraph>();
      rc = mixed ? build_graph_mixed(*G, *L64, *L32, members) : build_graph64(*G, *L64, members);
      if (rc == PCG_OK) owner.solve = std::move(G);
    }
    graph = owner.solve.get();
  } else {
    auto key = batch_key(hs, nbatch);
    std::shared_ptr<BatchPlan> bp;
    {
      std::lock_guard<std::mutex> lk(g_batch_mu);
      for (auto it = g_batches.begin(); it != g_batches.end(); ++it)
        if ((*it)->key == key && (*it)->prec == o.prec) {
          bp = *it;
          g_batches.erase(it);
          g_batches.push_front(bp);
          break;
        }
    }
    if (!bp) {
      bp = std::make_shared<BatchPlan>();
      bp->key = key;
      bp->prec = o.prec;
      if ((rc = plan_build(bp->L64, hs, nbatch, !mixed, hs[0]->ls, s))) return rc;
      if (mixed && (rc = plan_build32(bp->L32, hs, nbatch, true, hs[0]->ls, s))) return rc;
      if (mixed ? bp->L32.graph_ok : bp->L64.graph_ok) {
        auto G = std::make_unique<SolveGraph>();
        rc = mixed ? build_graph_mixed(*G, bp->L64, bp->L32, members) : build_graph64(*G, bp->L64, members);
        if (rc == PCG_OK) bp->graph = std::move(G);
      }
      std::lock_guard<std::mutex> lk(g_batch_mu);
      g_batches.push_front(bp);
      while (g_batches.size() > kBatchCache) g_batches.pop_back();
    }
    L64 = &bp->L64;
    L32 = mixed ? &bp->L32 : nullptr;
    graph = bp->graph.get();
    pend->keep = bp;
  }

  std::vector<Member> M(nbatch);
  for (int i = 0; i < nbatch; ++i) {
    M[i].h = hs[i]; M[i].b = b[i]; M[i].x = x[i]; M[i].stats = stats ? &stats[i] : nullptr;
    M[i].st_host = hs[i]->st_host;
  }
  if (!graph) {
    // no conditional graphs (or the chunked loop was asked for): the
    // host-driven solve, synchronous
    rc = mixed ? solve_members_mixed(*L64, *L32, hs[0]->ls_host, M, o, s)
               : solve_members64(*L64, hs[0]->ls_host, M, o, s);
    if (rc) return rc;
    int first_bad = PCG_OK;
    for (auto &m : M)
      if (m.final_status != PCG_OK && first_bad == PCG_OK) first_bad = m.final_status;
    pend->status = first_bad;
    CK(cudaEventCreateWithFlags(&pend->done, cudaEventDisableTiming));
    CK(cudaEventRecord(pend->done, s));
    for (pcg_handle *h : members) h->pending = pend;
    return PCG_OK;
  }

  // inputs: b, x0 (or x = 0), zeroed directions, then the states
  int budget = 0;
  for (pcg_handle *h : members) budget = std::max(budget, std::max(h->G.n, 1));
  if (o.max_iter > 0) budget = o.max_iter;
  for (auto &m : M)
    if ((rc = member_pack(m, o, s))) return rc;
  {
    SolveState **stp = graph->st64;
    int32_t *nwp = graph->n_wet;
    int n = graph->n;
    double rtol = o.rtol, irt = o.inner_rtol;
    int mi = o.max_iter, mr = o.max_replace, mo = o.max_outer, bud = budget;
    LaunchState *ls = mixed ? L32->ls : L64->ls;
    void *args[] = {&stp, &nwp, &n, &rtol, &mi, &mr, &irt, &mo, &bud, &ls};
    CK(cudaLaunchKernel((const void *)k_ctl_begin, dim3(1), dim3(CTL_THREADS), args, 0, s));
    note_launches(1);
  }
  CK(cudaGraphLaunch(graph->exec, s));
  for (auto &m : M)
    if ((rc = member_store(m, s))) return rc;
  for (pcg_handle *h : members)
    CK(cudaMemcpyAsync(h->st_host, h->p64.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(pend->ls_host, mixed ? L32->ls : L64->ls, sizeof(LaunchState), cudaMemcpyDeviceToHost, s));
  pend->graph = true;
  pend->outer_kernels = graph->outer_kernels;
  pend->inner_kernels = graph->inner_kernels;
  CK(cudaEventCreateWithFlags(&pend->done, cudaEventDisableTiming));
  CK(cudaEventRecord(pend->done, s));
  for (pcg_handle *h : members) h->pending = pend;
  return PCG_OK;
}

}  // extern "C"
