// Internal host-side structures of libpcg shared by api.cu and server.cu.
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <cstdlib>
#include <memory>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "pcg_internal.h"

namespace pcg {

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_error(std::string(#call) + " failed: " + cudaGetErrorString(e_));                \
      return PCG_ECUDA;                                                                    \
    }                                                                                      \
  } while (0)

struct KernelSet {
  const void *k1[4] = {}, *k2[3] = {};      // per launch kind (K1_*, K2_*), fixed stride
  const void *k1_claim = nullptr, *k2_claim = nullptr;   // K1_ITER / K2_ITER claiming units (binary32 only)
  const void *fin = nullptr, *pack = nullptr, *unpack = nullptr;
  size_t smem1 = 0, smem2 = 0;
  int tx = 0;        // strip width: threads of the small kernels
  int tb = 0;        // threads of the stencil and preconditioner kernels (tx + a producer warp)
  int rb1 = 1, rb2 = 1;                       // rows per streamed group of the two kernels
  int ws = 0, we = 0, wt = 0, wr = 0, wz = 0; // box widths of the streamed fields
  int ctas1 = 0, ctas2 = 0;                   // resident CTAs on the device (persistent grid size)
  bool ok = false;
};

// The kernel of a loop launch: the claiming instantiation of an iteration
// kind where the plan claims and the set has one, else the fixed stride.
inline const void *loop_kernel(const KernelSet &ks, int which, int kind, bool dynamic) {
  if (which == 1) return (dynamic && kind == K1_ITER && ks.k1_claim) ? ks.k1_claim : ks.k1[kind];
  return (dynamic && kind == K2_ITER && ks.k2_claim) ? ks.k2_claim : ks.k2[kind];
}

// Strips whose preconditioner t phase (TX + 2R columns) fills whole warps:
// 64 - 2R columns for binary64, 124 for binary32 (a multiple of 4, for the
// 16-byte alignment of the tensor tiles), for tril(A) and tril(A^2).
inline int exact_width(int elem_size, int pattern) {
  if (pattern != PCG_PAT_TRIL_A && pattern != PCG_PAT_TRIL_A2) return 0;
  if (elem_size == 8) return pattern == PCG_PAT_TRIL_A2 ? 60 : 62;
  return 124;
}
// Wider binary64 strips, used on wide grids (see choose_tx): for tril(A) 124 columns, whose r'
// pass is 128 columns (4 whole warps) and whose t pass is 126; its ring is
// small enough for 5 CTAs per SM, and it beats two 62-column strips (fewer
// halo columns per point). For tril(A^2) 92 columns (t pass 96 = 3 whole
// warps, 4 CTAs per SM): 3 % fewer FP64 instructions per point than 60-column
// strips, and faster with units of at most 64 rows; at 124 columns its ring
// leaves 3 CTAs per SM, which is slower.
inline int wide_width(int elem_size, int pattern) {
  if (elem_size != 8) return 0;
  return pattern == PCG_PAT_TRIL_A ? 124 : pattern == PCG_PAT_TRIL_A2 ? 92 : 0;
}
// Tallest unit the makespan model may choose for a strip width: the 92-column
// binary64 tril(A^2) strips measured fastest with 48-64 rows at 4322 x 3059
// (0.577-0.581 ms per iteration, against 0.594 at the model's 96 and 0.606 at 128).
inline int max_unit_rows(int elem_size, int tx, int pattern) {
  return (elem_size == 8 && pattern == PCG_PAT_TRIL_A2 && tx == wide_width(8, pattern)) ? 64 : 128;
}
inline bool valid_width(int tx, int pattern) {
  return tx == 64 || tx == 128 || tx == exact_width(8, pattern) || tx == exact_width(4, pattern) ||
         tx == wide_width(8, pattern);
}

// Bound on every device wait of a launch (mbarrier waits of the streamed
// rings): PCG_WAIT_TIMEOUT_MS milliseconds if set and positive, else 2 s.
inline uint64_t default_timeout_ns() {
  const char *e = getenv("PCG_WAIT_TIMEOUT_MS");
  double ms = e ? atof(e) : 2000.0;
  if (!(ms > 0)) ms = 2000.0;
  return (uint64_t)(ms * 1e6);
}

// kernel sets per precision and strip width (kernels_*.cu)
KernelSet kernels_f64_64(int pattern, int q);
KernelSet kernels_f64_128(int pattern, int q);
KernelSet kernels_f64_exact(int tx, int pattern);
KernelSet kernels_f64_wide(int tx, int pattern);
KernelSet kernels_f32_64(int pattern, int q);
KernelSet kernels_f32_128(int pattern, int q);
KernelSet kernels_f32_exact(int tx, int pattern);

// CTAs of a launch of kernel 1 or 2 over n units: one per unit up to the
// number resident at once; the CTAs then stride over the units.
inline int persistent_grid(const KernelSet &k, int which, int n_units) {
  const int cap = which == 1 ? k.ctas1 : k.ctas2;
  return n_units < cap ? n_units : cap;
}

enum { PL_CE = 0, PL_CN, PL_A, PL_DINV, PL_Z0 };

template <typename T>
struct DevPlanes {
  int nx = 0, ny = 0, pitch = 0, gx = 0, tx = 0, ty = 0, nz = 0, nw = 0, n_units = 0;
  size_t plane_elems = 0;
  T *mem = nullptr;
  T *zwrap = nullptr;
  TensorMapBytes *tm = nullptr;    // device [TM_COUNT], when a kernel streams several rows per copy
  double *partial = nullptr;
  SolveState *st = nullptr;
  GridDev<T> gd{};
  GridDev<T> *gd_dev = nullptr;
  Unit *units_dev = nullptr;       // this grid alone (g = 0)
  std::vector<Unit> units;
  KernelSet ks;
  size_t bytes = 0;

  int plane_count() const { return PL_Z0 + nz + 8; }
  T *plane(int idx) const { return mem + (size_t)idx * plane_elems + (size_t)GY * pitch + gx; }
  T *plane_start(int idx) const { return mem + (size_t)idx * plane_elems; }
  int vec(int k) const { return PL_Z0 + nz + k; }   // 0 x, 1 s, 2 q, 3 r0, 4 r1, 5 d0, 6 d1, 7 b

  void release() {
    cudaFree(mem); cudaFree(zwrap); cudaFree(partial); cudaFree(st); cudaFree(gd_dev); cudaFree(units_dev);
    cudaFree(tm);
    mem = nullptr; zwrap = nullptr; partial = nullptr; st = nullptr; gd_dev = nullptr; units_dev = nullptr;
    tm = nullptr;
  }
};

// A whole-solve graph (csrc/solve.cu) over the members of a plan: outer
// conditional loop of passes, inner conditional loop of PCG iterations.
struct SolveGraph {
  cudaGraphExec_t exec = nullptr;
  SolveState **st64 = nullptr, **st32 = nullptr;   // device arrays of the members' states
  int32_t *n_wet = nullptr;                         // device array of the members' wet counts
  int n = 0;
  int outer_kernels = 0;    // kernel nodes of one pass outside the inner loop
  int inner_kernels = 0;    // kernel nodes of one inner loop body
  ~SolveGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    cudaFree(st64);
    cudaFree(st32);
    cudaFree(n_wet);
  }
};

// The grids advanced together by one loop: grouped by kernel set, each group
// with its descriptor array and concatenated unit list on the device.
struct PlanGroup {
  KernelSet ks;
  int n_units = 0;
  const void *gd_dev = nullptr;
  const Unit *units_dev = nullptr;
};

struct LoopPlan {
  std::vector<PlanGroup> groups;
  LaunchState *ls = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  bool graph_ok = false;
  int body_kernels = 0;            // kernel nodes in the loop body
  bool dynamic = false;            // iteration kernels claim units one at a time, where their set can
  std::vector<void *> owned;       // device allocations of a batch plan
  std::unique_ptr<SolveGraph> solve;   // whole-solve graph of a handle alone (built on first use)
  bool solve_tried = false;            // its construction was attempted (and may have failed)
  ~LoopPlan() {
    solve.reset();
    if (exec) cudaGraphExecDestroy(exec);
    for (void *p : owned) cudaFree(p);
  }
};

struct Pending;

}  // namespace pcg

struct pcg_handle {
  pcg::HostGrid G;
  pcg::HostFactor F;
  int pattern = 0, band_q = 0;
  double tau = 0.0;
  int tx = 0, ty = 0;                     // strips of the binary64 planes
  int tx32 = 0, ty32 = 0;                 // strips of the binary32 planes
  pcg::DevPlanes<double> p64;
  pcg::DevPlanes<float> p32;              // binary32 copies for the mixed-precision inner solves (lazy)
  pcg::SolveState *st32_host = nullptr;   // pinned mirror of p32's state
  pcg::LaunchState *ls = nullptr;        // device
  pcg::LaunchState *ls_host = nullptr;   // pinned
  pcg::SolveState *st_host = nullptr;    // pinned mirror
  double *stage = nullptr;               // device [ny][nx] staging for host buffers
  // Copies between host buffers and stage. A solve's copies run on the
  // handle's copy stream, so that they overlap other work on the solve's
  // stream (another handle's solve); every other call copies on its own stream.
  // ev_stage marks the last enqueued use of stage, whichever stream it is on.
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_unpacked = nullptr, ev_stage = nullptr;
  std::unique_ptr<pcg::LoopPlan> plan64;
  std::unique_ptr<pcg::LoopPlan> plan32;
  size_t bytes = 0;
  uint64_t serial = 0;                    // process-unique number of this handle
  uint32_t version = 0;                   // bumped whenever its device planes are rebuilt
  std::shared_ptr<pcg::Pending> pending;  // the solve enqueued on it and not yet synchronised
  int last_status = PCG_OK;               // status of its last synchronised solve
};

namespace pcg {

// A solve call enqueued and not yet synchronised (pcg_sync). Every member
// handle of the call points to it.
struct Pending {
  std::shared_ptr<void> keep;             // batch plan whose graph the enqueued work runs
  std::vector<pcg_handle *> hs;           // members, in call order
  pcg_stats *stats = nullptr;             // caller's [hs.size()] statistics, filled at synchronisation
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;             // recorded on s after the call's last work there
  bool mixed = false;
  bool graph = false;                     // run by a whole-solve graph (else solved at the call)
  int status = PCG_OK;                    // status of a call solved at the call
  int outer_kernels = 0, inner_kernels = 0;
  LaunchState *ls_host = nullptr;         // pinned copy of the launch state, for the launch count
  std::chrono::steady_clock::time_point t0;
  Pending() = default;
  Pending(const Pending &) = delete;
  Pending &operator=(const Pending &) = delete;
  ~Pending() {
    if (done) cudaEventDestroy(done);
  }
};

}  // namespace pcg

namespace pcg {

// one grid of a solve in progress
struct Member {
  pcg_handle *h = nullptr;
  const double *b = nullptr;
  double *x = nullptr;
  pcg_stats *stats = nullptr;
  SolveState *st_host = nullptr;
  int replacements = 0;
  int final_status = -1;
  // mixed precision bookkeeping
  int inner_iters = 0, inner_solves = 0;
  double relres64 = 0.0;
  double scale = 1.0;
};

// phases of a solve, shared by pcg_solve_batched and the solver server
int member_load(Member &m, const pcg_opts &o, bool pack_x0, cudaStream_t s);     // inputs and state
int member_pack(Member &m, const pcg_opts &o, cudaStream_t s);                   // inputs only (b, x0, d = 0)
int solve_members64(LoopPlan &L, LaunchState *ls_host, std::vector<Member> &M, const pcg_opts &o, cudaStream_t s);
void handle_init_serial(pcg_handle *h);
// Wait for the solve enqueued on h, if any, and release it; returns its status.
int handle_finish_pending(pcg_handle *h);
int members_arm(LoopPlan &L, LaunchState *ls_host, int active, int max_launches, cudaStream_t s);
int members_init(LoopPlan &L, cudaStream_t s);                                   // r0, s0, rho0 for not-done grids
int members_loop(LoopPlan &L, LaunchState *ls_host, int max_launches, cudaStream_t s);
int members_close(LoopPlan &L, cudaStream_t s);                                  // x update, true residual
// After members_close and a read-back of the states: decide per member. Returns
// true if it must restart (its done flag has been cleared on the device).
bool member_decide(Member &m, const pcg_opts &o, bool overrun, cudaStream_t s, int *err);
int member_store(Member &m, cudaStream_t s);                                      // unpack x
void member_stats(Member &m);
int plan_single(pcg_handle *h);                                                   // h->plan64
int upload_planes64(pcg_handle *h, cudaStream_t s);   // h->p64 from h->G, h->F, h->tx, h->ty
int ensure_f32(pcg_handle *h, cudaStream_t s);                                     // h->p32, h->plan32
int plan_build32(LoopPlan &L, pcg_handle *const *hs, int n, bool with_graph, LaunchState *ls, cudaStream_t s);
int solve_members_mixed(LoopPlan &L64, LoopPlan &L32, LaunchState *ls_host, std::vector<Member> &M,
                        const pcg_opts &o, cudaStream_t s);
bool mixed_prepare_inner(Member &m, const pcg_opts &o, int budget, int outer, cudaStream_t s, int *err);
int mixed_apply_correction(Member &m, cudaStream_t s);
void mixed_stats(Member &m);
// which: 1 stencil kernel, 2 preconditioner kernel, 0 final x update; kind: K1_* / K2_*
int single_launch(pcg_handle *h, bool f32, int which, int kind, cudaStream_t s);
int plan_build(LoopPlan &L, pcg_handle *const *hs, int n, bool with_graph, LaunchState *ls, cudaStream_t s);
// One-operand applies (no solve state of their own): clear the status word of
// the grid's device state before the launch; after it, synchronise the stream
// and return the status a kernel recorded there (PCG_ETIMEOUT when one of its
// bounded waits gave up), PCG_OK otherwise.
int apply_status_clear(SolveState *st, cudaStream_t s);
// Count kernel launches issued outside api.cu (pcg_kernel_launches).
void note_launches(uint64_t n);
int apply_status_read(SolveState *st, cudaStream_t s);
std::string status_name(int s);
void fill_opts(const pcg_opts *o, pcg_opts &out);
bool is_device_ptr(const void *p);

}  // namespace pcg
