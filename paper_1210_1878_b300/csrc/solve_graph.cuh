// Whole-solve graphs: the device-side control kernels of a solve (defined in
// solve.cu) and the helpers that add the loop kernels of a plan to a graph.
// Shared by solve.cu (single grids and batches) and shard.cu (row bands).
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <vector>

#include "handle.cuh"

namespace pcg {

constexpr int CTL_THREADS = 256;
constexpr int MAX_PASSES = 1024;   // runaway guard of the outer loop of a solve graph

__global__ void k_ctl_begin(SolveState *const *st, const int32_t *n_wet, int n, double rtol, int max_iter_opt,
                            int max_replace, double inner_rtol, int max_outer, int budget, LaunchState *ls);
__global__ void k_ctl_arm(SolveState *const *st, int n, LaunchState *ls, cudaGraphConditionalHandle cond_in,
                          uint64_t budget_ns);
__global__ void k_ctl_decide64(SolveState *const *st, int n, LaunchState *ls, cudaGraphConditionalHandle cond_out);

// ------------------------------------------------------------ graph building
struct Builder {
  cudaGraph_t g = nullptr;
  std::vector<cudaGraphNode_t> deps;
  cudaError_t err = cudaSuccess;
  int kernels = 0;

  explicit Builder(cudaGraph_t graph) : g(graph) {}
  void kernel(const void *f, dim3 grid, dim3 block, size_t smem, void **args) {
    if (err != cudaSuccess || grid.x == 0) return;
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(f);
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    cudaGraphNode_t node;
    err = cudaGraphAddKernelNode(&node, g, deps.empty() ? nullptr : deps.data(), deps.size(), &kp);
    if (err == cudaSuccess) { deps.assign(1, node); ++kernels; }
  }
  // A WHILE node on `h` after the current dependencies; returns its body graph.
  cudaGraph_t while_node(cudaGraphConditionalHandle h) {
    if (err != cudaSuccess) return nullptr;
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    err = cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp);
    if (err != cudaSuccess) return nullptr;
    deps.assign(1, node);
    return cp.conditional.phGraph_out[0];
  }
};

// The persistent loop kernels of every group of L (one launch kind), as nodes.
inline void add_groups(Builder &B, const LoopPlan &L, int which, int kind, int use_cond, bool guard_first) {
  bool guarded = false;
  for (const PlanGroup &G : L.groups) {
    if (G.n_units <= 0) continue;
    const int guard = (guard_first && !guarded) ? 1 : 0;
    guarded = guarded || guard;
    KParams p{};
    p.grids = G.gd_dev;
    p.units = G.units_dev;
    p.ls = L.ls;
    p.kind = kind;
    p.use_cond = use_cond;
    p.guard = guard;
    p.dbg_skip_unit = -1;
    p.timeout_ns = default_timeout_ns();
    p.n_units = G.n_units;
    void *args[] = {&p};
    if (which == 1)
      B.kernel(loop_kernel(G.ks, 1, kind, L.dynamic), dim3(persistent_grid(G.ks, 1, G.n_units)), dim3(G.ks.tb),
               G.ks.smem1, args);
    else
      B.kernel(loop_kernel(G.ks, 2, kind, L.dynamic), dim3(persistent_grid(G.ks, 2, G.n_units)), dim3(G.ks.tb),
               G.ks.smem2, args);
  }
}

inline void add_finalize(Builder &B, const LoopPlan &L) {
  for (const PlanGroup &G : L.groups) {
    if (G.n_units <= 0) continue;
    KParams p{};
    p.grids = G.gd_dev;
    p.units = G.units_dev;
    p.ls = L.ls;
    p.dbg_skip_unit = -1;
    void *args[] = {&p};
    B.kernel(G.ks.fin, dim3(G.n_units), dim3(G.ks.tx), 0, args);
  }
}

inline uint64_t loop_budget_ns() {
  const char *e = getenv("PCG_LOOP_BUDGET_S");
  const double budget_s = (e && atof(e) > 0) ? atof(e) : 300.0;
  return (uint64_t)(budget_s * 1e9);
}

}  // namespace pcg
