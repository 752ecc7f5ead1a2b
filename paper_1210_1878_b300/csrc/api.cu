// Host side of libpcg: device planes, launch plans, the device-resident PCG
// loop (a CUDA graph whose conditional WHILE node repeats the two kernels of
// an iteration until every grid's stopping test has fired), and the C ABI.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "handle.cuh"

namespace pcg {

static thread_local std::string g_err;
void set_error(const std::string &m) { g_err = m; }


// ------------------------------------------------------------ kernel table
// The kernel instantiations live in kernels_*.cu (compiled in parallel).
template <typename T>
static KernelSet pick(int tx, int pattern, int q) {
  if constexpr (sizeof(T) == 8) {
    if (tx == 64) return kernels_f64_64(pattern, q);
    if (tx == 128) return kernels_f64_128(pattern, q);
    if (tx == exact_width(8, pattern)) return kernels_f64_exact(tx, pattern);
    if (tx == wide_width(8, pattern)) return kernels_f64_wide(tx, pattern);
  } else {
    if (tx == 64) return kernels_f32_64(pattern, q);
    if (tx == 128) return kernels_f32_128(pattern, q);
    if (tx == exact_width(4, pattern)) return kernels_f32_exact(tx, pattern);
  }
  return KernelSet{};
}

static std::mutex g_attr_mu;
static int prepare_set(KernelSet &k) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  // every instantiation of each kernel, the claiming ones included (they share
  // the persistent grid size)
  std::vector<const void *> f1(k.k1, k.k1 + 4), f2(k.k2, k.k2 + 3);
  if (k.k1_claim) f1.push_back(k.k1_claim);
  if (k.k2_claim) f2.push_back(k.k2_claim);
  for (const void *f : f1) CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem1));
  for (const void *f : f2) CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem2));
  int dev = 0, nsm = 0, b1 = 0, b2 = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  b1 = b2 = 1 << 20;
  for (const void *f : f1) {
    int b = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, k.tb, k.smem1));
    b1 = std::min(b1, b);
  }
  for (const void *f : f2) {
    int b = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, k.tb, k.smem2));
    b2 = std::min(b2, b);
  }
  if (b1 < 1 || b2 < 1) { set_error("kernel does not fit on an SM"); return PCG_ECUDA; }
  k.ctas1 = b1 * nsm;
  k.ctas2 = b2 * nsm;
  return PCG_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

static_assert(sizeof(CUtensorMap) == sizeof(TensorMapBytes), "tensor map size");

}  // namespace pcg

namespace pcg {

static size_t elem_round(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Tensor map of plane idx (all stored columns and rows, row-major with the
// plane's pitch) whose box is w columns by rb rows.
template <typename T>
static int make_tensor_map(TensorMapBytes &out, const DevPlanes<T> &P, int idx, int w, int rb) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) { set_error("cuTensorMapEncodeTiled unavailable"); return PCG_ECUDA; }
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)P.pitch, (cuuint64_t)(P.ny + 2 * GY)};
  const cuuint64_t strides[1] = {(cuuint64_t)P.pitch * sizeof(T)};
  const cuuint32_t box[2] = {(cuuint32_t)w, (cuuint32_t)rb};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(&m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                         (void *)P.plane_start(idx), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_error("tensor map encoding failed (" + std::to_string((int)r) + ")"); return PCG_ECUDA; }
  std::memcpy(&out, &m, sizeof(m));
  return PCG_OK;
}

template <typename T>
static int upload_tensor_maps(DevPlanes<T> &P) {
  const KernelSet &k = P.ks;
  if (k.rb1 == 1 && k.rb2 == 1) return PCG_OK;
  std::vector<TensorMapBytes> tm(TM_COUNT);
  std::memset(tm.data(), 0, sizeof(TensorMapBytes) * TM_COUNT);
  int rc;
  struct Spec { int slot, plane, w, rb; };
  std::vector<Spec> specs;
  if (k.rb1 > 1) {
    specs.insert(specs.end(), {{TM_WS_S, P.vec(1), k.ws, k.rb1}, {TM_WS_D0, P.vec(5), k.ws, k.rb1},
                               {TM_WS_D1, P.vec(6), k.ws, k.rb1}, {TM_WS_X, P.vec(0), k.ws, k.rb1},
                               {TM_WT_CN, PL_CN, k.wt, k.rb1}, {TM_WT_A, PL_A, k.wt, k.rb1},
                               {TM_WT_X, P.vec(0), k.wt, k.rb1}, {TM_WT_B, P.vec(7), k.wt, k.rb1},
                               {TM_WE_CE, PL_CE, k.we, k.rb1}});
  }
  if (k.rb2 > 1) {
    specs.insert(specs.end(), {{TM_WR_R0, P.vec(3), k.wr, k.rb2}, {TM_WR_R1, P.vec(4), k.wr, k.rb2},
                               {TM_WR_Q, P.vec(2), k.wr, k.rb2}, {TM_WZ_DI, PL_DINV, k.wz, k.rb2}});
    for (int z = 0; z < P.nz; ++z) specs.push_back({TM_WZ_Z0 + z, PL_Z0 + z, k.wz, k.rb2});
  }
  for (const Spec &sp : specs)
    if ((rc = make_tensor_map<T>(tm[sp.slot], P, sp.plane, sp.w, sp.rb))) return rc;
  CK(cudaMalloc(&P.tm, sizeof(TensorMapBytes) * TM_COUNT));
  CK(cudaMemcpy(P.tm, tm.data(), sizeof(TensorMapBytes) * TM_COUNT, cudaMemcpyHostToDevice));
  P.bytes += sizeof(TensorMapBytes) * TM_COUNT;
  return PCG_OK;
}

template <typename T>
static int upload_planes(pcg_handle *h, DevPlanes<T> &P, cudaStream_t s) {
  const HostGrid &G = h->G;
  const HostFactor &F = h->F;
  P.nx = G.nx; P.ny = G.ny;
  P.tx = sizeof(T) == 4 ? h->tx32 : h->tx;
  P.ty = sizeof(T) == 4 ? h->ty32 : h->ty;
  P.gx = 128 / (int)sizeof(T);
  const int ntx = (G.nx + P.tx - 1) / P.tx;
  if (ntx > INT16_MAX || (G.ny + P.ty - 1) / P.ty > INT16_MAX) {   // strip coordinates are 16-bit
    set_error("more than 32767 strips in one direction: use wider (tile_x) or taller (tile_y) strips");
    return PCG_EINVAL;
  }
  P.pitch = (int)elem_round((size_t)P.gx + (size_t)ntx * P.tx + P.gx, 128 / sizeof(T));
  P.nz = F.slots.n; P.nw = F.slots.n_wrap;
  P.plane_elems = (size_t)(G.ny + 2 * GY) * P.pitch;
  P.ks = pick<T>(P.tx, h->pattern, h->band_q);
  if (!P.ks.ok) { set_error("no kernel for this pattern / tile width"); return PCG_EINVAL; }
  int rc = prepare_set(P.ks);
  if (rc) return rc;
  // units: strips holding a wet cell
  const int nty = (G.ny + P.ty - 1) / P.ty;
  P.units.clear();
  for (int sy = 0; sy < nty; ++sy)
    for (int sx = 0; sx < ntx; ++sx) {
      bool any = false;
      for (int j = sy * P.ty; j < std::min(G.ny, (sy + 1) * P.ty) && !any; ++j)
        for (int i = sx * P.tx; i < std::min(G.nx, (sx + 1) * P.tx); ++i)
          if (G.idx[(size_t)j * G.nx + i] >= 0) { any = true; break; }
      if (any) {
        Unit u{};
        u.g = 0; u.sx = (int16_t)sx; u.sy = (int16_t)sy; u.u = (int32_t)P.units.size();
        P.units.push_back(u);
      }
    }
  P.n_units = (int)P.units.size();
  const size_t nplanes = P.plane_count();
  const size_t bytes_planes = nplanes * P.plane_elems * sizeof(T);
  if (cudaMalloc(&P.mem, bytes_planes) != cudaSuccess) { cudaGetLastError(); set_error("device allocation of the grid planes failed"); return PCG_ENOMEM; }
  CK(cudaMemsetAsync(P.mem, 0, bytes_planes, s));
  CK(cudaMalloc(&P.zwrap, sizeof(T) * (size_t)G.ny * std::max(P.nw, 1)));
  CK(cudaMalloc(&P.partial, sizeof(double) * 2 * (size_t)std::max(P.n_units, 1)));
  CK(cudaMalloc(&P.st, sizeof(SolveState)));
  CK(cudaMemsetAsync(P.st, 0, sizeof(SolveState), s));
  CK(cudaMalloc(&P.gd_dev, sizeof(GridDev<T>)));
  CK(cudaMalloc(&P.units_dev, sizeof(Unit) * (size_t)std::max(P.n_units, 1)));
  P.bytes = bytes_planes + sizeof(T) * (size_t)G.ny * std::max(P.nw, 1) + sizeof(double) * 2 * P.n_units +
            sizeof(SolveState) + sizeof(GridDev<T>) + sizeof(Unit) * P.n_units;

  // static planes, built on the host row by row with their periodic copies
  std::vector<T> buf(P.plane_elems);
  auto put = [&](int idx, auto value_of) -> int {
    std::fill(buf.begin(), buf.end(), (T)0);
    for (int j = 0; j < G.ny; ++j) {
      T *row = buf.data() + (size_t)(j + GY) * P.pitch + P.gx;
      for (int i = 0; i < G.nx; ++i) row[i] = (T)value_of(i, j);
      for (int c = -GHOST; c < 0; ++c) row[c] = row[((c % G.nx) + G.nx) % G.nx];
      for (int c = G.nx; c < G.nx + GHOST; ++c) row[c] = row[c % G.nx];
    }
    CK(cudaMemcpy(P.mem + (size_t)idx * P.plane_elems, buf.data(), P.plane_elems * sizeof(T), cudaMemcpyHostToDevice));
    return PCG_OK;
  };
  auto kk = [&](int i, int j) { return G.idx[(size_t)j * G.nx + i]; };
  if ((rc = put(PL_CE, [&](int i, int j) { return G.ce[(size_t)j * G.nx + i]; }))) return rc;
  if ((rc = put(PL_CN, [&](int i, int j) { return G.cn[(size_t)j * G.nx + i]; }))) return rc;
  if ((rc = put(PL_A, [&](int i, int j) { int k = kk(i, j); return k >= 0 ? G.diag[k] : 0.0; }))) return rc;
  if ((rc = put(PL_DINV, [&](int i, int j) { int k = kk(i, j); return k >= 0 ? 1.0 / F.d[k] : 0.0; }))) return rc;
  for (int sidx = 0; sidx < P.nz; ++sidx)
    if ((rc = put(PL_Z0 + sidx, [&](int i, int j) { int k = kk(i, j); return k >= 0 ? F.z[(size_t)sidx * F.n + k] : 0.0; }))) return rc;
  if (P.nw > 0) {
    std::vector<T> zw((size_t)G.ny * P.nw);
    for (size_t e = 0; e < zw.size(); ++e) zw[e] = (T)F.zwrap[e];
    CK(cudaMemcpy(P.zwrap, zw.data(), sizeof(T) * zw.size(), cudaMemcpyHostToDevice));
  }
  // descriptor
  GridDev<T> &gd = P.gd;
  std::memset(&gd, 0, sizeof(gd));
  gd.nx = G.nx; gd.ny = G.ny; gd.pitch = P.pitch; gd.ty = P.ty;
  gd.n_units = P.n_units; gd.n_wrap = P.nw;
  gd.ce = P.plane(PL_CE); gd.cn = P.plane(PL_CN); gd.a = P.plane(PL_A); gd.dinv = P.plane(PL_DINV);
  for (int sidx = 0; sidx < P.nz; ++sidx) gd.z[sidx] = P.plane(PL_Z0 + sidx);
  gd.zwrap = P.zwrap;
  gd.x = P.plane(P.vec(0)); gd.s = P.plane(P.vec(1)); gd.q = P.plane(P.vec(2));
  gd.r[0] = P.plane(P.vec(3)); gd.r[1] = P.plane(P.vec(4));
  gd.d[0] = P.plane(P.vec(5)); gd.d[1] = P.plane(P.vec(6));
  gd.b = P.plane(P.vec(7));
  gd.partial = P.partial; gd.st = P.st;
  gd.row_off = 0; gd.own0 = 0; gd.own1 = G.ny;
  if ((rc = upload_tensor_maps(P))) return rc;
  gd.tm = P.tm;
  CK(cudaMemcpy(P.gd_dev, &gd, sizeof(gd), cudaMemcpyHostToDevice));
  if (P.n_units > 0) CK(cudaMemcpy(P.units_dev, P.units.data(), sizeof(Unit) * P.n_units, cudaMemcpyHostToDevice));
  return PCG_OK;
}

static KParams kparams(const LoopPlan &L, const PlanGroup &g, int kind, int use_cond, int guard) {
  KParams p{};
  p.grids = g.gd_dev;
  p.units = g.units_dev;
  p.ls = L.ls;
  p.kind = kind;
  p.use_cond = use_cond;
  p.guard = guard;
  p.dbg_skip_unit = -1;
  p.timeout_ns = default_timeout_ns();
  return p;
}

static std::atomic<uint64_t> g_launches{0};
void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static int launch(const void *f, int grid, int block, size_t smem, KParams p, cudaStream_t s) {
  if (grid <= 0) return PCG_OK;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  void *args[] = {&p};
  CK(cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s));
  return PCG_OK;
}

// Kernel 1 (which = 1) or 2 over n_units units, persistent CTAs (claiming
// units where `dynamic` and the set has a claiming instantiation of the kind).
static int launch_k(const KernelSet &ks, int which, int n_units, KParams p, cudaStream_t s, bool dynamic = false) {
  p.n_units = n_units;
  if (p.kind < 0 || p.kind >= (which == 1 ? 4 : 3)) { set_error("invalid launch kind"); return PCG_EINVAL; }
  return launch(loop_kernel(ks, which, p.kind, dynamic), persistent_grid(ks, which, n_units), ks.tb,
                which == 1 ? ks.smem1 : ks.smem2, p, s);
}

static int build_loop_graph(LoopPlan &L) {
  if (getenv("PCG_LOOP_CHUNKED")) return PCG_ECUDA;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) { cudaGetLastError(); cudaGraphDestroy(g); set_error("conditional graphs unavailable"); return PCG_ECUDA; }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  e = cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &cp);
  if (e != cudaSuccess) { cudaGetLastError(); cudaGraphDestroy(g); set_error("conditional node unavailable"); return PCG_ECUDA; }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  // kernel params must outlive node creation only (they are copied)
  std::vector<KParams> params;
  params.reserve(2 * L.groups.size());
  std::vector<void *> argv(2 * L.groups.size());
  cudaGraphNode_t prev = nullptr;
  bool have_prev = false, guarded = false;
  for (int pass = 0; pass < 2; ++pass) {
    for (size_t gi = 0; gi < L.groups.size(); ++gi) {
      const PlanGroup &G = L.groups[gi];
      if (G.n_units <= 0) continue;
      const int guard = (pass == 1 && !guarded) ? 1 : 0;   // the first preconditioner launch of the body
      guarded = guarded || guard;
      params.push_back(kparams(L, G, pass == 0 ? (int)K1_ITER : (int)K2_ITER, 1, guard));
      params.back().n_units = G.n_units;
      void *args[] = {&params.back()};
      cudaKernelNodeParams kp{};
      kp.func = const_cast<void *>(loop_kernel(G.ks, pass == 0 ? 1 : 2, pass == 0 ? (int)K1_ITER : (int)K2_ITER,
                                               L.dynamic));
      kp.gridDim = dim3(persistent_grid(G.ks, pass == 0 ? 1 : 2, G.n_units));
      kp.blockDim = dim3(G.ks.tb);
      kp.sharedMemBytes = (unsigned)(pass == 0 ? G.ks.smem1 : G.ks.smem2);
      kp.kernelParams = args;
      cudaGraphNode_t node;
      e = cudaGraphAddKernelNode(&node, body, have_prev ? &prev : nullptr, have_prev ? 1 : 0, &kp);
      if (e != cudaSuccess) { cudaGetLastError(); cudaGraphDestroy(g); set_error("kernel node creation failed"); return PCG_ECUDA; }
      prev = node; have_prev = true;
    }
  }
  if (!guarded) { cudaGraphDestroy(g); set_error("no work units: no loop graph"); return PCG_ECUDA; }
  L.body_kernels = (int)params.size();
  e = cudaGraphInstantiate(&L.exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { cudaGetLastError(); L.exec = nullptr; set_error("graph instantiation failed"); return PCG_ECUDA; }
  L.cond = h;
  L.graph_ok = true;
  return PCG_OK;
}

// Arm the plan's launch state: `active` grids still iterating, a cap of
// max_launches loop bodies. Must precede the init kernels of a round, so that
// grids finishing already there are counted off.
int members_arm(LoopPlan &L, LaunchState *ls_host, int active, int max_launches, cudaStream_t s) {
  ls_host->active = active;
  ls_host->launches = 0;
  ls_host->max_launches = max_launches;
  ls_host->stop = 0;
  ls_host->cond = L.cond;
  ls_host->t0_ns = 0;
  ls_host->timed_out = 0;
  ls_host->cond_cleared = 0;
  ls_host->claim_next = 0;
  ls_host->claim_exit = 0;
  const char *e = getenv("PCG_LOOP_BUDGET_S");
  const double budget_s = (e && atof(e) > 0) ? atof(e) : 300.0;
  ls_host->budget_ns = (uint64_t)(budget_s * 1e9);
  CK(cudaMemcpyAsync(L.ls, ls_host, sizeof(LaunchState), cudaMemcpyHostToDevice, s));
  return PCG_OK;
}

// Run the loop body until every grid of the plan is done, or max_launches
// bodies have run (the guard in the first stencil launch ends it).
int members_loop(LoopPlan &L, LaunchState *ls_host, int max_launches, cudaStream_t s) {
  if (L.graph_ok) {
    CK(cudaGraphLaunch(L.exec, s));
    return PCG_OK;
  }
  // without conditional graphs: chunks of iterations, polling the active count
  const int chunk = 16;
  for (int done = 0; done < max_launches;) {
    const int n = std::min(chunk, max_launches - done);
    for (int c = 0; c < n; ++c) {
      bool guarded = false;
      for (int pass = 0; pass < 2; ++pass)
        for (size_t gi = 0; gi < L.groups.size(); ++gi) {
          const PlanGroup &G = L.groups[gi];
          if (G.n_units <= 0) continue;
          const int guard = (pass == 1 && !guarded) ? 1 : 0;
          guarded = guarded || guard;
          int rc = launch_k(G.ks, pass == 0 ? 1 : 2, G.n_units,
                            kparams(L, G, pass == 0 ? (int)K1_ITER : (int)K2_ITER, 0, guard), s, L.dynamic);
          if (rc) return rc;
        }
    }
    done += n;
    CK(cudaMemcpyAsync(ls_host, L.ls, sizeof(LaunchState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ls_host->active <= 0 || ls_host->stop) break;
  }
  return PCG_OK;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Pack a user [ny][nx] binary64 vector into plane `which` (0 b, 1 x, 2 r0, 3 d0).
// A host `user` vector goes through h->stage: copied on s, or with
// `on_copy_stream` on the handle's copy stream (s then waits for the copy).
// Either way the copy waits for the previous use of stage.
template <typename T>
static int pack_user(pcg_handle *h, DevPlanes<T> &P, const double *user, int which, cudaStream_t s,
                     bool on_copy_stream = false) {
  const double *srcp = user;
  const bool host = !is_device_ptr(user);
  if (host) {
    const size_t bytes = sizeof(double) * (size_t)P.nx * P.ny;
    if (on_copy_stream) {
      CK(cudaStreamWaitEvent(h->copy_stream, h->ev_stage, 0));
      CK(cudaMemcpyAsync(h->stage, user, bytes, cudaMemcpyHostToDevice, h->copy_stream));
      CK(cudaEventRecord(h->ev_in, h->copy_stream));
      CK(cudaStreamWaitEvent(s, h->ev_in, 0));
    } else {
      CK(cudaStreamWaitEvent(s, h->ev_stage, 0));
      CK(cudaMemcpyAsync(h->stage, user, bytes, cudaMemcpyHostToDevice, s));
    }
    srcp = h->stage;
  }
  KParams p{};
  p.grids = P.gd_dev; p.units = P.units_dev;
  if (P.n_units > 0) {
    void *args[] = {&p, (void *)&srcp, &which};
    g_launches.fetch_add(1, std::memory_order_relaxed);
    CK(cudaLaunchKernel(P.ks.pack, dim3(P.n_units), dim3(P.tx), args, 0, s));
  }
  if (host) CK(cudaEventRecord(h->ev_stage, s));   // stage is free once the pack has read it
  return PCG_OK;
}

// Unpack plane `which` (0 x, 1 s, 2 q) into a user [ny][nx] binary64 vector.
// A host `user` vector goes through h->stage (after its previous use), copied
// back on s, or with `on_copy_stream` on the handle's copy stream.
template <typename T>
static int unpack_user(pcg_handle *h, DevPlanes<T> &P, double *user, int which, cudaStream_t s,
                       bool on_copy_stream = false) {
  const bool dev = is_device_ptr(user);
  double *dst = dev ? user : h->stage;
  if (!dev) CK(cudaStreamWaitEvent(s, h->ev_stage, 0));
  const GridDev<T> *gdp = P.gd_dev;
  void *args[] = {(void *)&gdp, (void *)&dst, &which};
  const size_t n = (size_t)P.nx * P.ny;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  CK(cudaLaunchKernel(P.ks.unpack, dim3(std::max(blocks, 1)), dim3(256), args, 0, s));
  if (!dev) {
    if (on_copy_stream) {
      CK(cudaEventRecord(h->ev_unpacked, s));
      CK(cudaStreamWaitEvent(h->copy_stream, h->ev_unpacked, 0));
      CK(cudaMemcpyAsync(user, h->stage, sizeof(double) * n, cudaMemcpyDeviceToHost, h->copy_stream));
      CK(cudaEventRecord(h->ev_stage, h->copy_stream));
    } else {
      CK(cudaMemcpyAsync(user, h->stage, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(h->ev_stage, s));
    }
  }
  return PCG_OK;
}

int upload_planes64(pcg_handle *h, cudaStream_t s) { return upload_planes<double>(h, h->p64, s); }

int plan_single(pcg_handle *h) {
  if (h->plan64) return PCG_OK;
  auto L = std::make_unique<LoopPlan>();
  PlanGroup g;
  g.ks = h->p64.ks;
  g.n_units = h->p64.n_units;
  g.gd_dev = h->p64.gd_dev;
  g.units_dev = h->p64.units_dev;
  L->groups.push_back(g);
  L->ls = h->ls;
  if (build_loop_graph(*L) != PCG_OK) L->graph_ok = false;
  g_err.clear();
  h->plan64 = std::move(L);
  return PCG_OK;
}

// Plan over several grids: members grouped by kernel set.
template <typename T>
static int plan_build_t(LoopPlan &L, pcg_handle *const *hs, int n, bool with_graph, LaunchState *ls,
                        DevPlanes<T> pcg_handle::*planes, cudaStream_t s) {
  if (n > INT16_MAX) { set_error("more than 32767 grids in one plan"); return PCG_EINVAL; }   // 16-bit grid index
  L.ls = ls;
  // Claiming pays where the units finish unevenly: the grids of a batch differ
  // in size and retire at different iterations. The binary64 kernels keep the
  // fixed stride, which gives each SM's FP64 pipe an equal share (their sets
  // have no claiming instantiation).
  L.dynamic = n > 1;
  std::vector<std::vector<int>> groups;
  for (int i = 0; i < n; ++i) {
    bool placed = false;
    for (auto &g : groups)
      if ((hs[g[0]]->*planes).ks.k2[0] == (hs[i]->*planes).ks.k2[0] &&
          (hs[g[0]]->*planes).ks.k1[0] == (hs[i]->*planes).ks.k1[0]) {
        g.push_back(i); placed = true; break;
      }
    if (!placed) groups.push_back({i});
  }
  for (auto &g : groups) {
    std::vector<GridDev<T>> gds;
    std::vector<Unit> units;
    for (size_t mi = 0; mi < g.size(); ++mi) {
      auto &P = hs[g[mi]]->*planes;
      gds.push_back(P.gd);
      gds.back().u_off = (int32_t)units.size();       // the member's units are contiguous
      for (Unit u : P.units) { u.g = (int16_t)mi; units.push_back(u); }
    }
    void *gd_dev = nullptr, *un_dev = nullptr;
    CK(cudaMalloc(&gd_dev, sizeof(GridDev<T>) * gds.size()));
    L.owned.push_back(gd_dev);
    CK(cudaMalloc(&un_dev, sizeof(Unit) * std::max<size_t>(units.size(), 1)));
    L.owned.push_back(un_dev);
    CK(cudaMemcpyAsync(gd_dev, gds.data(), sizeof(GridDev<T>) * gds.size(), cudaMemcpyHostToDevice, s));
    if (!units.empty()) CK(cudaMemcpyAsync(un_dev, units.data(), sizeof(Unit) * units.size(), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));   // the host vectors above go out of scope
    PlanGroup pg;
    pg.ks = (hs[g[0]]->*planes).ks;
    pg.n_units = (int)units.size();
    pg.gd_dev = gd_dev;
    pg.units_dev = (const Unit *)un_dev;
    L.groups.push_back(pg);
  }
  if (with_graph && build_loop_graph(L) != PCG_OK) L.graph_ok = false;
  g_err.clear();
  return PCG_OK;
}

int plan_build(LoopPlan &L, pcg_handle *const *hs, int n, bool with_graph, LaunchState *ls, cudaStream_t s) {
  return plan_build_t<double>(L, hs, n, with_graph, ls, &pcg_handle::p64, s);
}

int plan_build32(LoopPlan &L, pcg_handle *const *hs, int n, bool with_graph, LaunchState *ls, cudaStream_t s) {
  return plan_build_t<float>(L, hs, n, with_graph, ls, &pcg_handle::p32, s);
}

// The binary32 planes of a handle (coefficients, Z and D^-1 rounded to
// binary32; same strips and units as the binary64 planes) and their loop plan.
int ensure_f32(pcg_handle *h, cudaStream_t s) {
  if (h->plan32) return PCG_OK;
  int rc = upload_planes<float>(h, h->p32, s);
  if (rc) { h->p32.release(); return rc; }
  if (!h->st32_host && cudaMallocHost(&h->st32_host, sizeof(SolveState)) != cudaSuccess) {
    cudaGetLastError(); set_error("pinned allocation failed"); return PCG_ENOMEM;
  }
  h->bytes += h->p32.bytes;
  auto L = std::make_unique<LoopPlan>();
  L->ls = h->ls;
  PlanGroup g;
  g.ks = h->p32.ks;
  g.n_units = h->p32.n_units;
  g.gd_dev = h->p32.gd_dev;
  g.units_dev = h->p32.units_dev;
  L->groups.push_back(g);
  if (build_loop_graph(*L) != PCG_OK) L->graph_ok = false;
  g_err.clear();
  h->plan32 = std::move(L);
  return PCG_OK;
}

void fill_opts(const pcg_opts *o, pcg_opts &out) {
  if (o) out = *o;
  else { std::memset(&out, 0, sizeof(out)); out.rtol = 1e-10; }
  if (!(out.rtol >= 0.0)) out.rtol = 1e-10;
  if (out.max_replace < 0) out.max_replace = 3;
  if (out.inner_rtol <= 0) out.inner_rtol = 1e-5;
  if (out.max_outer <= 0) out.max_outer = 30;
}

// Inputs of one member: b, x0 (or x = 0; with pack_x0 false and use_x0 set,
// the x plane keeps the grid's last solution: a warm start), zeroed
// directions, and the device state.
static int member_inputs(Member &m, const pcg_opts &o, bool pack_x0, cudaStream_t s) {
  auto &P = m.h->p64;
  int rc;
  if ((rc = pack_user(m.h, m.h->p64, m.b, 0, s, true))) return rc;
  if (o.use_x0) {
    if (pack_x0 && (rc = pack_user(m.h, m.h->p64, m.x, 1, s, true))) return rc;
  } else {
    CK(cudaMemsetAsync(P.plane_start(P.vec(0)), 0, P.plane_elems * sizeof(double), s));
  }
  for (int v : {5, 6}) CK(cudaMemsetAsync(P.plane_start(P.vec(v)), 0, P.plane_elems * sizeof(double), s));
  return PCG_OK;
}

int member_pack(Member &m, const pcg_opts &o, cudaStream_t s) { return member_inputs(m, o, true, s); }

int member_load(Member &m, const pcg_opts &o, bool pack_x0, cudaStream_t s) {
  auto &P = m.h->p64;
  int rc;
  const int max_iter = o.max_iter > 0 ? o.max_iter : std::max(m.h->G.n, 1);
  if ((rc = member_inputs(m, o, pack_x0, s))) return rc;
  SolveState &st = *m.st_host;
  std::memset(&st, 0, sizeof(st));
  st.final_status = -1;
  st.rtol = o.rtol;
  st.max_iter = max_iter;
  st.status = PCG_OK;
  st.done = (m.h->G.n == 0) ? 1 : 0;
  st.retired = st.done;
  CK(cudaMemcpyAsync(P.st, &st, sizeof(SolveState), cudaMemcpyHostToDevice, s));
  m.replacements = 0;
  m.final_status = st.retired ? PCG_OK : -1;
  return PCG_OK;
}

int members_init(LoopPlan &L, cudaStream_t s) {
  int rc;
  for (auto &G : L.groups)
    if ((rc = launch_k(G.ks, 1, G.n_units, kparams(L, G, K1_RESID_INIT, 0, 0), s))) return rc;
  for (auto &G : L.groups)
    if ((rc = launch_k(G.ks, 2, G.n_units, kparams(L, G, K2_INIT, 0, 0), s))) return rc;
  return PCG_OK;
}

int members_close(LoopPlan &L, cudaStream_t s) {
  int rc;
  for (auto &G : L.groups)
    if ((rc = launch(G.ks.fin, G.n_units, G.ks.tx, 0, kparams(L, G, 0, 0, 0), s))) return rc;
  for (auto &G : L.groups)
    if ((rc = launch_k(G.ks, 1, G.n_units, kparams(L, G, K1_RESID_CHECK, 0, 0), s))) return rc;
  return PCG_OK;
}

bool member_decide(Member &m, const pcg_opts &o, bool overrun, cudaStream_t s, int *err) {
  *err = PCG_OK;
  if (m.final_status >= 0) return false;
  SolveState &st = *m.st_host;
  int fs = -1;
  if (st.status != PCG_OK) fs = st.status;
  else if (!st.done && overrun) fs = PCG_ETIMEOUT;
  else if (!st.done) return false;                 // still iterating (chunked advance)
  else if (st.bzero) fs = PCG_OK;
  else {
    const double tr = std::sqrt(st.rr_true) / std::sqrt(st.bb);
    if (tr <= o.rtol) fs = PCG_OK;
    else if (st.iter >= st.max_iter || m.replacements >= o.max_replace) fs = PCG_ENOTCONV;
  }
  cudaError_t e;
  if (fs >= 0) {
    m.final_status = fs;
    st.retired = 1;
    e = cudaMemcpyAsync(&m.h->p64.st->retired, &st.retired, sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); *err = PCG_ECUDA; }
    return false;
  }
  // restart from the true residual (it is in the current r plane)
  m.replacements++;
  st.done = 0;
  e = cudaMemcpyAsync(&m.h->p64.st->done, &st.done, sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); *err = PCG_ECUDA; }
  return true;
}

int member_store(Member &m, cudaStream_t s) { return unpack_user(m.h, m.h->p64, m.x, 0, s, true); }

void member_stats(Member &m) {
  SolveState &st = *m.st_host;
  if (!m.stats) return;
  m.stats->iters = st.iter;
  m.stats->outer_iters = 1 + m.replacements;
  m.stats->status = m.final_status;
  m.stats->replacements = m.replacements;
  m.stats->relres = st.bb > 0 ? std::sqrt(st.rr) / std::sqrt(st.bb) : 0.0;
  m.stats->true_relres = st.bb > 0 ? std::sqrt(st.rr_true) / std::sqrt(st.bb) : 0.0;
}

// Binary64 solve of every member of the plan: Algorithm 1 on the device, the
// true-residual check, and restarts from the true residual where it fails.
int solve_members64(LoopPlan &L, LaunchState *ls_host, std::vector<Member> &M, const pcg_opts &o,
                    cudaStream_t s) {
  int rc;
  int max_iter_all = 0;
  for (auto &m : M) {
    if ((rc = member_load(m, o, true, s))) return rc;
    max_iter_all = std::max(max_iter_all, m.st_host->max_iter);
  }
  int active = 0;
  for (auto &m : M) active += m.final_status < 0 ? 1 : 0;
  while (active > 0) {
    if ((rc = members_arm(L, ls_host, active, max_iter_all + 64, s))) return rc;
    if ((rc = members_init(L, s))) return rc;
    if ((rc = members_loop(L, ls_host, max_iter_all + 64, s))) return rc;
    if ((rc = members_close(L, s))) return rc;
    for (auto &m : M) CK(cudaMemcpyAsync(m.st_host, m.h->p64.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ls_host, L.ls, sizeof(LaunchState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (L.graph_ok) g_launches.fetch_add((uint64_t)std::max(ls_host->launches, 0) * L.body_kernels, std::memory_order_relaxed);
    const bool overrun = (ls_host->stop && ls_host->active > 0) || ls_host->timed_out;
    active = 0;
    for (auto &m : M) {
      int err;
      const bool again = member_decide(m, o, overrun, s, &err);
      if (err) return err;
      if (again) ++active;
      else if (m.final_status < 0) m.final_status = PCG_ETIMEOUT;   // the loop ended without this grid
    }
  }
  for (auto &m : M) if ((rc = member_store(m, s))) return rc;
  CK(cudaStreamSynchronize(s));
  for (auto &m : M) member_stats(m);
  return PCG_OK;
}

// Mixed precision, one refinement step of member m, after its binary64
// residual r = b - A x has been computed and its state read back: either the
// member is finished (returns true with final_status set and the state
// retired on the device), or its binary32 inner solve is prepared -- the
// right-hand side r scaled to unit root-mean-square by a power of two, x32
// and the directions cleared, the inner state armed -- and false is returned.
bool mixed_prepare_inner(Member &m, const pcg_opts &o, int budget, int outer, cudaStream_t s, int *err) {
  *err = PCG_OK;
  auto &P32 = m.h->p32;
  SolveState &st = *m.st_host;
  int fs = -1;
  if (st.status != PCG_OK) fs = st.status;
  else if (st.bzero) {
    if (cudaMemsetAsync(m.h->p64.plane_start(m.h->p64.vec(0)), 0, m.h->p64.plane_elems * sizeof(double), s) != cudaSuccess)
      *err = PCG_ECUDA;
    m.relres64 = 0.0;
    fs = PCG_OK;
  } else {
    m.relres64 = std::sqrt(st.rr) / std::sqrt(st.bb);
    if (!(m.relres64 > o.rtol)) fs = PCG_OK;
    else if (!std::isfinite(m.relres64)) fs = PCG_EBREAKDOWN;
    else if (outer >= o.max_outer || m.inner_iters >= budget) fs = PCG_ENOTCONV;
  }
  SolveState st32{};
  st32.status = PCG_OK;
  st32.final_status = -1;
  if (fs >= 0) {
    m.final_status = fs;
    st.retired = 1; st.done = 1;
    if (cudaMemcpyAsync(&m.h->p64.st->done, &st.done, sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(&m.h->p64.st->retired, &st.retired, sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess)
      *err = PCG_ECUDA;
    st32.done = 1; st32.retired = 1;
  } else {
    const double rms = std::sqrt(st.rr / std::max(m.h->G.n, 1));
    m.scale = std::ldexp(1.0, -std::ilogb(rms > 0 ? rms : 1.0));
    const GridDev<double> *g64 = m.h->p64.gd_dev;
    const GridDev<float> *g32 = P32.gd_dev;
    const Unit *un = m.h->p64.units_dev;
    double sc = m.scale;
    void *args[] = {(void *)&g64, (void *)&g32, (void *)&un, &sc};
    const void *f = (const void *)k_residual_to_f32;
    if (m.h->p64.n_units > 0) {
      g_launches.fetch_add(1, std::memory_order_relaxed);
      if (cudaLaunchKernel(f, dim3(m.h->p64.n_units), dim3(m.h->tx), args, 0, s) != cudaSuccess) *err = PCG_ECUDA;
    }
    // Inner tolerance. Far from the finish: o.inner_rtol (the binary32 solve
    // cannot go much below ~1e-6 relative). Within a decade of the finish
    // (the reduction still needed, rtol / relres, is at least inner_rtol / 10):
    // half the needed reduction, so that binary32 rounding in the correction
    // does not leave the solve just above rtol and cost a whole extra pass.
    const double need = o.rtol / m.relres64;
    st32.rtol = need >= 0.1 * o.inner_rtol ? std::max(0.5 * need, 0.1 * o.inner_rtol) : o.inner_rtol;
    st32.max_iter = std::max(1, budget - m.inner_iters);
  }
  *m.h->st32_host = st32;
  if (cudaMemcpyAsync(P32.st, m.h->st32_host, sizeof(SolveState), cudaMemcpyHostToDevice, s) != cudaSuccess) *err = PCG_ECUDA;
  if (*err) set_error("CUDA call failed in the refinement step");
  return fs >= 0;
}

// Mixed precision: after member m's inner solve finished (its binary32 state
// read back into st32_host and its last x32 update applied), x += e / scale
// in binary64. Returns a pcg_status.
int mixed_apply_correction(Member &m, cudaStream_t s) {
  const SolveState &st32 = *m.h->st32_host;
  m.inner_iters += st32.iter;
  m.inner_solves += 1;
  if (st32.status == PCG_EBREAKDOWN && st32.iter == 0) { m.final_status = PCG_EBREAKDOWN; return PCG_OK; }
  const GridDev<double> *g64 = m.h->p64.gd_dev;
  const GridDev<float> *g32 = m.h->p32.gd_dev;
  const Unit *un = m.h->p64.units_dev;
  double inv = 1.0 / m.scale;
  void *args[] = {(void *)&g64, (void *)&g32, (void *)&un, &inv};
  const void *f = (const void *)k_correct_f64;
  if (m.h->p64.n_units > 0) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    CK(cudaLaunchKernel(f, dim3(m.h->p64.n_units), dim3(m.h->tx), args, 0, s));
  }
  return PCG_OK;
}

// Mixed precision: iterative refinement in binary64 around binary32 PCG
// solves. Each outer step computes the binary64 residual r = b - A x (the
// binary64 stencil kernel), stops if ||r|| / ||b|| <= rtol, otherwise solves
// A e = r in binary32 (r scaled by a power of two, inner tolerance
// inner_rtol) and updates x += e in binary64.
int solve_members_mixed(LoopPlan &L64, LoopPlan &L32, LaunchState *ls_host, std::vector<Member> &M,
                        const pcg_opts &o, cudaStream_t s) {
  int rc;
  for (auto &m : M) {
    if ((rc = member_load(m, o, true, s))) return rc;
    m.inner_iters = 0; m.inner_solves = 0; m.relres64 = 0.0;
  }
  int budget_default = 0;
  for (auto &m : M) budget_default = std::max(budget_default, std::max(m.h->G.n, 1));
  const int budget = o.max_iter > 0 ? o.max_iter : budget_default;
  for (int outer = 0;; ++outer) {
    int remaining = 0;
    for (auto &m : M) remaining += m.final_status < 0 ? 1 : 0;
    if (remaining == 0) break;
    // binary64 residual of every unfinished grid
    if ((rc = members_arm(L64, ls_host, remaining, 1, s))) return rc;
    for (auto &G : L64.groups)
      if ((rc = launch_k(G.ks, 1, G.n_units, kparams(L64, G, K1_RESID_INIT, 0, 0), s))) return rc;
    for (auto &m : M) CK(cudaMemcpyAsync(m.st_host, m.h->p64.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int inner = 0;
    for (auto &m : M) {
      if (m.final_status >= 0) {
        SolveState st32{};
        st32.status = PCG_OK; st32.done = 1; st32.retired = 1;
        st32.final_status = -1;
        *m.h->st32_host = st32;
        CK(cudaMemcpyAsync(m.h->p32.st, m.h->st32_host, sizeof(SolveState), cudaMemcpyHostToDevice, s));
        continue;
      }
      int err;
      if (!mixed_prepare_inner(m, o, budget, outer, s, &err)) ++inner;
      if (err) return err;
    }
    if (inner == 0) continue;
    // binary32 inner solves of all of them together
    if ((rc = members_arm(L32, ls_host, inner, budget + 64, s))) return rc;
    if ((rc = members_init(L32, s))) return rc;
    if ((rc = members_loop(L32, ls_host, budget + 64, s))) return rc;
    for (auto &G : L32.groups)
      if ((rc = launch(G.ks.fin, G.n_units, G.ks.tx, 0, kparams(L32, G, 0, 0, 0), s))) return rc;
    for (auto &m : M) CK(cudaMemcpyAsync(m.h->st32_host, m.h->p32.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ls_host, L32.ls, sizeof(LaunchState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (L32.graph_ok) g_launches.fetch_add((uint64_t)std::max(ls_host->launches, 0) * L32.body_kernels, std::memory_order_relaxed);
    for (auto &m : M) {
      if (m.final_status >= 0 || m.h->st32_host->retired) continue;
      if ((rc = mixed_apply_correction(m, s))) return rc;
    }
  }
  for (auto &m : M) if ((rc = member_store(m, s))) return rc;
  CK(cudaStreamSynchronize(s));
  for (auto &m : M) mixed_stats(m);
  return PCG_OK;
}

void mixed_stats(Member &m) {
  if (!m.stats) return;
  m.stats->iters = m.inner_iters;
  m.stats->outer_iters = m.inner_solves;
  m.stats->status = m.final_status;
  m.stats->replacements = 0;
  m.stats->relres = m.relres64;
  m.stats->true_relres = m.relres64;
}

int apply_status_clear(SolveState *st, cudaStream_t s) {
  CK(cudaMemsetAsync(&st->status, 0, sizeof(int32_t), s));
  return PCG_OK;
}

int apply_status_read(SolveState *st, cudaStream_t s) {
  CK(cudaStreamSynchronize(s));
  int32_t v = PCG_OK;
  CK(cudaMemcpy(&v, &st->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (v != PCG_OK) {
    set_error("a device wait of the apply gave up (" + status_name(v) + "); the output is incomplete");
    return v;
  }
  return PCG_OK;
}

// Single-grid launches used by the server for the steps it runs per request.
int single_launch(pcg_handle *h, bool f32, int which, int kind, cudaStream_t s) {
  LoopPlan &L = f32 ? *h->plan32 : *h->plan64;
  const PlanGroup &G = L.groups[0];
  if (which == 1) return launch_k(G.ks, 1, G.n_units, kparams(L, G, kind, 0, 0), s);
  if (which == 2) return launch_k(G.ks, 2, G.n_units, kparams(L, G, kind, 0, 0), s);
  return launch(G.ks.fin, G.n_units, G.ks.tx, 0, kparams(L, G, 0, 0, 0), s);
}

std::string status_name(int s) {
  switch (s) {
    case PCG_OK: return "ok";
    case PCG_EINVAL: return "invalid argument";
    case PCG_ENOMEM: return "out of memory";
    case PCG_EBUDGET: return "over the HBM budget";
    case PCG_ENOTCONV: return "did not converge";
    case PCG_EBREAKDOWN: return "breakdown";
    case PCG_ETIMEOUT: return "timeout";
    case PCG_ECUDA: return "CUDA error";
    case PCG_ECANCELLED: return "cancelled";
    default: return "unknown status";
  }
}

// Strip width. binary64 kernels are bound by the FP64 pipe: narrow strips
// (more CTAs per SM) whose t phase fills whole warps where the pattern allows
// (64 - 2R columns); on wider grids the wider whole-warp strips (tril(A):
// 124 columns from WIDE_MIN_NX columns; tril(A^2): 92 from WIDE_MIN_NX_A2). binary32 kernels: of the wide strip (124 or 128
// columns) and 64, the one that wastes the fewest columns, ties to the wider
// strip (fewer halo columns per point).
static constexpr int WIDE_MIN_NX = 2048;
// tril(A^2)'s 92-column strip: measured 4.3-4.4 % faster solves at 1442 x 1021 and
// 722 x 511 and 2.5 % faster iterations at 4322 x 3059, equal at 362 x 292
static constexpr int WIDE_MIN_NX_A2 = 700;
static int choose_tx(int nx, int elem_size, int pattern) {
  const int ex = exact_width(elem_size, pattern);
  if (elem_size == 8) {
    const int wide = wide_width(8, pattern);
    if (wide && nx >= (pattern == PCG_PAT_TRIL_A2 ? WIDE_MIN_NX_A2 : WIDE_MIN_NX)) return wide;
    return ex ? ex : 64;
  }
  const int wide = ex ? ex : 128;
  const int ww = (nx + wide - 1) / wide * wide, w64 = (nx + 63) / 64 * 64;
  return (ww - nx <= (w64 - nx) + 16) ? wide : 64;
}

// Strip height, fallback: about 600 units when the grid allows, a multiple
// of 8 rows in min_ty..64.
static int choose_ty(int nx, int ny, int tx, int min_ty) {
  const int ntx = (nx + tx - 1) / tx;
  const int ty = (int)((double)ntx * ny / 600.0) / 8 * 8;
  return std::max(min_ty, std::min(64, ty));
}

// Strip height: the candidate that minimises a makespan model of one
// iteration's two persistent launches over the grid's active units. CTA c of
// a launch with G resident CTAs takes units c, c + G, ... (band-major order,
// as upload_planes builds them); a launch lasts as long as its slowest CTA's
// chain of steps. A unit of h rows costs h + 3 steps in k_stencil and
// h + 2 LD + 2 in k_precond (the pipeline depths) plus UNIT_STEPS for its
// reduction and the refill of the stream; a k_precond step weighs 1.5
// k_stencil steps. Few units (small grids) make every CTA's chain one short
// unit; many units make the count per CTA, and its rounding, decide.
// Measured on 4322 x 3059 (three strip / precision pairs, 7 to 9 heights
// each), 1442 x 1021, 722 x 511 and 182 x 149 (both precisions, 7 heights),
// the model's height was the fastest one every time (up to 2.7x faster than
// a fixed 64 rows for binary32 on small grids), except for the 92-column
// binary64 strips, whose heights are capped (max_unit_rows).
static int model_ty(const HostGrid &G, int tx, const KernelSet &ks, int ld, int max_ty) {
  constexpr double UNIT_STEPS = 10.0;
  static const int cand[] = {4, 8, 16, 24, 32, 40, 48, 56, 64, 72, 80, 96, 112, 128};
  const int ntx = (G.nx + tx - 1) / tx;
  std::vector<uint8_t> row_wet((size_t)ntx * G.ny, 0);     // [strip][row]: any wet cell
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i)
      if (G.idx[(size_t)j * G.nx + i] >= 0) row_wet[(size_t)(i / tx) * G.ny + j] = 1;
  const int g1 = std::max(ks.ctas1, 1), g2 = std::max(ks.ctas2, 1);
  std::vector<double> c1(g1), c2(g2);
  int best_ty = max_ty;
  double best = 1e300;
  for (int ty : cand) {
    if (ty > max_ty) break;                            // (max_unit_rows)
    if ((G.ny + ty - 1) / ty > INT16_MAX) continue;    // strip coordinates are 16-bit
    std::fill(c1.begin(), c1.end(), 0.0);
    std::fill(c2.begin(), c2.end(), 0.0);
    long k = 0;
    const int nty = (G.ny + ty - 1) / ty;
    for (int sy = 0; sy < nty; ++sy) {
      const int j0 = sy * ty, j1 = std::min(G.ny, j0 + ty);
      for (int sx = 0; sx < ntx; ++sx) {
        bool any = false;
        for (int j = j0; j < j1 && !any; ++j) any = row_wet[(size_t)sx * G.ny + j] != 0;
        if (!any) continue;
        c1[k % g1] += (j1 - j0) + 3 + UNIT_STEPS;
        c2[k % g2] += (j1 - j0) + 2 * ld + 2 + UNIT_STEPS;
        ++k;
      }
    }
    const double cost = *std::max_element(c1.begin(), c1.end()) + 1.5 * *std::max_element(c2.begin(), c2.end());
    if (cost < best) { best = cost; best_ty = ty; }
    if (ty >= G.ny) break;                             // taller strips give the same units
  }
  return best_ty;
}

// ------------------------------------------------------------ strip autotuner
// Tuned strip shapes, per grid shape, pattern and precision, for the process:
// a tuned shape is used by every later handle of that shape.
struct TuneKey {
  int nx, ny, pattern, q, prec, objective;
  bool operator<(const TuneKey &o) const {
    return std::tie(nx, ny, pattern, q, prec, objective) < std::tie(o.nx, o.ny, o.pattern, o.q, o.prec, o.objective);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tuned;

static bool tuned_shape(int nx, int ny, int pattern, int q, int prec, int objective, int *tx, int *ty) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(TuneKey{nx, ny, pattern, q, prec, objective});
  if (it == g_tuned.end()) return false;
  *tx = it->second.first;
  *ty = it->second.second;
  return true;
}

// Rebuild the device planes of one precision of h with strips tx x ty (the
// handle's last solution in those planes is lost).
static int retile(pcg_handle *h, int prec, int tx, int ty, cudaStream_t s) {
  int rc;
  if (prec == PCG_MIXED) {
    if (h->plan32 && h->tx32 == tx && h->ty32 == ty) return PCG_OK;
    h->version++;                                   // cached batch plans of the old planes no longer match
    if (h->plan32) h->bytes -= h->p32.bytes;
    h->plan32.reset();
    h->p32.release();
    h->p32 = DevPlanes<float>{};
    h->tx32 = tx;
    h->ty32 = ty;
    return ensure_f32(h, s);
  }
  if (h->tx == tx && h->ty == ty) return PCG_OK;
  CK(cudaStreamSynchronize(s));
  h->version++;
  h->bytes -= h->p64.bytes;
  if (h->plan32) { h->plan32->solve.reset(); h->plan32->solve_tried = false; }   // it spans the binary64 planes too
  h->plan64.reset();
  h->p64.release();
  h->p64 = DevPlanes<double>{};
  h->tx = tx;
  h->ty = ty;
  if ((rc = upload_planes(h, h->p64, s))) return rc;
  h->bytes += h->p64.bytes;
  return plan_single(h);
}

}  // namespace pcg

using namespace pcg;

extern "C" {

const char *pcg_status_string(int status) {
  static thread_local std::string s;
  s = status_name(status);
  return s.c_str();
}

const char *pcg_last_error_message(void) { return g_err.c_str(); }

static int factor_host(const pcg_grid *grid, const ainv_opts *opts, HostGrid &G, HostFactor &F) {
  if (!opts) { set_error("opts is NULL"); return PCG_EINVAL; }
  const int pattern = opts->pattern;
  if (pattern == PCG_PAT_FULL) { set_error("the dense pattern is available in the CPU oracle only"); return PCG_EINVAL; }
  if (pattern < 0 || pattern > PCG_PAT_DIAG) { set_error("unknown pattern"); return PCG_EINVAL; }
  if (pattern == PCG_PAT_BAND_T && (opts->band_q < 1 || opts->band_q > 8)) { set_error("band_q must be 1..8"); return PCG_EINVAL; }
  std::string err;
  int rc = host_grid_build(grid, pattern, G, err);
  if (rc) { set_error(err); return rc; }
  if (pattern == PCG_PAT_BAND_T && grid->nx <= opts->band_q) { set_error("band_q must be < nx"); return PCG_EINVAL; }
  rc = host_ainv(G, pattern, opts->drop_tol, opts->band_q, F, err);
  if (rc) { set_error(err); return rc; }
  return PCG_OK;
}

static void export_factor(const HostGrid &G, const HostFactor &F, double *D, int32_t *rows, double *vals) {
  const int n = G.n, nx = G.nx;
  for (int k = 0; k < n; ++k) {
    if (D) D[k] = F.d[k];
    if (!rows || !vals) continue;
    for (int e = 0; e < 8; ++e) { rows[(size_t)k * 8 + e] = -1; vals[(size_t)k * 8 + e] = 0.0; }
    int e = 0;
    const int i = G.pi[k], j = G.pj[k];
    for (int s = 0; s < F.slots.n; ++s) {
      const double v = F.z[(size_t)s * n + k];
      if (v == 0.0) continue;
      const int ii = ((i + F.slots.dx[s]) % nx + nx) % nx, jj = j + F.slots.dy[s];
      rows[(size_t)k * 8 + e] = G.idx[(size_t)jj * nx + ii];
      vals[(size_t)k * 8 + e] = v;
      ++e;
    }
    for (int w = 0; w < F.slots.n_wrap; ++w) {
      if (i != nx - 1 - F.slots.wcol[w]) continue;
      const double v = F.zwrap[(size_t)j * F.slots.n_wrap + w];
      if (v == 0.0) continue;
      const int ii = ((F.slots.wdx[w] - 1 - F.slots.wcol[w]) % nx + nx) % nx;
      rows[(size_t)k * 8 + e] = G.idx[(size_t)j * nx + ii];
      vals[(size_t)k * 8 + e] = v;
      ++e;
    }
  }
}

int ainv_factor_host(const pcg_grid *grid, const ainv_opts *opts, int32_t *n_wet_out, double *D, int32_t *rows,
                     double *vals) {
  try {
    HostGrid G;
    HostFactor F;
    int rc = factor_host(grid, opts, G, F);
    if (rc) return rc;
    if (n_wet_out) *n_wet_out = G.n;
    export_factor(G, F, D, rows, vals);
    return PCG_OK;
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return PCG_ENOMEM;
  } catch (...) {
    set_error("unexpected host failure");
    return PCG_EINVAL;
  }
}

}  // extern "C"

// The device side of a handle whose host grid, factor and strips are set:
// binary64 planes, launch state, pinned mirrors, the staging buffer and its
// copy stream and events.
static int handle_device_init(pcg_handle *h, cudaStream_t s) {
  const size_t cells = (size_t)h->G.nx * h->G.ny;
  int rc = upload_planes(h, h->p64, s);
  if (rc) { h->p64.release(); return rc; }
  if (cudaMalloc(&h->ls, sizeof(LaunchState)) != cudaSuccess) { cudaGetLastError(); h->p64.release(); set_error("device allocation failed"); return PCG_ENOMEM; }
  if (cudaMallocHost(&h->ls_host, sizeof(LaunchState)) != cudaSuccess ||
      cudaMallocHost(&h->st_host, sizeof(SolveState)) != cudaSuccess) {
    cudaGetLastError(); set_error("pinned allocation failed"); return PCG_ENOMEM;
  }
  if (cudaMalloc(&h->stage, sizeof(double) * cells) != cudaSuccess) {
    cudaGetLastError(); set_error("device allocation failed"); return PCG_ENOMEM;
  }
  if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_unpacked, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_stage, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError(); set_error("stream or event creation failed"); return PCG_ECUDA;
  }
  h->bytes = h->p64.bytes + sizeof(LaunchState) + sizeof(double) * cells;
  CK(cudaStreamSynchronize(s));
  return PCG_OK;
}

extern "C" {

int ainv_setup(const pcg_grid *grid, const ainv_opts *opts, void *cuda_stream, pcg_handle **out) {
  if (!out) { set_error("out is NULL"); return PCG_EINVAL; }
  *out = nullptr;
  try {
    auto h = std::make_unique<pcg_handle>();
    handle_init_serial(h.get());
    int rc = factor_host(grid, opts, h->G, h->F);
    if (rc) return rc;
    if (grid->nx < GHOST) {   // the loop kernels store each column with at most one periodic copy per side
      set_error("device grids must be at least 4 columns wide");
      return PCG_EINVAL;
    }
    h->pattern = opts->pattern;
    h->band_q = opts->band_q;
    h->tau = opts->drop_tol;
    if (opts->tile_x != 0 && !valid_width(opts->tile_x, opts->pattern)) {
      set_error("tile_x must be 64, 128 or a whole-warp width of the pattern (tril(A^2): 60 or 92 binary64, 124 "
                "binary32; tril(A): 62 or 124 binary64, 124 binary32)");
      return PCG_EINVAL;
    }
    if (opts->tile_y != 0 && (opts->tile_y < 4 || opts->tile_y > 256)) { set_error("tile_y must be 4..256"); return PCG_EINVAL; }
    // an explicit width applies to the precisions that have kernels for it; the
    // other precision keeps its default width
    const bool x64 = opts->tile_x && pick<double>(opts->tile_x, opts->pattern, opts->band_q).ok;
    const bool x32 = opts->tile_x && pick<float>(opts->tile_x, opts->pattern, opts->band_q).ok;
    h->tx = x64 ? opts->tile_x : choose_tx(grid->nx, 8, opts->pattern);
    h->tx32 = x32 ? opts->tile_x : choose_tx(grid->nx, 4, opts->pattern);
    h->ty = opts->tile_y ? opts->tile_y : choose_ty(grid->nx, grid->ny, h->tx, 4);
    h->ty32 = opts->tile_y ? opts->tile_y : choose_ty(grid->nx, grid->ny, h->tx32, 64);
    if (!opts->tile_y) {                        // heights from the makespan model where the kernels exist
      const int ld = opts->pattern == PCG_PAT_TRIL_A2 ? 2 : (opts->pattern == PCG_PAT_TRIL_A ? 1 : 0);
      KernelSet k64 = pick<double>(h->tx, opts->pattern, opts->band_q);
      if (k64.ok && prepare_set(k64) == PCG_OK) h->ty = model_ty(h->G, h->tx, k64, ld, max_unit_rows(8, h->tx, opts->pattern));
      KernelSet k32 = pick<float>(h->tx32, opts->pattern, opts->band_q);
      if (k32.ok && prepare_set(k32) == PCG_OK) h->ty32 = model_ty(h->G, h->tx32, k32, ld, max_unit_rows(4, h->tx32, opts->pattern));
    }
    if (!opts->tile_x && !opts->tile_y) {       // shapes tuned earlier in this process win (latency objective)
      tuned_shape(grid->nx, grid->ny, opts->pattern, opts->band_q, PCG_FP64, 0, &h->tx, &h->ty);
      tuned_shape(grid->nx, grid->ny, opts->pattern, opts->band_q, PCG_MIXED, 0, &h->tx32, &h->ty32);
    }
    if ((rc = handle_device_init(h.get(), (cudaStream_t)cuda_stream))) return rc;
    *out = h.release();
    return PCG_OK;
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return PCG_ENOMEM;
  }
}

int pcg_clone(const pcg_handle *src, void *cuda_stream, pcg_handle **out) {
  if (!out) { set_error("out is NULL"); return PCG_EINVAL; }
  *out = nullptr;
  if (!src) { set_error("NULL handle"); return PCG_EINVAL; }
  try {
    auto h = std::make_unique<pcg_handle>();
    handle_init_serial(h.get());
    h->G = src->G;
    h->F = src->F;
    h->pattern = src->pattern;
    h->band_q = src->band_q;
    h->tau = src->tau;
    h->tx = src->tx; h->ty = src->ty;
    h->tx32 = src->tx32; h->ty32 = src->ty32;
    int rc = handle_device_init(h.get(), (cudaStream_t)cuda_stream);
    if (rc) return rc;
    *out = h.release();
    return PCG_OK;
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return PCG_ENOMEM;
  }
}

int pcg_spmv(pcg_handle *h, const double *v, double *q, void *cuda_stream) {
  if (!h || !v || !q) { set_error("NULL argument"); return PCG_EINVAL; }
  handle_finish_pending(h);   // one piece of work in flight per handle
  cudaStream_t s = (cudaStream_t)cuda_stream;
  auto &P = h->p64;
  int rc;
  if ((rc = apply_status_clear(P.st, s))) return rc;
  if ((rc = pack_user(h, h->p64, v, 3, s))) return rc;
  KParams p{};
  p.grids = P.gd_dev; p.units = P.units_dev; p.ls = h->ls; p.kind = K1_SPMV; p.dbg_skip_unit = -1;
  p.timeout_ns = default_timeout_ns();
  if ((rc = launch_k(P.ks, 1, P.n_units, p, s))) return rc;
  if ((rc = unpack_user(h, h->p64, q, 2, s))) return rc;
  return apply_status_read(P.st, s);
}

int pcg_precond_apply(pcg_handle *h, const double *r, double *sv, void *cuda_stream) {
  if (!h || !r || !sv) { set_error("NULL argument"); return PCG_EINVAL; }
  handle_finish_pending(h);   // one piece of work in flight per handle
  cudaStream_t s = (cudaStream_t)cuda_stream;
  auto &P = h->p64;
  int rc;
  if ((rc = apply_status_clear(P.st, s))) return rc;
  if ((rc = pack_user(h, h->p64, r, 2, s))) return rc;
  KParams p{};
  p.grids = P.gd_dev; p.units = P.units_dev; p.ls = h->ls; p.kind = K2_APPLY; p.dbg_skip_unit = -1;
  p.timeout_ns = default_timeout_ns();
  if ((rc = launch_k(P.ks, 2, P.n_units, p, s))) return rc;
  if ((rc = unpack_user(h, h->p64, sv, 1, s))) return rc;
  return apply_status_read(P.st, s);
}

int pcg_apply_f32(pcg_handle *h, int32_t op, const double *v, double *out, void *cuda_stream) {
  if (!h || !v || !out || (op != 0 && op != 1)) { set_error("invalid arguments"); return PCG_EINVAL; }
  handle_finish_pending(h);   // one piece of work in flight per handle
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int rc;
  if ((rc = ensure_f32(h, s))) return rc;
  auto &P = h->p32;
  // op 0: v into d[0], q = A v; op 1: v into r[0], s = M^-1 v
  if ((rc = apply_status_clear(P.st, s))) return rc;
  if ((rc = pack_user(h, P, v, op == 0 ? 3 : 2, s))) return rc;
  KParams p{};
  p.grids = P.gd_dev; p.units = P.units_dev; p.ls = h->ls; p.kind = op == 0 ? (int)K1_SPMV : (int)K2_APPLY;
  p.dbg_skip_unit = -1;
  p.timeout_ns = default_timeout_ns();
  if ((rc = launch_k(P.ks, op == 0 ? 1 : 2, P.n_units, p, s))) return rc;
  if ((rc = unpack_user(h, P, out, op == 0 ? 2 : 1, s))) return rc;
  return apply_status_read(P.st, s);
}

int pcg_profile_kernels(pcg_handle *h, const double *b, int32_t iters, int32_t prec, double *ms_stencil,
                        double *ms_precond, void *cuda_stream) {
  if (!h || !b || iters <= 0 || (prec != PCG_FP64 && prec != PCG_MIXED)) { set_error("invalid arguments"); return PCG_EINVAL; }
  handle_finish_pending(h);   // one piece of work in flight per handle
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int rc;
  if ((rc = plan_single(h))) return rc;
  if (prec == PCG_MIXED && (rc = ensure_f32(h, s))) return rc;
  pcg_opts o;
  fill_opts(nullptr, o);
  o.rtol = 0.0;                       // iterate the requested number of times
  o.max_iter = iters + 1;
  o.use_x0 = 0;
  Member m;
  m.h = h; m.b = b; m.x = nullptr; m.st_host = h->st_host;
  if ((rc = member_load(m, o, false, s))) return rc;   // packs b, zeroes x
  LoopPlan *L = h->plan64.get();
  SolveState *st_dev = h->p64.st;
  SolveState *st_host = h->st_host;
  if (prec == PCG_MIXED) {
    // the binary32 system with right-hand side b (scale 1)
    const GridDev<double> *g64 = h->p64.gd_dev;
    const GridDev<float> *g32 = h->p32.gd_dev;
    const Unit *un = h->p64.units_dev;
    // b64 -> r64 plane 0 by a residual pass with x = 0, then to binary32
    if ((rc = members_arm(*L, h->ls_host, 1, 1, s))) return rc;
    const PlanGroup &G64 = L->groups[0];
    if ((rc = launch_k(G64.ks, 1, G64.n_units, kparams(*L, G64, K1_RESID_INIT, 0, 0), s))) return rc;
    double sc = 1.0;
    void *args[] = {(void *)&g64, (void *)&g32, (void *)&un, &sc};
    const void *f = (const void *)k_residual_to_f32;
    if (h->p64.n_units > 0) CK(cudaLaunchKernel(f, dim3(h->p64.n_units), dim3(h->tx), args, 0, s));
    auto &P32 = h->p32;
    CK(cudaMemsetAsync(P32.plane_start(P32.vec(0)), 0, P32.plane_elems * sizeof(float), s));
    for (int v : {5, 6}) CK(cudaMemsetAsync(P32.plane_start(P32.vec(v)), 0, P32.plane_elems * sizeof(float), s));
    SolveState st32{};
    st32.status = PCG_OK; st32.rtol = 0.0; st32.max_iter = iters + 1;
    *h->st32_host = st32;
    CK(cudaMemcpyAsync(P32.st, h->st32_host, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    L = h->plan32.get();
    st_dev = P32.st;
    st_host = h->st32_host;
  }
  if ((rc = members_arm(*L, h->ls_host, 1, iters + 8, s))) return rc;
  if ((rc = members_init(*L, s))) return rc;
  const PlanGroup &G = L->groups[0];
  std::vector<cudaEvent_t> ev(4 * iters);
  for (auto &e : ev) CK(cudaEventCreate(&e));
  for (int it = 0; it < iters; ++it) {
    CK(cudaEventRecord(ev[4 * it], s));
    if ((rc = launch_k(G.ks, 1, G.n_units, kparams(*L, G, K1_ITER, 0, 0), s))) return rc;
    CK(cudaEventRecord(ev[4 * it + 1], s));
    CK(cudaEventRecord(ev[4 * it + 2], s));
    if ((rc = launch_k(G.ks, 2, G.n_units, kparams(*L, G, K2_ITER, 0, 0), s))) return rc;
    CK(cudaEventRecord(ev[4 * it + 3], s));
  }
  CK(cudaStreamSynchronize(s));
  double t1 = 0, t2 = 0;
  for (int it = 0; it < iters; ++it) {
    float a = 0, c = 0;
    CK(cudaEventElapsedTime(&a, ev[4 * it], ev[4 * it + 1]));
    CK(cudaEventElapsedTime(&c, ev[4 * it + 2], ev[4 * it + 3]));
    t1 += a; t2 += c;
  }
  for (auto &e : ev) cudaEventDestroy(e);
  CK(cudaMemcpyAsync(st_host, st_dev, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st_host->done && st_host->iter < iters) {
    set_error("the iteration stopped early (converged or broke down) while profiling");
    return PCG_EINVAL;
  }
  if (ms_stencil) *ms_stencil = t1 / iters;
  if (ms_precond) *ms_precond = t2 / iters;
  return PCG_OK;
}

uint64_t pcg_kernel_launches(void) { return g_launches.load(); }

int pcg_ainv_export(const pcg_handle *h, int32_t *n_wet_out, double *D, int32_t *rows, double *vals) {
  if (!h) { set_error("NULL handle"); return PCG_EINVAL; }
  if (n_wet_out) *n_wet_out = h->G.n;
  export_factor(h->G, h->F, D, rows, vals);
  return PCG_OK;
}

size_t pcg_resident_bytes(const pcg_handle *h) { return h ? h->bytes : 0; }

int32_t pcg_n_wet(const pcg_handle *h) { return h ? h->G.n : 0; }

int pcg_autotune(pcg_handle *h, int32_t prec, int32_t objective, int32_t *tile_x, int32_t *tile_y,
                 void *cuda_stream) {
  if (!h || (prec != PCG_FP64 && prec != PCG_MIXED) || (objective != 0 && objective != 1)) {
    set_error("invalid arguments");
    return PCG_EINVAL;
  }
  handle_finish_pending(h);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int rc, tx = 0, ty = 0;
  const int nx = h->G.nx, ny = h->G.ny;
  if (!tuned_shape(nx, ny, h->pattern, h->band_q, prec, objective, &tx, &ty)) {
    // right-hand side: ones (land is zeroed by the packing), in the staging plane
    {
      std::vector<double> ones((size_t)nx * ny, 1.0);
      CK(cudaMemcpyAsync(h->stage, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));
    }
    double best = 1e300;
    int last_ty = -1;
    const int ex = exact_width(prec == PCG_MIXED ? 4 : 8, h->pattern);
    const int wide = prec == PCG_MIXED ? 0 : wide_width(8, h->pattern);
    for (int cx : {64, 128, ex, wide}) {
      if (cx == 0) continue;
      last_ty = -1;
      for (int cy : {8, 16, 32, 64}) {
        const int eff = std::min(cy, (ny + 7) / 8 * 8);     // a taller strip than the grid is the same shape
        if (eff == last_ty) continue;
        last_ty = eff;
        if ((rc = retile(h, prec, cx, cy, s))) return rc;
        double m1 = 0, m2 = 0;
        if ((rc = pcg_profile_kernels(h, h->stage, 3, prec, &m1, &m2, s))) return rc;
        if ((rc = pcg_profile_kernels(h, h->stage, 10, prec, &m1, &m2, s))) return rc;
        double cost = m1 + m2;
        if (objective == 1) {
          // share of the GPU: a launch over n units holds min(n, resident) of
          // the resident CTAs for its duration
          const KernelSet &ks = prec == PCG_MIXED ? h->p32.ks : h->p64.ks;
          const int nu = prec == PCG_MIXED ? h->p32.n_units : h->p64.n_units;
          cost = m1 * std::min(nu, ks.ctas1) / (double)ks.ctas1 + m2 * std::min(nu, ks.ctas2) / (double)ks.ctas2;
        }
        if (cost < best) { best = cost; tx = cx; ty = cy; }
      }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[TuneKey{nx, ny, h->pattern, h->band_q, prec, objective}] = {tx, ty};
  }
  if ((rc = retile(h, prec, tx, ty, s))) return rc;
  CK(cudaStreamSynchronize(s));
  if (tile_x) *tile_x = tx;
  if (tile_y) *tile_y = ty;
  return PCG_OK;
}

int pcg_tiles(pcg_handle *h, int32_t prec, int32_t *tile_x, int32_t *tile_y) {
  if (!h || !tile_x || !tile_y || (prec != PCG_FP64 && prec != PCG_MIXED)) { set_error("invalid arguments"); return PCG_EINVAL; }
  *tile_x = prec == PCG_MIXED ? h->tx32 : h->tx;
  *tile_y = prec == PCG_MIXED ? h->ty32 : h->ty;
  return PCG_OK;
}

void pcg_free(pcg_handle *h) {
  if (!h) return;
  handle_finish_pending(h);
  h->plan64.reset();
  h->plan32.reset();
  h->p64.release();
  h->p32.release();
  cudaFreeHost(h->st32_host);
  cudaFree(h->ls);
  if (h->ev_stage) cudaEventSynchronize(h->ev_stage);
  cudaFree(h->stage);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  for (cudaEvent_t e : {h->ev_in, h->ev_unpacked, h->ev_stage})
    if (e) cudaEventDestroy(e);
  cudaFreeHost(h->ls_host);
  cudaFreeHost(h->st_host);
  delete h;
}

// Test hook: run one preconditioner launch in which the first row copy of
// unit `unit` is never issued, with every device wait bounded by timeout_ms.
// The wait must give up, flag PCG_ETIMEOUT in the grid's state and return;
// the function reports the status the device recorded.
int pcg_debug_wait_timeout(pcg_handle *h, int32_t unit, double timeout_ms, void *cuda_stream) {
  if (!h || unit < 0 || unit >= h->p64.n_units) { set_error("invalid arguments"); return PCG_EINVAL; }
  handle_finish_pending(h);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  auto &P = h->p64;
  SolveState st{};
  st.status = PCG_OK; st.rtol = 1e-10; st.max_iter = 1; st.bb = 1.0;
  CK(cudaMemcpyAsync(P.st, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  LaunchState ls{};
  ls.active = 1;
  CK(cudaMemcpyAsync(h->ls, &ls, sizeof(ls), cudaMemcpyHostToDevice, s));
  KParams p{};
  p.grids = P.gd_dev; p.units = P.units_dev; p.ls = h->ls; p.kind = K2_INIT;
  p.dbg_skip_unit = unit;
  p.timeout_ns = (uint64_t)(timeout_ms * 1e6);
  int rc = launch_k(P.ks, 2, P.n_units, p, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->st_host, P.st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return h->st_host->status;
}

}  // extern "C"
