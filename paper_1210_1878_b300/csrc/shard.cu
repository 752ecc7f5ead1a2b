// Row-band sharding of one grid: the layout in which a single large grid is
// split over several GPUs, run here as bands of one GPU.
//
// The grid's rows are cut into contiguous bands of about equal wet count. A
// band keeps planes for its own rows plus `halo` rows of each neighbour
// (halo = max(1, LD): the stencil reads one row across, the preconditioner's
// Z^T pulls from LD rows below and Z pushes to LD rows above). Its static
// planes (A, Z, D^-1 and the periodic side table) are those rows of the whole
// grid's, so the factor is built once, on the host, for the whole grid. Every
// kernel of the iteration runs over the bands' own rows; the rows a band reads
// beyond them are refreshed by an exchange step after the kernel that
// produced them:
//
//   after the stencil kernel        d (both ping-pong planes), depth 1; q, depth LD
//   after the preconditioner kernel s, depth 1; r (both planes), depth LD
//   after the initial residual      r, depth LD
//   before a residual b - A x       x, depth 1
//
// Across GPUs the exchange is a send / receive of the same row blocks between
// neighbouring ranks and the reductions are two allreduces per iteration (the
// partial sums of (d, q), and of (s, r) and (r, r)). On one GPU the bands'
// units share one launch and one reduction state, so the last unit of any band
// to arrive adds every band's partials in unit order, and the exchange is a
// device-to-device copy of the row blocks (one kernel per exchange point).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "solve_graph.cuh"

namespace pcg {

// One row block copied between two band planes.
struct HaloCopy {
  const double *src;
  double *dst;
  int64_t n;     // elements
};

// Every copy of one exchange point: block c copies list[c].
static __global__ void __launch_bounds__(256) k_halo_exchange(const HaloCopy *list) {
  const HaloCopy c = list[blockIdx.x];
  for (int64_t e = threadIdx.x; e < c.n; e += blockDim.x) c.dst[e] = c.src[e];
}

// Halo depth of a pattern: the stencil reads one row across a band edge; the
// preconditioner reads LD rows below and LD rows above.
static int halo_depth(int pattern) {
  const int ld = pattern == PCG_PAT_TRIL_A2 ? 2 : (pattern == PCG_PAT_TRIL_A ? 1 : 0);
  return std::max(1, ld);
}
static int pattern_ld(int pattern) { return pattern == PCG_PAT_TRIL_A2 ? 2 : (pattern == PCG_PAT_TRIL_A ? 1 : 0); }

// Bands of contiguous rows with about n_wet / nbands wet points each, every
// band at least `halo` rows (its boundary rows fill a neighbour's halo).
static int band_rows(int nx, int ny, const uint8_t *wet, int pattern, int nbands, std::vector<int> &row0, int &halo,
                     std::string &err) {
  halo = halo_depth(pattern);
  if (nbands < 1) { err = "nbands must be at least 1"; return PCG_EINVAL; }
  if ((long)nbands * halo > ny) { err = "too many bands: each needs at least " + std::to_string(halo) + " rows"; return PCG_EINVAL; }
  std::vector<long> cum(ny + 1, 0);
  for (int j = 0; j < ny; ++j) {
    long w = 0;
    for (int i = 0; i < nx; ++i) w += wet[(size_t)j * nx + i] ? 1 : 0;
    cum[j + 1] = cum[j] + w;
  }
  const long n = cum[ny];
  row0.assign(nbands + 1, 0);
  row0[nbands] = ny;
  for (int b = 1; b < nbands; ++b) {
    const long target = (n * b + nbands / 2) / nbands;
    int r = (int)(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
    r = std::max(r, row0[b - 1] + halo);
    r = std::min(r, ny - (nbands - b) * halo);
    row0[b] = r;
  }
  return PCG_OK;
}

// Rows [a, c) of the whole grid as a grid of their own (local row 0 = row a),
// with the whole grid's factor restricted to them.
static void slice(const HostGrid &G, const HostFactor &F, int a, int c, HostGrid &g, HostFactor &f) {
  const int nx = G.nx, ny = c - a;
  g.nx = nx; g.ny = ny;
  g.idx.assign((size_t)nx * ny, -1);
  g.ce.assign(G.ce.begin() + (size_t)a * nx, G.ce.begin() + (size_t)c * nx);
  g.cn.assign(G.cn.begin() + (size_t)a * nx, G.cn.begin() + (size_t)c * nx);
  g.pi.clear(); g.pj.clear(); g.diag.clear();
  std::vector<int> glob;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const int k = G.idx[(size_t)(j + a) * nx + i];
      if (k < 0) continue;
      g.idx[(size_t)j * nx + i] = (int)glob.size();
      g.pi.push_back(i); g.pj.push_back(j);
      g.diag.push_back(G.diag[k]);
      glob.push_back(k);
    }
  g.n = (int)glob.size();
  f.n = g.n;
  f.slots = F.slots;
  f.d.resize(g.n);
  f.z.assign((size_t)F.slots.n * g.n, 0.0);
  for (int l = 0; l < g.n; ++l) {
    f.d[l] = F.d[glob[l]];
    for (int sidx = 0; sidx < F.slots.n; ++sidx) f.z[(size_t)sidx * g.n + l] = F.z[(size_t)sidx * F.n + glob[l]];
  }
  const int nw = F.slots.n_wrap;
  f.zwrap.assign(F.zwrap.begin() + (size_t)a * nw, F.zwrap.begin() + (size_t)c * nw);
}

}  // namespace pcg

using namespace pcg;

struct pcg_shard {
  pcg_handle *h = nullptr;               // the whole grid
  int nb = 0, halo = 0, ld = 0;
  std::vector<int> row0;                 // [nb + 1] band boundaries (rows)
  std::vector<std::unique_ptr<pcg_handle>> bands;
  SolveState *st = nullptr;              // the one reduction state of all bands
  SolveState *st_host = nullptr;
  double *partial = nullptr;             // [units of all bands][2]
  LaunchState *ls = nullptr, *ls_host = nullptr;
  int n_units = 0;
  LoopPlan plan;                         // one group: every band's units
  HaloCopy *ex[4] = {};                  // exchange points: 0 x; 1 r; 2 d and q; 3 s and r
  int nex[4] = {};
  std::unique_ptr<SolveGraph> graph;
  int graph_kernels_outer = 0, graph_kernels_inner = 0;

  ~pcg_shard() {
    graph.reset();
    cudaFree(st); cudaFree(partial); cudaFree(ls);
    cudaFreeHost(st_host); cudaFreeHost(ls_host);
    for (HaloCopy *p : ex) cudaFree(p);
    for (auto &b : bands) b->p64.release();
  }
};

namespace {

int build_shard_graph(pcg_shard &S) {
  auto G = std::make_unique<SolveGraph>();
  std::vector<SolveState *> sts{S.st};
  std::vector<int32_t> nw{S.h->G.n};
  CK(cudaMalloc(&G->st64, sizeof(SolveState *)));
  CK(cudaMemcpy(G->st64, sts.data(), sizeof(SolveState *), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&G->n_wet, sizeof(int32_t)));
  CK(cudaMemcpy(G->n_wet, nw.data(), sizeof(int32_t), cudaMemcpyHostToDevice));
  G->n = 1;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle c_out = 0, c_in = 0;
  Builder top(g);
  top.err = cudaGraphConditionalHandleCreate(&c_out, g, 1, cudaGraphCondAssignDefault);
  cudaGraph_t body = top.while_node(c_out);
  Builder P(body ? body : g);
  P.err = top.err;
  if (P.err == cudaSuccess) P.err = cudaGraphConditionalHandleCreate(&c_in, body, 0, 0);
  SolveState **stp = G->st64;
  int n = 1;
  LaunchState *ls = S.ls;
  uint64_t bns = loop_budget_ns();
  auto exchange = [&](Builder &B, int which) {
    if (S.nex[which] == 0) return;
    const HaloCopy *list = S.ex[which];
    void *args[] = {(void *)&list};
    B.kernel((const void *)k_halo_exchange, dim3(S.nex[which]), dim3(256), 0, args);
  };
  {
    void *args[] = {&stp, &n, &ls, &c_in, &bns};
    P.kernel((const void *)k_ctl_arm, dim3(1), dim3(CTL_THREADS), 0, args);
  }
  exchange(P, 0);                                      // x rows for r = b - A x
  add_groups(P, S.plan, 1, K1_RESID_INIT, 0, false);
  exchange(P, 1);                                      // r rows for the preconditioner
  add_groups(P, S.plan, 2, K2_INIT, 0, false);
  exchange(P, 3);                                      // s and r rows
  cudaGraph_t ib = P.while_node(c_in);
  Builder I(ib ? ib : g);
  I.err = P.err;
  add_groups(I, S.plan, 1, K1_ITER, 1, false);
  exchange(I, 2);                                      // d and q rows
  add_groups(I, S.plan, 2, K2_ITER, 1, true);
  exchange(I, 3);                                      // s and r rows
  P.err = I.err;
  add_finalize(P, S.plan);
  exchange(P, 0);                                      // x rows for the true residual
  add_groups(P, S.plan, 1, K1_RESID_CHECK, 0, false);
  {
    void *args[] = {&stp, &n, &ls, &c_out};
    P.kernel((const void *)k_ctl_decide64, dim3(1), dim3(CTL_THREADS), 0, args);
  }
  if (P.err != cudaSuccess || I.err != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    set_error("sharded solve graph construction failed");
    return PCG_ECUDA;
  }
  const cudaError_t e = cudaGraphInstantiate(&G->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { cudaGetLastError(); G->exec = nullptr; set_error("sharded solve graph instantiation failed"); return PCG_ECUDA; }
  G->outer_kernels = P.kernels;
  G->inner_kernels = I.kernels;
  S.graph = std::move(G);
  return PCG_OK;
}

}  // namespace

extern "C" {

int pcg_band_plan(int32_t nx, int32_t ny, const uint8_t *wet, int32_t pattern, int32_t nbands, int32_t *row0,
                  int32_t *halo) {
  if (!wet || !row0 || !halo || nx < 1 || ny < 1) { set_error("invalid arguments"); return PCG_EINVAL; }
  std::vector<int> r;
  int hd = 0;
  std::string err;
  const int rc = band_rows(nx, ny, wet, pattern, nbands, r, hd, err);
  if (rc) { set_error(err); return rc; }
  for (int b = 0; b <= nbands; ++b) row0[b] = r[b];
  *halo = hd;
  return PCG_OK;
}

int pcg_shard_create(pcg_handle *h, int32_t nbands, void *cuda_stream, pcg_shard **out) {
  if (!h || !out) { set_error("NULL argument"); return PCG_EINVAL; }
  *out = nullptr;
  if (nbands < 2) { set_error("a sharded solve needs at least 2 bands"); return PCG_EINVAL; }
  handle_finish_pending(h);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  try {
    auto S = std::make_unique<pcg_shard>();
    S->h = h;
    S->nb = nbands;
    S->ld = pattern_ld(h->pattern);
    const HostGrid &G = h->G;
    std::vector<uint8_t> wet((size_t)G.nx * G.ny);
    for (size_t e = 0; e < wet.size(); ++e) wet[e] = G.idx[e] >= 0 ? 1 : 0;
    std::string err;
    int rc = band_rows(G.nx, G.ny, wet.data(), h->pattern, nbands, S->row0, S->halo, err);
    if (rc) { set_error(err); return rc; }
    const int H = S->halo;
    // band planes: own rows plus the halo rows of each neighbour
    std::vector<GridDev<double>> gds;
    std::vector<Unit> units;
    for (int b = 0; b < nbands; ++b) {
      const int lo = b > 0 ? H : 0, hi = b < nbands - 1 ? H : 0;
      const int a = S->row0[b] - lo, c = S->row0[b + 1] + hi;
      auto bh = std::make_unique<pcg_handle>();
      slice(G, h->F, a, c, bh->G, bh->F);
      bh->pattern = h->pattern; bh->band_q = h->band_q; bh->tau = h->tau;
      bh->tx = h->tx; bh->ty = h->ty;
      if ((rc = upload_planes64(bh.get(), s))) { bh->p64.release(); return rc; }
      const auto &P = bh->p64;
      GridDev<double> gd = P.gd;
      gd.row_off = a;
      gd.own0 = lo;
      gd.own1 = lo + (S->row0[b + 1] - S->row0[b]);
      gd.u_off = (int32_t)units.size();
      // units: strips of the own rows holding a wet cell (rows own0 + sy * ty ...)
      const int ntx = (G.nx + h->tx - 1) / h->tx;
      const int own = gd.own1 - gd.own0, nty = (own + h->ty - 1) / h->ty;
      for (int sy = 0; sy < nty; ++sy)
        for (int sx = 0; sx < ntx; ++sx) {
          bool any = false;
          for (int j = gd.own0 + sy * h->ty; j < std::min(gd.own1, gd.own0 + (sy + 1) * h->ty) && !any; ++j)
            for (int i = sx * h->tx; i < std::min(G.nx, (sx + 1) * h->tx); ++i)
              if (bh->G.idx[(size_t)j * G.nx + i] >= 0) { any = true; break; }
          if (!any) continue;
          Unit u{};
          u.g = (int16_t)b; u.sx = (int16_t)sx; u.sy = (int16_t)sy; u.u = (int32_t)units.size();
          units.push_back(u);
        }
      gds.push_back(gd);
      S->bands.push_back(std::move(bh));
    }
    S->n_units = (int)units.size();
    if (S->n_units == 0) { set_error("the grid has no wet point"); return PCG_EINVAL; }
    // one reduction state and one partial array for all bands
    CK(cudaMalloc(&S->st, sizeof(SolveState)));
    CK(cudaMemset(S->st, 0, sizeof(SolveState)));
    CK(cudaMalloc(&S->partial, sizeof(double) * 2 * S->n_units));
    CK(cudaMalloc(&S->ls, sizeof(LaunchState)));
    CK(cudaMemset(S->ls, 0, sizeof(LaunchState)));
    if (cudaMallocHost(&S->st_host, sizeof(SolveState)) != cudaSuccess ||
        cudaMallocHost(&S->ls_host, sizeof(LaunchState)) != cudaSuccess) {
      cudaGetLastError(); set_error("pinned allocation failed"); return PCG_ENOMEM;
    }
    for (auto &gd : gds) { gd.st = S->st; gd.partial = S->partial; gd.n_units = S->n_units; }
    void *gd_dev = nullptr, *un_dev = nullptr;
    CK(cudaMalloc(&gd_dev, sizeof(GridDev<double>) * gds.size()));
    S->plan.owned.push_back(gd_dev);
    CK(cudaMalloc(&un_dev, sizeof(Unit) * units.size()));
    S->plan.owned.push_back(un_dev);
    CK(cudaMemcpy(gd_dev, gds.data(), sizeof(GridDev<double>) * gds.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(un_dev, units.data(), sizeof(Unit) * units.size(), cudaMemcpyHostToDevice));
    PlanGroup pg;
    pg.ks = S->bands[0]->p64.ks;
    pg.n_units = S->n_units;
    pg.gd_dev = gd_dev;
    pg.units_dev = (const Unit *)un_dev;
    S->plan.groups.push_back(pg);
    S->plan.ls = S->ls;
    // exchange lists: for every pair of neighbouring bands and every plane of
    // an exchange point, its boundary rows up into the upper band's lower halo
    // and down into the lower band's upper halo
    struct Field { int vec, depth; };
    const std::vector<std::vector<Field>> points = {
        {{0, 1}},                                   // x
        {{3, S->ld}, {4, S->ld}},                   // r (both planes)
        {{5, 1}, {6, 1}, {2, S->ld}},               // d (both planes), q
        {{1, 1}, {3, S->ld}, {4, S->ld}}};          // s, r (both planes)
    for (int pt = 0; pt < 4; ++pt) {
      std::vector<HaloCopy> list;
      for (int b = 0; b + 1 < nbands; ++b) {
        const auto &L = S->bands[b]->p64, &U = S->bands[b + 1]->p64;
        const GridDev<double> &gl = gds[b], &gu = gds[b + 1];
        for (const Field &f : points[pt]) {
          if (f.depth <= 0) continue;
          const int64_t n = (int64_t)f.depth * L.pitch;
          auto row = [](const DevPlanes<double> &P, int idx, int r) { return P.plane_start(idx) + (size_t)(GY + r) * P.pitch; };
          list.push_back({row(L, L.vec(f.vec), gl.own1 - f.depth), row(U, U.vec(f.vec), gu.own0 - f.depth), n});
          list.push_back({row(U, U.vec(f.vec), gu.own0), row(L, L.vec(f.vec), gl.own1), n});
        }
      }
      S->nex[pt] = (int)list.size();
      if (!list.empty()) {
        CK(cudaMalloc(&S->ex[pt], sizeof(HaloCopy) * list.size()));
        CK(cudaMemcpy(S->ex[pt], list.data(), sizeof(HaloCopy) * list.size(), cudaMemcpyHostToDevice));
      }
    }
    if ((rc = build_shard_graph(*S))) return rc;
    *out = S.release();
    return PCG_OK;
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return PCG_ENOMEM;
  }
}

int pcg_shard_bands(const pcg_shard *sh, int32_t *nbands, int32_t *row0, int32_t *halo) {
  if (!sh) { set_error("NULL shard"); return PCG_EINVAL; }
  if (nbands) *nbands = sh->nb;
  if (row0) for (int b = 0; b <= sh->nb; ++b) row0[b] = sh->row0[b];
  if (halo) *halo = sh->halo;
  return PCG_OK;
}

int pcg_shard_solve(pcg_shard *sh, const double *b, double *x, const pcg_opts *opts, pcg_stats *stats,
                    void *cuda_stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!sh || !b || !x) { set_error("NULL argument"); return PCG_EINVAL; }
  if (!is_device_ptr(b) || !is_device_ptr(x)) { set_error("b and x must be device pointers"); return PCG_EINVAL; }
  pcg_opts o;
  fill_opts(opts, o);
  if (o.prec != PCG_FP64) { set_error("the sharded solve is binary64"); return PCG_EINVAL; }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const PlanGroup &G = sh->plan.groups[0];
  // inputs of every band: b on its own rows, x0 (or 0) and zero directions on all its rows
  for (auto &bh : sh->bands) {
    auto &P = bh->p64;
    if (!o.use_x0) CK(cudaMemsetAsync(P.plane_start(P.vec(0)), 0, P.plane_elems * sizeof(double), s));
    for (int v : {5, 6}) CK(cudaMemsetAsync(P.plane_start(P.vec(v)), 0, P.plane_elems * sizeof(double), s));
  }
  {
    KParams p{};
    p.grids = G.gd_dev;
    p.units = G.units_dev;
    for (int which = 0; which < (o.use_x0 ? 2 : 1); ++which) {
      const double *src = which == 0 ? b : x;
      void *args[] = {&p, (void *)&src, &which};
      CK(cudaLaunchKernel(G.ks.pack, dim3(G.n_units), dim3(G.ks.tx), args, 0, s));
      note_launches(1);
    }
  }
  {
    SolveState **stp = sh->graph->st64;
    int32_t *nwp = sh->graph->n_wet;
    int n = 1;
    double rtol = o.rtol, irt = o.inner_rtol;
    int mi = o.max_iter, mr = o.max_replace, mo = o.max_outer, bud = std::max(sh->h->G.n, 1);
    LaunchState *ls = sh->ls;
    void *args[] = {&stp, &nwp, &n, &rtol, &mi, &mr, &irt, &mo, &bud, &ls};
    CK(cudaLaunchKernel((const void *)k_ctl_begin, dim3(1), dim3(CTL_THREADS), args, 0, s));
    note_launches(1);
  }
  CK(cudaGraphLaunch(sh->graph->exec, s));
  for (int bi = 0; bi < sh->nb; ++bi) {
    const GridDev<double> *gdp = reinterpret_cast<const GridDev<double> *>(G.gd_dev) + bi;
    double *dst = x;
    int which = 0;
    void *args[] = {(void *)&gdp, (void *)&dst, &which};
    const auto &P = sh->bands[bi]->p64;
    const size_t cells = (size_t)P.nx * P.ny;
    const int blocks = (int)std::min<size_t>((cells + 255) / 256, 148 * 16);
    CK(cudaLaunchKernel(G.ks.unpack, dim3(std::max(blocks, 1)), dim3(256), args, 0, s));
    note_launches(1);
  }
  CK(cudaMemcpyAsync(sh->st_host, sh->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(sh->ls_host, sh->ls, sizeof(LaunchState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const SolveState &st = *sh->st_host;
  const LaunchState &ls = *sh->ls_host;
  note_launches((uint64_t)std::max(ls.passes, 0) * sh->graph->outer_kernels +
                (uint64_t)std::max(ls.bodies_total, 0) * sh->graph->inner_kernels);
  const int status = st.final_status >= 0 ? st.final_status : PCG_ETIMEOUT;
  if (stats) {
    stats->iters = st.iter;
    stats->outer_iters = 1 + st.replacements;
    stats->status = status;
    stats->replacements = st.replacements;
    stats->relres = st.bb > 0 ? std::sqrt(st.rr) / std::sqrt(st.bb) : 0.0;
    stats->true_relres = st.bb > 0 ? std::sqrt(st.rr_true) / std::sqrt(st.bb) : 0.0;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status != PCG_OK) set_error("sharded solve finished with status: " + status_name(status));
  return status;
}

void pcg_shard_free(pcg_shard *sh) { delete sh; }

}  // extern "C"
