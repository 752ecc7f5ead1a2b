// Host side of ainv_setup: input validation, assembly of the five-point
// operator, and the factored approximate inverse M^-1 = Z D^-1 Z^T built by
// LEFT-looking conjugate orthogonalisation (Section 3: "computed by means of a
// conjugate-orthogonalization procedure" restricted to a sparsity pattern; the
// paper runs this step serially on the CPU, Section 4).
//
// Left-looking form: column j starts as e_j; for every earlier column i whose
// row of A meets the pattern of column j (in increasing i), p = a_i^T z_j,
// z_j <- z_j - (p / d_i) z_i kept to the pattern of j, then entries with
// |z_mj| sqrt(a_mm / a_jj) < tau are dropped; finally d_j = a_j^T z_j. The
// sequence of operations on each column is the same as in the right-looking
// form (same i order, same finished z_i), so both give the same factor.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "pcg_internal.h"

namespace pcg {

SlotSet slot_set(int pattern, int band_q) {
  SlotSet s;
  auto add = [&](int dx, int dy) { s.dx[s.n] = dx; s.dy[s.n] = dy; ++s.n; };
  switch (pattern) {
    case PCG_PAT_TRIL_A:
      add(-1, 0); add(0, -1);
      s.n_wrap = 1; s.wcol[0] = 0; s.wdx[0] = 1;            // (nx-1, j) -> (0, j)
      s.lower_rows = 1; s.reach = 1;
      break;
    case PCG_PAT_TRIL_A2:
      add(-2, 0); add(-1, 0); add(-1, -1); add(0, -1); add(1, -1); add(0, -2);
      s.n_wrap = 3;
      s.wcol[0] = 0; s.wdx[0] = 1;                          // (nx-1, j) -> (0, j)
      s.wcol[1] = 0; s.wdx[1] = 2;                          // (nx-1, j) -> (1, j)
      s.wcol[2] = 1; s.wdx[2] = 2;                          // (nx-2, j) -> (0, j)
      s.lower_rows = 2; s.reach = 2;
      break;
    case PCG_PAT_BAND_T:
      for (int t = 1; t <= band_q; ++t) add(-t, 0);
      s.lower_rows = 0; s.reach = band_q;
      break;
    case PCG_PAT_DIAG:
    default:
      break;
  }
  return s;
}

static bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

int host_grid_build(const pcg_grid *g, int pattern, HostGrid &G, std::string &err) {
  if (!g) { err = "grid is NULL"; return PCG_EINVAL; }
  if (!g->wet || !g->c_e || !g->c_n || !g->shift) { err = "grid has a NULL field"; return PCG_EINVAL; }
  const int32_t nx = g->nx, ny = g->ny;
  if (nx < 3 || ny < 1) { err = "grid must be at least 3 x 1 (nx >= 3: the periodic row needs distinct east and west neighbours)"; return PCG_EINVAL; }
  if (pattern == PCG_PAT_TRIL_A2 && nx < 5) { err = "pattern tril(A^2) needs nx >= 5"; return PCG_EINVAL; }
  if ((int64_t)nx * ny > (int64_t)1 << 30) { err = "grid too large"; return PCG_EINVAL; }
  G.nx = nx; G.ny = ny;
  const size_t N = (size_t)nx * ny;
  G.idx.assign(N, -1);
  int32_t n = 0;
  for (size_t p = 0; p < N; ++p)
    if (g->wet[p]) G.idx[p] = n++;
  G.n = n;
  G.pi.resize(n); G.pj.resize(n);
  G.ce.assign(N, 0.0); G.cn.assign(N, 0.0);
  G.diag.assign(n, 0.0);
  for (int32_t j = 0; j < ny; ++j) {
    for (int32_t i = 0; i < nx; ++i) {
      const size_t p = (size_t)j * nx + i;
      const int32_t k = G.idx[p];
      if (k < 0) continue;
      G.pi[k] = i; G.pj[k] = j;
      if (!(std::isfinite(g->shift[p]) && g->shift[p] > 0.0)) {
        err = "shift must be positive and finite on every wet cell (i=" + std::to_string(i) + ", j=" + std::to_string(j) + ")";
        return PCG_EINVAL;
      }
      const int32_t ie = (i + 1) % nx;
      if (g->wet[(size_t)j * nx + ie]) {
        if (!finite_nonneg(g->c_e[p])) { err = "c_e must be >= 0 and finite"; return PCG_EINVAL; }
        G.ce[p] = g->c_e[p];
      }
      if (j + 1 < ny && g->wet[(size_t)(j + 1) * nx + i]) {
        if (!finite_nonneg(g->c_n[p])) { err = "c_n must be >= 0 and finite"; return PCG_EINVAL; }
        G.cn[p] = g->c_n[p];
      }
    }
  }
  for (int32_t k = 0; k < n; ++k) {
    const int32_t i = G.pi[k], j = G.pj[k];
    const int32_t iw = (i - 1 + nx) % nx;
    double a = g->shift[(size_t)j * nx + i];
    a += G.ce[(size_t)j * nx + i];                       // east face
    a += G.ce[(size_t)j * nx + iw];                      // west face
    if (j + 1 < ny) a += G.cn[(size_t)j * nx + i];       // north face
    if (j > 0) a += G.cn[(size_t)(j - 1) * nx + i];      // south face
    G.diag[k] = a;
  }
  return PCG_OK;
}

namespace {

// Neighbourhood of point k in the graph of the matrix the factor is built
// from (A, or its east-west part T for the banded pattern), with coefficients.
struct Nb {
  int32_t m[5];
  double a[5];
  int cnt;
};

struct Builder {
  const HostGrid &G;
  bool tri;                 // use T (east-west couplings only, no periodic face)
  Builder(const HostGrid &g, bool t) : G(g), tri(t) {}

  // row k of the source matrix, columns ascending
  Nb row(int32_t k) const {
    Nb r; r.cnt = 0;
    const int32_t nx = G.nx, ny = G.ny, i = G.pi[k], j = G.pj[k];
    auto push = [&](int32_t m, double a) {
      if (m < 0 || a == 0.0) return;
      r.m[r.cnt] = m; r.a[r.cnt] = a; ++r.cnt;
    };
    const int32_t iw = (i - 1 + nx) % nx, ie = (i + 1) % nx;
    if (!tri && j > 0) push(G.idx[(size_t)(j - 1) * nx + i], -G.cn[(size_t)(j - 1) * nx + i]);
    if (!tri || i > 0) push(G.idx[(size_t)j * nx + iw], -G.ce[(size_t)j * nx + iw]);
    push(k, G.diag[k]);
    if (!tri || i + 1 < nx) push(G.idx[(size_t)j * nx + ie], -G.ce[(size_t)j * nx + i]);
    if (!tri && j + 1 < ny) push(G.idx[(size_t)(j + 1) * nx + i], -G.cn[(size_t)j * nx + i]);
    // ascending column order
    for (int a = 1; a < r.cnt; ++a) {
      int32_t mm = r.m[a]; double aa = r.a[a]; int b = a - 1;
      while (b >= 0 && r.m[b] > mm) { r.m[b + 1] = r.m[b]; r.a[b + 1] = r.a[b]; --b; }
      r.m[b + 1] = mm; r.a[b + 1] = aa;
    }
    return r;
  }
};

}  // namespace

int host_ainv(const HostGrid &G, int pattern, double tau, int band_q, HostFactor &F, std::string &err) {
  const int32_t n = G.n, nx = G.nx, ny = G.ny;
  const SlotSet S = slot_set(pattern, band_q);
  F.n = n; F.slots = S;
  F.d.assign(n, 0.0);
  F.z.assign((size_t)S.n * n, 0.0);
  F.zwrap.assign((size_t)ny * std::max(S.n_wrap, 1), 0.0);
  if (!(tau >= 0.0) || !std::isfinite(tau)) { err = "drop_tol must be >= 0"; return PCG_EINVAL; }
  const bool tri = (pattern == PCG_PAT_BAND_T);
  const int q = (pattern == PCG_PAT_TRIL_A) ? 1 : (pattern == PCG_PAT_TRIL_A2) ? 2 : (pattern == PCG_PAT_BAND_T) ? band_q : 0;
  Builder B(G, tri);
  const int NS = S.n + S.n_wrap;      // positions of a column besides the diagonal

  // Per-column position list: pos[t] = row index m of position t (or -1),
  // t = 0..NS-1 off-diagonal (slots then side-table entries), NS = diagonal.
  std::vector<int32_t> stamp(n, -1);
  std::vector<int32_t> cand;
  cand.reserve(64);
  std::vector<int32_t> pos(NS + 1), pos_i(NS + 1);
  std::vector<double> zj(NS + 1), zi(NS + 1);

  // rows of the pattern of column k: within q graph steps of k, index < k
  auto pattern_rows = [&](int32_t k, int32_t *out) {
    const int32_t i = G.pi[k], j = G.pj[k];
    for (int t = 0; t <= NS; ++t) out[t] = -1;
    out[NS] = k;
    if (q == 0) return;
    // breadth-first reach within q steps (q <= 8, neighbourhoods are tiny)
    int32_t front[512], next[512], seen[1024];
    int nf = 1, ns = 1;
    front[0] = k; seen[0] = k;
    for (int step = 0; step < q; ++step) {
      int nn = 0;
      for (int f = 0; f < nf; ++f) {
        Nb r = B.row(front[f]);
        for (int c = 0; c < r.cnt; ++c) {
          int32_t m = r.m[c];
          bool dup = false;
          for (int u = 0; u < ns; ++u) if (seen[u] == m) { dup = true; break; }
          if (dup) continue;
          seen[ns++] = m; next[nn++] = m;
        }
      }
      std::memcpy(front, next, sizeof(int32_t) * nn); nf = nn;
    }
    for (int u = 1; u < ns; ++u) {
      const int32_t m = seen[u];
      if (m >= k) continue;
      const int ddy = G.pj[m] - j;
      int slot = -1;
      if (ddy < 0) {
        // a row below: the plane of the periodic offset of smallest magnitude
        int pdx = G.pi[m] - i;
        if (pdx > nx / 2) pdx -= nx;
        if (pdx < -(nx / 2)) pdx += nx;
        for (int s = 0; s < S.n; ++s)
          if (S.dx[s] == pdx && S.dy[s] == ddy) { slot = s; break; }
      } else {
        // the same row: m < k means G.pi[m] < i. A short westward step is a
        // plane; a long one can only come through the periodic face.
        const int w = i - G.pi[m];
        if (w <= S.reach) {
          for (int s = 0; s < S.n; ++s)
            if (S.dx[s] == -w && S.dy[s] == 0) { slot = s; break; }
        } else {
          for (int t = 0; t < S.n_wrap; ++t)
            if (i == nx - 1 - S.wcol[t] && G.pi[m] == ((S.wdx[t] - 1 - S.wcol[t]) % nx + nx) % nx) { slot = S.n + t; break; }
        }
      }
      if (slot < 0 || out[slot] >= 0) { err = "internal: pattern entry without a slot"; return; }
      out[slot] = m;
    }
  };

  std::vector<int32_t> posall((size_t)n * (NS + 1));
  for (int32_t k = 0; k < n; ++k) pattern_rows(k, &posall[(size_t)k * (NS + 1)]);
  if (!err.empty()) return PCG_EINVAL;

  // values of finished columns, per position
  std::vector<double> zall((size_t)n * (NS + 1), 0.0);

  auto find = [&](const int32_t *p, int32_t m) -> int {
    for (int t = 0; t <= NS; ++t) if (p[t] == m) return t;
    return -1;
  };

  for (int32_t j = 0; j < n; ++j) {
    const int32_t *pj_ = &posall[(size_t)j * (NS + 1)];
    double *z = &zall[(size_t)j * (NS + 1)];
    for (int t = 0; t < NS; ++t) z[t] = 0.0;
    z[NS] = 1.0;
    // earlier columns i whose row of the source matrix meets the pattern of j
    cand.clear();
    for (int t = 0; t <= NS; ++t) {
      const int32_t m = pj_[t];
      if (m < 0) continue;
      Nb r = B.row(m);
      for (int c = 0; c < r.cnt; ++c) {
        const int32_t i = r.m[c];
        if (i < j && stamp[i] != j) { stamp[i] = j; cand.push_back(i); }
      }
    }
    std::sort(cand.begin(), cand.end());
    const double ajj = G.diag[j];
    for (int32_t i : cand) {
      // p = a_i^T z_j over the rows of a_i (ascending)
      Nb r = B.row(i);
      double p = 0.0;
      for (int c = 0; c < r.cnt; ++c) {
        const int t = find(pj_, r.m[c]);
        if (t >= 0) p += r.a[c] * z[t];
      }
      if (p == 0.0) continue;
      const double f = p / F.d[i];
      const int32_t *pi_ = &posall[(size_t)i * (NS + 1)];
      const double *zi_ = &zall[(size_t)i * (NS + 1)];
      // z_j -= f z_i over rows of column i in ascending order, kept to the pattern of j
      int order[32], no = 0;
      for (int t = 0; t <= NS; ++t) if (pi_[t] >= 0) order[no++] = t;
      std::sort(order, order + no, [&](int a, int b) { return pi_[a] < pi_[b]; });
      for (int o = 0; o < no; ++o) {
        const int t = order[o];
        if (zi_[t] == 0.0) continue;
        const int u = find(pj_, pi_[t]);
        if (u >= 0) z[u] -= f * zi_[t];
      }
      if (tau > 0.0) {
        for (int t = 0; t < NS; ++t) {
          const int32_t m = pj_[t];
          if (m < 0) continue;
          if (std::fabs(z[t]) * std::sqrt(G.diag[m] / ajj) < tau) z[t] = 0.0;
        }
      }
    }
    // pivot d_j = a_j^T z_j
    Nb r = B.row(j);
    double dj = 0.0;
    for (int c = 0; c < r.cnt; ++c) {
      const int t = find(pj_, r.m[c]);
      if (t >= 0) dj += r.a[c] * z[t];
    }
    if (!(dj > 0.0) || !std::isfinite(dj)) {
      err = "non-positive pivot in the approximate inverse at unknown " + std::to_string(j);
      return PCG_EBREAKDOWN;
    }
    F.d[j] = dj;
  }
  // scatter into slot planes and the side table
  for (int32_t k = 0; k < n; ++k) {
    const int32_t *p = &posall[(size_t)k * (NS + 1)];
    const double *z = &zall[(size_t)k * (NS + 1)];
    for (int s = 0; s < S.n; ++s) if (p[s] >= 0) F.z[(size_t)s * n + k] = z[s];
    for (int w = 0; w < S.n_wrap; ++w) if (p[S.n + w] >= 0) F.zwrap[(size_t)G.pj[k] * S.n_wrap + w] = z[S.n + w];
  }
  return PCG_OK;
}

}  // namespace pcg
