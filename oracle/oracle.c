/*
 * FP64 CPU oracle for the AINV-preconditioned conjugate gradient solve of the
 * ocean free-surface elliptic system (Cuomo, De Michele, Farina, Chinnici,
 * "A PCG implementation of an elliptic kernel in an ocean global circulation
 * model based on GPU libraries").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the CUDA library computes. Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header, table or helper with the library.
 *
 * Everything is IEEE binary64, sequential, summed in natural order. Built with
 * -ffp-contract=off so that no multiply-add is fused behind our back.
 *
 * Sections followed:
 *   operator ............ Section 3, Eq. 9 (five-point system), negated to the
 *                         SPD form the paper states, plus the mass shift that
 *                         the D^{n+1} term of Section 2, Eq. 2 contributes.
 *                         Unknowns: wet points in the natural ordering of
 *                         Section 3 (west->east fastest, then south->north),
 *                         east-west periodic, north/south closed.
 *   preconditioner ...... Section 3 (last part): factored approximate inverse
 *                         M^-1 = Z D^-1 Z^T built by the conjugate
 *                         (A-)orthogonalisation of the unit vectors, restricted
 *                         to a sparsity pattern; classic right-looking AINV.
 *                         Pattern and drop tolerance are applied after every
 *                         update of a column.
 *   solver .............. Algorithm 1 (FSAI-PCG) with two readings: the new
 *                         direction is d = s + beta d (standard PCG; the
 *                         printed r is a typo) and, on exit, the true residual
 *                         b - A x is checked and, if it fails the tolerance, the
 *                         iteration restarts from it (at most max_replace times).
 *   Jacobi .............. Section 3, Eqs. 10-12: diagonal preconditioner, which
 *                         is the same AINV with the one-entry pattern {k}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { O_OK = 0, O_EINVAL = 1, O_ENOMEM = 2, O_ENOTCONV = 4, O_EBREAKDOWN = 5 };
enum { O_PAT_TRIL_A = 0, O_PAT_TRIL_A2 = 1, O_PAT_FULL = 2, O_PAT_BAND_T = 3, O_PAT_DIAG = 4 };

typedef struct {
  int32_t nx, ny, n;
  int32_t *idx;              /* [ny*nx]: unknown number of (i,j) or -1 on land */
  int32_t *pi, *pj;          /* [n]: grid coordinates of unknown k */
  int64_t *rowptr;           /* CSR of A, columns ascending */
  int32_t *col;
  double *val;
  /* matrix the preconditioner is built from (A itself, or T) */
  int64_t *srowptr;
  int32_t *scol;
  double *sval;
  /* Z stored column by column over its pattern (rows ascending, diagonal last) */
  int64_t *zptr;
  int32_t *zrow;
  double *zval;
  double *d;
  int have_z;
} oproblem;

typedef struct {
  int32_t iters, status, replacements, pad;
  double relres, true_relres, bnorm;
} oracle_stats;

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s ? s : 1); }

/* ------------------------------------------------------------------ operator */

/* Append (c, v) to a short row list, merging equal columns. */
static int row_add(int32_t *cols, double *vals, int cnt, int32_t c, double v) {
  for (int t = 0; t < cnt; ++t)
    if (cols[t] == c) { vals[t] += v; return cnt; }
  cols[cnt] = c; vals[cnt] = v;
  return cnt + 1;
}

static void row_sort(int32_t *cols, double *vals, int cnt) {
  for (int a = 1; a < cnt; ++a) {
    int32_t c = cols[a]; double v = vals[a]; int b = a - 1;
    while (b >= 0 && cols[b] > c) { cols[b + 1] = cols[b]; vals[b + 1] = vals[b]; --b; }
    cols[b + 1] = c; vals[b + 1] = v;
  }
}

oproblem *oracle_problem_new(int32_t nx, int32_t ny, const uint8_t *wet, const double *c_e,
                             const double *c_n, const double *shift) {
  if (nx < 1 || ny < 1) return NULL;
  oproblem *P = (oproblem *)xcalloc(1, sizeof(oproblem));
  P->nx = nx; P->ny = ny;
  P->idx = (int32_t *)xcalloc((size_t)nx * ny, sizeof(int32_t));
  int32_t n = 0;
  for (int32_t j = 0; j < ny; ++j)
    for (int32_t i = 0; i < nx; ++i)
      P->idx[(size_t)j * nx + i] = wet[(size_t)j * nx + i] ? n++ : -1;
  P->n = n;
  P->pi = (int32_t *)xcalloc(n, sizeof(int32_t));
  P->pj = (int32_t *)xcalloc(n, sizeof(int32_t));
  P->rowptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  P->col = (int32_t *)xcalloc((size_t)n * 5, sizeof(int32_t));
  P->val = (double *)xcalloc((size_t)n * 5, sizeof(double));
  int64_t nnz = 0;
  for (int32_t j = 0; j < ny; ++j) {
    for (int32_t i = 0; i < nx; ++i) {
      int32_t k = P->idx[(size_t)j * nx + i];
      if (k < 0) continue;
      P->pi[k] = i; P->pj[k] = j;
      int32_t cols[5]; double vals[5]; int cnt = 0;
      double diag = shift[(size_t)j * nx + i];
      /* the four faces of cell (i,j); a face counts only if both cells are wet */
      int32_t iw = (i - 1 + nx) % nx, ie = (i + 1) % nx;
      struct { int32_t ii, jj; double c; int ok; } face[4] = {
        { iw, j, c_e[(size_t)j * nx + iw], nx > 1 },                 /* west  */
        { ie, j, c_e[(size_t)j * nx + i], nx > 1 },                  /* east  */
        { i, j - 1, j > 0 ? c_n[(size_t)(j - 1) * nx + i] : 0.0, j > 0 },   /* south */
        { i, j + 1, j + 1 < ny ? c_n[(size_t)j * nx + i] : 0.0, j + 1 < ny }, /* north */
      };
      for (int f = 0; f < 4; ++f) {
        if (!face[f].ok) continue;
        int32_t m = P->idx[(size_t)face[f].jj * nx + face[f].ii];
        if (m < 0 || face[f].c == 0.0) continue;
        diag += face[f].c;
        if (m == k) { diag -= face[f].c; continue; }   /* a face of a cell with itself (nx == 1) */
        cnt = row_add(cols, vals, cnt, m, -face[f].c);
      }
      cnt = row_add(cols, vals, cnt, k, diag);
      row_sort(cols, vals, cnt);
      for (int t = 0; t < cnt; ++t) { P->col[nnz] = cols[t]; P->val[nnz] = vals[t]; ++nnz; }
      P->rowptr[k + 1] = nnz;
    }
  }
  return P;
}

void oracle_problem_free(oproblem *P) {
  if (!P) return;
  free(P->idx); free(P->pi); free(P->pj); free(P->rowptr); free(P->col); free(P->val);
  if (P->srowptr != P->rowptr) { free(P->srowptr); free(P->scol); free(P->sval); }
  free(P->zptr); free(P->zrow); free(P->zval); free(P->d);
  free(P);
}

int32_t oracle_n(const oproblem *P) { return P->n; }
int64_t oracle_nnz(const oproblem *P) { return P->rowptr[P->n]; }

void oracle_get_csr(const oproblem *P, int64_t *rowptr, int32_t *col, double *val, int32_t *pi, int32_t *pj) {
  memcpy(rowptr, P->rowptr, sizeof(int64_t) * ((size_t)P->n + 1));
  memcpy(col, P->col, sizeof(int32_t) * (size_t)P->rowptr[P->n]);
  memcpy(val, P->val, sizeof(double) * (size_t)P->rowptr[P->n]);
  memcpy(pi, P->pi, sizeof(int32_t) * (size_t)P->n);
  memcpy(pj, P->pj, sizeof(int32_t) * (size_t)P->n);
}

/* y = A x over the wet unknowns. */
void oracle_spmv(const oproblem *P, const double *x, double *y) {
  for (int32_t k = 0; k < P->n; ++k) {
    double acc = 0.0;
    for (int64_t t = P->rowptr[k]; t < P->rowptr[k + 1]; ++t) acc += P->val[t] * x[P->col[t]];
    y[k] = acc;
  }
}

static double dot(const double *a, const double *b, int32_t n) {
  double acc = 0.0;
  for (int32_t k = 0; k < n; ++k) acc += a[k] * b[k];
  return acc;
}

/* ------------------------------------------------------------ preconditioner */

static double sdiag(const oproblem *P, int32_t k) {
  for (int64_t t = P->srowptr[k]; t < P->srowptr[k + 1]; ++t)
    if (P->scol[t] == k) return P->sval[t];
  return 0.0;
}

/* The east-west tridiagonal part T of A (Section 3, pattern-selection step 1):
 * the diagonal of A plus the couplings of each point with its west and east
 * neighbours in the same latitude row, without the periodic wrap face. */
static void build_T(oproblem *P) {
  int32_t n = P->n;
  P->srowptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  P->scol = (int32_t *)xcalloc((size_t)n * 3, sizeof(int32_t));
  P->sval = (double *)xcalloc((size_t)n * 3, sizeof(double));
  int64_t nnz = 0;
  for (int32_t k = 0; k < n; ++k) {
    for (int64_t t = P->rowptr[k]; t < P->rowptr[k + 1]; ++t) {
      int32_t m = P->col[t];
      int keep = (m == k) || (P->pj[m] == P->pj[k] && abs(P->pi[m] - P->pi[k]) == 1);
      if (keep) { P->scol[nnz] = m; P->sval[nnz] = P->val[t]; ++nnz; }
    }
    P->srowptr[k + 1] = nnz;
  }
}

/* Pattern of column k of Z: the rows m <= k with (S^q)_{mk} structurally
 * non-zero, i.e. m within q steps of k in the graph of S. */
static int32_t pattern_of(const oproblem *P, int32_t k, int q, int32_t *out, int32_t *stamp,
                          int32_t *frontier, int32_t *next) {
  int32_t cnt = 0, nf = 1;
  stamp[k] = k; frontier[0] = k; out[cnt++] = k;
  for (int step = 0; step < q; ++step) {
    int32_t nn = 0;
    for (int32_t f = 0; f < nf; ++f) {
      int32_t v = frontier[f];
      for (int64_t t = P->srowptr[v]; t < P->srowptr[v + 1]; ++t) {
        int32_t m = P->scol[t];
        if (stamp[m] == k) continue;
        stamp[m] = k; next[nn++] = m;
        if (m < k) out[cnt++] = m;
      }
    }
    memcpy(frontier, next, sizeof(int32_t) * (size_t)nn);
    nf = nn;
  }
  /* rows ascending (the diagonal k is the largest) */
  for (int32_t a = 1; a < cnt; ++a) {
    int32_t c = out[a], b = a - 1;
    while (b >= 0 && out[b] > c) { out[b + 1] = out[b]; --b; }
    out[b + 1] = c;
  }
  return cnt;
}

static int64_t zfind(const oproblem *P, int32_t j, int32_t m) {
  int64_t lo = P->zptr[j], hi = P->zptr[j + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (P->zrow[mid] == m) return mid;
    if (P->zrow[mid] < m) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* Build Z and D. pattern: O_PAT_*; tau: drop tolerance on the scaled entries
 * |z_mj| sqrt(s_mm / s_jj); band_q: q of the banded-T pattern. */
int oracle_ainv(oproblem *P, int32_t pattern, double tau, int32_t band_q) {
  int32_t n = P->n;
  free(P->zptr); free(P->zrow); free(P->zval); free(P->d);
  if (P->srowptr && P->srowptr != P->rowptr) { free(P->srowptr); free(P->scol); free(P->sval); }
  P->srowptr = NULL; P->have_z = 0;
  int q;
  switch (pattern) {
    case O_PAT_TRIL_A: q = 1; break;
    case O_PAT_TRIL_A2: q = 2; break;
    case O_PAT_DIAG: q = 0; break;
    case O_PAT_BAND_T: q = band_q; if (q < 0) return O_EINVAL; break;
    case O_PAT_FULL: q = n; break;
    default: return O_EINVAL;
  }
  if (pattern == O_PAT_BAND_T) build_T(P);
  else { P->srowptr = P->rowptr; P->scol = P->col; P->sval = P->val; }

  /* patterns */
  int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t *fa = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t *fb = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  for (int32_t k = 0; k < n; ++k) stamp[k] = -1;
  P->zptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  size_t cap = (size_t)n * 8 + 16, used = 0;
  P->zrow = (int32_t *)malloc(sizeof(int32_t) * cap);
  for (int32_t k = 0; k < n; ++k) {
    int32_t cnt;
    if (pattern == O_PAT_FULL) {
      cnt = k + 1;
      for (int32_t m = 0; m <= k; ++m) tmp[m] = m;
    } else {
      cnt = pattern_of(P, k, q, tmp, stamp, fa, fb);
    }
    if (used + (size_t)cnt > cap) {
      while (used + (size_t)cnt > cap) cap *= 2;
      P->zrow = (int32_t *)realloc(P->zrow, sizeof(int32_t) * cap);
    }
    memcpy(P->zrow + used, tmp, sizeof(int32_t) * (size_t)cnt);
    used += (size_t)cnt;
    P->zptr[k + 1] = (int64_t)used;
  }
  P->zval = (double *)xcalloc(used, sizeof(double));
  P->d = (double *)xcalloc(n, sizeof(double));
  for (int32_t k = 0; k < n; ++k) P->zval[P->zptr[k + 1] - 1] = 1.0;   /* z_k = e_k */

  /* rows -> columns whose pattern holds that row */
  int64_t *uptr = (int64_t *)xcalloc((size_t)n + 1, sizeof(int64_t));
  for (size_t t = 0; t < used; ++t) uptr[P->zrow[t] + 1]++;
  for (int32_t m = 0; m < n; ++m) uptr[m + 1] += uptr[m];
  int32_t *ucol = (int32_t *)malloc(sizeof(int32_t) * (used + 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  memcpy(fill, uptr, sizeof(int64_t) * ((size_t)n + 1));
  for (int32_t j = 0; j < n; ++j)
    for (int64_t t = P->zptr[j]; t < P->zptr[j + 1]; ++t) ucol[fill[P->zrow[t]]++] = j;
  free(fill);

  double *sd = (double *)malloc(sizeof(double) * ((size_t)n + 1));
  for (int32_t k = 0; k < n; ++k) sd[k] = sdiag(P, k);
  for (int32_t k = 0; k < n; ++k) stamp[k] = -1;
  int status = O_OK;

  for (int32_t i = 0; i < n && status == O_OK; ++i) {
    /* pivot d_i = s_i^T z_i */
    double di = 0.0;
    for (int64_t t = P->srowptr[i]; t < P->srowptr[i + 1]; ++t) {
      int64_t pos = zfind(P, i, P->scol[t]);
      if (pos >= 0) di += P->sval[t] * P->zval[pos];
    }
    if (!(di > 0.0) || !isfinite(di)) { status = O_EBREAKDOWN; break; }
    P->d[i] = di;
    /* every later column whose pattern meets the closed neighbourhood of row i */
    int32_t ncand = 0;
    for (int64_t t = P->srowptr[i]; t < P->srowptr[i + 1]; ++t) {
      int32_t m = P->scol[t];
      for (int64_t u = uptr[m]; u < uptr[m + 1]; ++u) {
        int32_t j = ucol[u];
        if (j > i && stamp[j] != i) { stamp[j] = i; tmp[ncand++] = j; }
      }
    }
    for (int32_t c = 0; c < ncand; ++c) {
      int32_t j = tmp[c];
      double pj = 0.0;                                   /* p_j = s_i^T z_j */
      for (int64_t t = P->srowptr[i]; t < P->srowptr[i + 1]; ++t) {
        int64_t pos = zfind(P, j, P->scol[t]);
        if (pos >= 0) pj += P->sval[t] * P->zval[pos];
      }
      if (pj == 0.0) continue;
      double f = pj / di;
      /* z_j <- z_j - (p_j / d_i) z_i, kept to the pattern of column j */
      for (int64_t t = P->zptr[i]; t < P->zptr[i + 1]; ++t) {
        if (P->zval[t] == 0.0) continue;
        int64_t pos = zfind(P, j, P->zrow[t]);
        if (pos >= 0) P->zval[pos] -= f * P->zval[t];
      }
      /* drop small scaled off-diagonal entries */
      if (tau > 0.0) {
        for (int64_t t = P->zptr[j]; t < P->zptr[j + 1] - 1; ++t) {
          int32_t m = P->zrow[t];
          if (fabs(P->zval[t]) * sqrt(sd[m] / sd[j]) < tau) P->zval[t] = 0.0;
        }
      }
    }
  }
  free(stamp); free(fa); free(fb); free(tmp); free(uptr); free(ucol); free(sd);
  if (status == O_OK) P->have_z = 1;
  return status;
}

int64_t oracle_z_nnz(const oproblem *P) { return P->zptr ? P->zptr[P->n] : 0; }

/* Z in compressed columns over its pattern (explicit zeros left by dropping kept) and D. */
void oracle_get_z(const oproblem *P, int64_t *colptr, int32_t *row, double *val, double *d) {
  int64_t nz = P->zptr[P->n];
  memcpy(colptr, P->zptr, sizeof(int64_t) * ((size_t)P->n + 1));
  memcpy(row, P->zrow, sizeof(int32_t) * (size_t)nz);
  memcpy(val, P->zval, sizeof(double) * (size_t)nz);
  memcpy(d, P->d, sizeof(double) * (size_t)P->n);
}

/* s = Z (D^-1 (Z^T r)) */
int oracle_apply(const oproblem *P, const double *r, double *s) {
  if (!P->have_z) return O_EINVAL;
  int32_t n = P->n;
  double *t = (double *)xcalloc(n, sizeof(double));
  for (int32_t j = 0; j < n; ++j) {
    double acc = 0.0;
    for (int64_t u = P->zptr[j]; u < P->zptr[j + 1]; ++u) acc += P->zval[u] * r[P->zrow[u]];
    t[j] = acc / P->d[j];
  }
  for (int32_t m = 0; m < n; ++m) s[m] = 0.0;
  for (int32_t j = 0; j < n; ++j)
    for (int64_t u = P->zptr[j]; u < P->zptr[j + 1]; ++u) s[P->zrow[u]] += P->zval[u] * t[j];
  free(t);
  return O_OK;
}

/* ------------------------------------------------------------------- solver */

/* Algorithm 1 with the readings stated at the top of this file.
 * b, x: wet-compressed vectors of length n. x holds x0 on entry when use_x0.
 * The histories (length hist_cap, may be NULL) receive alpha_k, beta_k and
 * ||r_{k+1}|| / ||b|| per iteration. */
int oracle_pcg(const oproblem *P, const double *b, double *x, int32_t use_x0, double rtol,
               int32_t max_iter, int32_t max_replace, oracle_stats *st, double *alpha_hist,
               double *beta_hist, double *res_hist, int32_t hist_cap) {
  int32_t n = P->n;
  memset(st, 0, sizeof(*st));
  if (!P->have_z) { st->status = O_EINVAL; return O_EINVAL; }
  if (!use_x0) for (int32_t k = 0; k < n; ++k) x[k] = 0.0;
  double *r = (double *)xcalloc(n, sizeof(double));
  double *s = (double *)xcalloc(n, sizeof(double));
  double *d = (double *)xcalloc(n, sizeof(double));
  double *q = (double *)xcalloc(n, sizeof(double));
  double bnorm = sqrt(dot(b, b, n));
  st->bnorm = bnorm;
  if (bnorm == 0.0) {                       /* A x = 0 has the solution x = 0 */
    for (int32_t k = 0; k < n; ++k) x[k] = 0.0;
    free(r); free(s); free(d); free(q);
    st->status = O_OK;
    return O_OK;
  }
  int32_t k = 0, status = O_OK;
  for (int32_t rep = 0;; ++rep) {
    /* r = b - A x;  s = M^-1 r;  d = s;  rho = (s, r) */
    oracle_spmv(P, x, q);
    for (int32_t m = 0; m < n; ++m) r[m] = b[m] - q[m];
    oracle_apply(P, r, s);
    for (int32_t m = 0; m < n; ++m) d[m] = s[m];
    double rho = dot(s, r, n);
    double rnorm = sqrt(dot(r, r, n));
    while (rnorm / bnorm > rtol && k < max_iter) {
      oracle_spmv(P, d, q);                          /* q = A d */
      double dq = dot(d, q, n);
      if (!(dq > 0.0) || !isfinite(dq)) { status = O_EBREAKDOWN; break; }
      double alpha = rho / dq;
      for (int32_t m = 0; m < n; ++m) x[m] += alpha * d[m];
      for (int32_t m = 0; m < n; ++m) r[m] -= alpha * q[m];
      oracle_apply(P, r, s);                         /* s = M^-1 r */
      double rho_new = dot(s, r, n);
      rnorm = sqrt(dot(r, r, n));
      double beta = rho_new / rho;
      for (int32_t m = 0; m < n; ++m) d[m] = s[m] + beta * d[m];
      rho = rho_new;
      if (alpha_hist && k < hist_cap) { alpha_hist[k] = alpha; beta_hist[k] = beta; res_hist[k] = rnorm / bnorm; }
      ++k;
      if (!isfinite(rho)) { status = O_EBREAKDOWN; break; }
    }
    st->relres = rnorm / bnorm;
    oracle_spmv(P, x, q);
    for (int32_t m = 0; m < n; ++m) r[m] = b[m] - q[m];
    st->true_relres = sqrt(dot(r, r, n)) / bnorm;
    if (status != O_OK) break;
    if (st->true_relres <= rtol) { status = O_OK; break; }
    if (k >= max_iter || rep >= max_replace) { status = O_ENOTCONV; break; }
    st->replacements = rep + 1;
  }
  st->iters = k;
  st->status = status;
  free(r); free(s); free(d); free(q);
  return status;
}
