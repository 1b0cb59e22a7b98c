/*
 * gmls_oracle.c -- plain FP64 CPU oracle for GMLS stencil generation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header or table with
 * the CUDA path.
 *
 * It follows the paper ("Parallel implementation of a compatible high-order
 * meshless method for the Stokes' equations", arXiv 2104.14447) step by step:
 *
 *   neighbours   -- every particle within the support of x_T (Sec. 2.1, the
 *                   set N_T under Eq. (optimization-discretized-4)); here the
 *                   k nearest by exact squared distance, or all inside a radius.
 *   basis        -- generic polynomial term tables supplied by the caller
 *                   (scaled Taylor monomials, Eq. basis-functions-3d; curls of
 *                   monomials for the divergence-free space, Sec. 2.2).
 *   weight       -- W(r) = (1 - r/eps)_+^p  (Eq. kernel, read with the
 *                   positive part and power p = 4).
 *   solve        -- c = (P^T W P)^{-1} P^T W u  (Eqs. matrix-A, matrix-B,
 *                   vector-c), evaluated with the oracle's own Householder QR
 *                   of sqrt(W) P, so the weights for a functional row lambda
 *                   are w = sqrt(W) .* Q R^{-T} lambda^T  (Eq.
 *                   polynomial-approximation-derivative).
 *   Neumann      -- the constrained problem of Sec. 2.3 (Eqs.
 *                   neumann-optimization-*, neumann-saddle-point-system)
 *                   solved by eliminating the single constraint with a
 *                   reflector (null-space method).
 *
 * Floating point: compile with -ffp-contract=off so that every product and
 * sum is rounded separately (the squared distance must be reproducible).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_TOO_FEW (-3)

/* ------------------------------------------------------------------------ */
/* Neighbour search (Sec. 2.1: "particles within a distance eps of x_T")     */
/* ------------------------------------------------------------------------ */

/* Squared distance ((dx*dx + dy*dy) + dz*dz), dx = x_j - x_T, left to right. */
static double sq_dist(int dim, const double* x, int64_t n, int64_t t, int64_t j) {
  double d2 = 0.0;
  for (int c = 0; c < dim; ++c) {
    double dc = x[c * n + j] - x[c * n + t];
    double p = dc * dc;
    d2 = (c == 0) ? p : d2 + p;
  }
  return d2;
}

/* Half-space side s = n . (x_j - x_T), same evaluation order. */
static double hs_side(int dim, const double* x, int64_t n, int64_t t, int64_t j, const double* nrm) {
  double s = 0.0;
  for (int c = 0; c < dim; ++c) {
    double dc = x[c * n + j] - x[c * n + t];
    double p = nrm[c] * dc;
    s = (c == 0) ? p : s + p;
  }
  return s;
}

/* Candidate ordering: by squared distance, then by global index. */
static int cand_less(double da, int32_t ia, double db, int32_t ib) {
  return (da < db) || (da == db && ia < ib);
}

/* Insert (d2, j) into a list kept sorted ascending, capped at cap entries. */
static void top_insert(double* kd, int32_t* ki, int* cnt, int cap, double d2, int32_t j) {
  int c = *cnt;
  if (c == cap && !cand_less(d2, j, kd[c - 1], ki[c - 1])) return;
  int pos = (c < cap) ? c : cap - 1;
  while (pos > 0 && cand_less(d2, j, kd[pos - 1], ki[pos - 1])) {
    kd[pos] = kd[pos - 1];
    ki[pos] = ki[pos - 1];
    --pos;
  }
  kd[pos] = d2;
  ki[pos] = j;
  if (c < cap) *cnt = c + 1;
}

/*
 * k nearest neighbours by brute force.
 *   x        : SoA coordinates, x[c*n + i]
 *   tgt      : target particle indices (n_tgt)
 *   hs       : optional half-space normals, hs[t*dim + c]; a target whose
 *              normal is all zero (or hs == NULL) is unfiltered.  A filtered
 *              target keeps only j with n . (x_j - x_T) <= 0.
 *   out_idx  : n_tgt * k neighbour indices sorted by (d2, index)
 *   out_eps  : eps_factor * sqrt(d2 of the k-th neighbour)
 */
int orc_knn_brute(int dim, int64_t n, const double* x, int64_t n_tgt, const int32_t* tgt, int k,
                  double eps_factor, const double* hs, int32_t* out_idx, double* out_eps) {
  if (dim < 1 || dim > 3 || k < 1 || n < 1) return ORC_EINVAL;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int64_t q = 0; q < n_tgt; ++q) {
    double* kd = (double*)malloc(sizeof(double) * (size_t)k);
    int32_t* ki = out_idx + q * (int64_t)k;
    int cnt = 0;
    int64_t t = tgt[q];
    const double* nrm = hs ? hs + q * dim : NULL;
    int use_hs = 0;
    if (nrm)
      for (int c = 0; c < dim; ++c)
        if (nrm[c] != 0.0) use_hs = 1;
    for (int64_t j = 0; j < n; ++j) {
      if (use_hs && hs_side(dim, x, n, t, j, nrm) > 0.0) continue;
      top_insert(kd, ki, &cnt, k, sq_dist(dim, x, n, t, j), (int32_t)j);
    }
    if (cnt < k) {
      bad = 1;
      for (int i = cnt; i < k; ++i) ki[i] = -1;
      out_eps[q] = 0.0;
    } else {
      out_eps[q] = eps_factor * sqrt(kd[k - 1]);
    }
    free(kd);
  }
  return bad ? ORC_TOO_FEW : ORC_OK;
}

/* A plain uniform grid over the bounding box (the oracle's own, CPU only). */
typedef struct {
  int dim;
  int64_t nc[3];
  double lo[3], h;
  int64_t* start; /* cell -> first slot, size ncell+1 */
  int32_t* items; /* slots -> particle index */
} orc_grid;

static int64_t grid_coord(const orc_grid* g, int c, double v) {
  int64_t q = (int64_t)floor((v - g->lo[c]) / g->h);
  if (q < 0) q = 0;
  if (q >= g->nc[c]) q = g->nc[c] - 1;
  return q;
}

static int grid_build(orc_grid* g, int dim, int64_t n, const double* x, double h) {
  g->dim = dim;
  g->h = h;
  int64_t ncell = 1;
  for (int c = 0; c < 3; ++c) {
    g->nc[c] = 1;
    g->lo[c] = 0.0;
  }
  for (int c = 0; c < dim; ++c) {
    double lo = x[c * n], hi = x[c * n];
    for (int64_t i = 1; i < n; ++i) {
      double v = x[c * n + i];
      if (v < lo) lo = v;
      if (v > hi) hi = v;
    }
    g->lo[c] = lo;
    g->nc[c] = (int64_t)floor((hi - lo) / h) + 1;
    ncell *= g->nc[c];
  }
  g->start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  g->items = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* cell_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!g->start || !g->items || !cell_of) return ORC_ENOMEM;
  for (int64_t i = 0; i < n; ++i) {
    int64_t cell = 0;
    for (int c = dim - 1; c >= 0; --c) cell = cell * g->nc[c] + grid_coord(g, c, x[c * n + i]);
    cell_of[i] = cell;
    g->start[cell + 1]++;
  }
  for (int64_t cidx = 0; cidx < ncell; ++cidx) g->start[cidx + 1] += g->start[cidx];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
  memcpy(fill, g->start, sizeof(int64_t) * (size_t)ncell);
  for (int64_t i = 0; i < n; ++i) g->items[fill[cell_of[i]]++] = (int32_t)i;
  free(fill);
  free(cell_of);
  return ORC_OK;
}

static void grid_free(orc_grid* g) {
  free(g->start);
  free(g->items);
}

/*
 * Visit every particle in the cells that overlap the box [x_T - R, x_T + R]
 * and keep those with d2 < R*R (after the optional half-space filter) in a
 * sorted list capped at cap.  Returns how many particles passed the filter
 * (which may exceed cap).
 */
static int64_t grid_gather(const orc_grid* g, const double* x, int64_t n, int64_t t, double R,
                           const double* nrm, int use_hs, double* kd, int32_t* ki, int* cnt, int cap) {
  int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int c = 0; c < g->dim; ++c) {
    lo[c] = grid_coord(g, c, x[c * n + t] - R);
    hi[c] = grid_coord(g, c, x[c * n + t] + R);
  }
  double R2 = R * R;
  int64_t passed = 0;
  *cnt = 0;
  for (int64_t cz = lo[2]; cz <= hi[2]; ++cz)
    for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
      for (int64_t cx = lo[0]; cx <= hi[0]; ++cx) {
        int64_t cell = (cz * g->nc[1] + cy) * g->nc[0] + cx;
        for (int64_t s = g->start[cell]; s < g->start[cell + 1]; ++s) {
          int32_t j = g->items[s];
          if (use_hs && hs_side(g->dim, x, n, t, j, nrm) > 0.0) continue;
          double d2 = sq_dist(g->dim, x, n, t, j);
          if (!(d2 < R2)) continue;
          ++passed;
          top_insert(kd, ki, cnt, cap, d2, j);
        }
      }
  return passed;
}

/*
 * k nearest neighbours through the grid.  For a trial radius R it collects
 * all particles with d2 < R^2; if at least k pass, the k nearest overall are
 * the k nearest of those (any other particle is at distance >= R).  Otherwise
 * R doubles.  Same outputs as orc_knn_brute.
 */
int orc_knn_grid(int dim, int64_t n, const double* x, int64_t n_tgt, const int32_t* tgt, int k, double eps_factor,
                 const double* hs, double cell_h, double r0, int32_t* out_idx, double* out_eps) {
  if (dim < 1 || dim > 3 || k < 1 || n < 1 || !(cell_h > 0.0) || !(r0 > 0.0)) return ORC_EINVAL;
  orc_grid g;
  if (grid_build(&g, dim, n, x, cell_h) != ORC_OK) return ORC_ENOMEM;
  double span = 0.0;
  for (int c = 0; c < dim; ++c) span += (double)g.nc[c] * cell_h;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int64_t q = 0; q < n_tgt; ++q) {
    double* kd = (double*)malloc(sizeof(double) * (size_t)k);
    int32_t* ki = out_idx + q * (int64_t)k;
    int64_t t = tgt[q];
    const double* nrm = hs ? hs + q * dim : NULL;
    int use_hs = 0;
    if (nrm)
      for (int c = 0; c < dim; ++c)
        if (nrm[c] != 0.0) use_hs = 1;
    double R = r0;
    int cnt = 0;
    for (;;) {
      int64_t passed = grid_gather(&g, x, n, t, R, nrm, use_hs, kd, ki, &cnt, k);
      if (passed >= k) break;
      if (R > 4.0 * span) break; /* the whole cloud is inside: too few */
      R *= 2.0;
    }
    if (cnt < k) {
      bad = 1;
      for (int i = cnt; i < k; ++i) ki[i] = -1;
      out_eps[q] = 0.0;
    } else {
      out_eps[q] = eps_factor * sqrt(kd[k - 1]);
    }
    free(kd);
  }
  grid_free(&g);
  return bad ? ORC_TOO_FEW : ORC_OK;
}

/*
 * Radius query: all j with d2 < eps^2 (strict: W vanishes at r = eps), after
 * the optional half-space filter, sorted by (d2, index), truncated at cap.
 * out_idx has n_tgt * cap slots; out_cnt[q] is the kept count.
 * Brute force over all particles.
 */
int orc_radius_brute(int dim, int64_t n, const double* x, int64_t n_tgt, const int32_t* tgt, const double* eps,
                     int cap, const double* hs, int32_t* out_idx, int32_t* out_cnt) {
  if (dim < 1 || dim > 3 || cap < 1) return ORC_EINVAL;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < n_tgt; ++q) {
    double* kd = (double*)malloc(sizeof(double) * (size_t)cap);
    int32_t* ki = out_idx + q * (int64_t)cap;
    int cnt = 0;
    int64_t t = tgt[q];
    const double* nrm = hs ? hs + q * dim : NULL;
    int use_hs = 0;
    if (nrm)
      for (int c = 0; c < dim; ++c)
        if (nrm[c] != 0.0) use_hs = 1;
    double e2 = eps[q] * eps[q];
    for (int64_t j = 0; j < n; ++j) {
      if (use_hs && hs_side(dim, x, n, t, j, nrm) > 0.0) continue;
      double d2 = sq_dist(dim, x, n, t, j);
      if (d2 < e2) top_insert(kd, ki, &cnt, cap, d2, (int32_t)j);
    }
    out_cnt[q] = cnt;
    for (int i = cnt; i < cap; ++i) ki[i] = -1;
    free(kd);
  }
  return ORC_OK;
}

/* Same as orc_radius_brute, through the grid. */
int orc_radius_grid(int dim, int64_t n, const double* x, int64_t n_tgt, const int32_t* tgt, const double* eps,
                    int cap, const double* hs, double cell_h, int32_t* out_idx, int32_t* out_cnt) {
  if (dim < 1 || dim > 3 || cap < 1 || !(cell_h > 0.0)) return ORC_EINVAL;
  orc_grid g;
  if (grid_build(&g, dim, n, x, cell_h) != ORC_OK) return ORC_ENOMEM;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < n_tgt; ++q) {
    double* kd = (double*)malloc(sizeof(double) * (size_t)cap);
    int32_t* ki = out_idx + q * (int64_t)cap;
    int cnt = 0;
    int64_t t = tgt[q];
    const double* nrm = hs ? hs + q * dim : NULL;
    int use_hs = 0;
    if (nrm)
      for (int c = 0; c < dim; ++c)
        if (nrm[c] != 0.0) use_hs = 1;
    /* d2 < eps*eps is the definition; R = eps makes grid_gather apply d2 < R*R. */
    grid_gather(&g, x, n, t, eps[q], nrm, use_hs, kd, ki, &cnt, cap);
    out_cnt[q] = cnt;
    for (int i = cnt; i < cap; ++i) ki[i] = -1;
    free(kd);
  }
  grid_free(&g);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Basis, weight, functionals                                                */
/* ------------------------------------------------------------------------ */

/*
 * A basis is a table of polynomial terms in the scaled offset
 * xi = (x - x_T) / eps.  Basis function i, component c is
 *     sum_{s in [off[i*nc + c], off[i*nc + c + 1])} coef[s] * xi^{expo[3s..3s+2]}.
 * The scalar Taylor basis of Eq. (basis-functions-3d) is one term per
 * function with coef 1/alpha!; a divergence-free basis (Sec. 2.2) has one to
 * two terms per component.
 */
typedef struct {
  int nb, nc;
  const int* off;
  const double* coef;
  const int* expo;
} orc_basis;

static double ipow(double v, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= v;
  return r;
}

static double eval_term_sum(const orc_basis* b, int i, int c, const double* xi) {
  double s = 0.0;
  for (int q = b->off[i * b->nc + c]; q < b->off[i * b->nc + c + 1]; ++q)
    s += b->coef[q] * ipow(xi[0], b->expo[3 * q]) * ipow(xi[1], b->expo[3 * q + 1]) * ipow(xi[2], b->expo[3 * q + 2]);
  return s;
}

static double factorial(int e) {
  double r = 1.0;
  for (int i = 2; i <= e; ++i) r *= i;
  return r;
}

/*
 * D^beta of basis function i, component c, at x = x_T, in physical
 * coordinates: d^beta/dx^beta (xi^gamma) at xi = 0 is gamma! eps^{-|beta|}
 * when beta == gamma and zero otherwise (Eq. polynomial-approximation-derivative
 * applied to the scaled monomials).
 */
static double deriv_at_target(const orc_basis* b, int i, int c, const int* beta, double eps) {
  double s = 0.0;
  for (int q = b->off[i * b->nc + c]; q < b->off[i * b->nc + c + 1]; ++q) {
    const int* g = b->expo + 3 * q;
    if (g[0] == beta[0] && g[1] == beta[1] && g[2] == beta[2])
      s += b->coef[q] * factorial(g[0]) * factorial(g[1]) * factorial(g[2]);
  }
  return s * ipow(1.0 / eps, beta[0] + beta[1] + beta[2]);
}

/*
 * A functional row is a list of terms (coef, component, beta):
 *     lambda(psi) = sum coef * D^beta psi_component (x_T).
 * lambda_i = lambda(psi_i) is the row the stencil reproduces.
 */
typedef struct {
  int nrows;
  const int* off;
  const double* coef;
  const int* comp;
  const int* beta;
} orc_functional;

static void functional_row(const orc_basis* b, const orc_functional* f, int r, double eps, double* lam) {
  for (int i = 0; i < b->nb; ++i) {
    double s = 0.0;
    for (int q = f->off[r]; q < f->off[r + 1]; ++q) s += f->coef[q] * deriv_at_target(b, i, f->comp[q], f->beta + 3 * q, eps);
    lam[i] = s;
  }
}

/* W(r) = (1 - r/eps)^p for r < eps, else 0 (Eq. kernel). Returns sqrt(W). */
static double sqrt_weight(double r, double eps, double p) {
  if (!(r < eps)) return 0.0;
  return pow(1.0 - r / eps, 0.5 * p);
}

/* ------------------------------------------------------------------------ */
/* Householder QR and the weighted least-squares weights                     */
/* ------------------------------------------------------------------------ */

/*
 * In-place Householder QR of the column-major M x n matrix A (ld = M).
 * On return the upper triangle holds R; column k below the diagonal holds the
 * reflector v_k (v_k[k] = 1 implied) and tau[k] its scale, so that
 * H_k = I - tau_k v_k v_k^T and A = H_0 H_1 ... H_{n-1} [R; 0].
 */
static void householder_qr(int M, int n, double* A, double* tau) {
  for (int k = 0; k < n; ++k) {
    double* a = A + (size_t)k * M;
    double sigma = 0.0;
    for (int i = k + 1; i < M; ++i) sigma += a[i] * a[i];
    double alpha = a[k];
    if (sigma == 0.0) {
      tau[k] = 0.0; /* already upper triangular in this column */
      continue;
    }
    double norm = sqrt(alpha * alpha + sigma);
    double beta = (alpha >= 0.0) ? -norm : norm;
    double scale = 1.0 / (alpha - beta);
    for (int i = k + 1; i < M; ++i) a[i] *= scale;
    tau[k] = (beta - alpha) / beta;
    a[k] = beta;
    for (int j = k + 1; j < n; ++j) {
      double* aj = A + (size_t)j * M;
      double dot = aj[k];
      for (int i = k + 1; i < M; ++i) dot += a[i] * aj[i];
      dot *= tau[k];
      aj[k] -= dot;
      for (int i = k + 1; i < M; ++i) aj[i] -= dot * a[i];
    }
  }
}

/* z <- H_0 H_1 ... H_{n-1} z  (apply Q to an M-vector). */
static void apply_q(int M, int n, const double* A, const double* tau, double* z) {
  for (int k = n - 1; k >= 0; --k) {
    if (tau[k] == 0.0) continue;
    const double* a = A + (size_t)k * M;
    double dot = z[k];
    for (int i = k + 1; i < M; ++i) dot += a[i] * z[i];
    dot *= tau[k];
    z[k] -= dot;
    for (int i = k + 1; i < M; ++i) z[i] -= dot * a[i];
  }
}

/* Solve R^T y = lam by forward substitution (R upper triangular, in A). */
static void solve_rt(int M, int n, const double* A, const double* lam, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = lam[i];
    for (int p = 0; p < i; ++p) s -= A[(size_t)i * M + p] * y[p];
    y[i] = s / A[(size_t)i * M + i];
  }
}

/*
 * One target.  Rows of the least-squares matrix are (neighbour j, component
 * c) in the order j*nc + c (Sec. 2.2 repeats W_j for every component).
 *
 *   x, n       : SoA cloud
 *   t          : target index; nbr/k its neighbours; eps its support
 *   wpow       : weight exponent p
 *   nrm        : NULL, or the outward unit normal for a Neumann target
 *   out_w      : nrows * (k*nc) weights, row-major
 *   out_beta   : nrows values (coefficient of h; zero without Neumann)
 *   out_diag   : [max|r_ii|, min|r_ii|] of the triangular factor
 */
int orc_stencil_one(int dim, int64_t n, const double* x, int64_t t, const int32_t* nbr, int k, double eps, double wpow,
                    const orc_basis* b, const orc_functional* f, const double* nrm, double* out_w, double* out_beta,
                    double* out_diag) {
  const int nc = b->nc;
  const int M = k * nc;
  int nb = b->nb;
  double* P = (double*)malloc(sizeof(double) * (size_t)M * nb); /* column-major */
  double* sw = (double*)malloc(sizeof(double) * (size_t)M);
  double* lam = (double*)malloc(sizeof(double) * (size_t)nb);
  double* tau = (double*)malloc(sizeof(double) * (size_t)nb);
  double* y = (double*)malloc(sizeof(double) * (size_t)nb);
  double* z = (double*)malloc(sizeof(double) * (size_t)M);
  double* pt = (double*)malloc(sizeof(double) * (size_t)M); /* p~_1 column (Neumann) */
  if (!P || !sw || !lam || !tau || !y || !z || !pt) return ORC_ENOMEM;

  /* sqrt(W) P, Eqs. matrix-P and matrix-W */
  for (int j = 0; j < k; ++j) {
    double xi[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < dim; ++c) xi[c] = (x[c * n + nbr[j]] - x[c * n + t]) / eps;
    double r = sqrt(sq_dist(dim, x, n, t, nbr[j]));
    double s = sqrt_weight(r, eps, wpow);
    for (int c = 0; c < nc; ++c) {
      sw[j * nc + c] = s;
      for (int i = 0; i < nb; ++i) P[(size_t)i * M + j * nc + c] = s * eval_term_sum(b, i, c, xi);
    }
  }

  /* Neumann (Sec. 2.3): F = grad p(x_T)^T n; c = H_F [c1; z], F^T c = rho c1. */
  int piv = -1;
  double rho = 0.0;
  double* vf = NULL;
  double vfvf = 0.0;
  if (nrm) {
    vf = (double*)malloc(sizeof(double) * (size_t)nb);
    double fn = 0.0;
    for (int i = 0; i < nb; ++i) {
      double s = 0.0;
      for (int c = 0; c < dim; ++c) {
        int beta[3] = {0, 0, 0};
        beta[c] = 1;
        s += nrm[c] * deriv_at_target(b, i, 0, beta, eps);
      }
      vf[i] = s;
      fn += s * s;
      if (piv < 0 || fabs(s) > fabs(vf[piv])) piv = i;
    }
    fn = sqrt(fn);
    if (!(fn > 0.0)) return ORC_EINVAL;
    rho = (vf[piv] >= 0.0) ? -fn : fn;
    vf[piv] -= rho; /* v = F - rho e_piv; H_F = I - 2 v v^T / (v^T v) */
    for (int i = 0; i < nb; ++i) vfvf += vf[i] * vf[i];
    /* P <- P H_F, row by row */
    for (int r = 0; r < M; ++r) {
      double d = 0.0;
      for (int i = 0; i < nb; ++i) d += P[(size_t)i * M + r] * vf[i];
      d *= 2.0 / vfvf;
      for (int i = 0; i < nb; ++i) P[(size_t)i * M + r] -= d * vf[i];
    }
    /* keep column piv (p~_1, still scaled by sqrt W) and drop it from P */
    for (int r = 0; r < M; ++r) pt[r] = P[(size_t)piv * M + r];
    for (int i = piv; i < nb - 1; ++i) memcpy(P + (size_t)i * M, P + (size_t)(i + 1) * M, sizeof(double) * (size_t)M);
    nb -= 1;
  }

  householder_qr(M, nb, P, tau);
  double rmax = 0.0, rmin = INFINITY;
  for (int i = 0; i < nb; ++i) {
    double r = fabs(P[(size_t)i * M + i]);
    if (r > rmax) rmax = r;
    if (r < rmin) rmin = r;
  }
  out_diag[0] = rmax;
  out_diag[1] = rmin;

  double* lamfull = (double*)malloc(sizeof(double) * (size_t)b->nb);
  for (int r = 0; r < f->nrows; ++r) {
    functional_row(b, f, r, eps, lamfull);
    double lam1 = 0.0;
    if (nrm) { /* lambda~ = lambda H_F; split off component piv */
      double d = 0.0;
      for (int i = 0; i < b->nb; ++i) d += lamfull[i] * vf[i];
      d *= 2.0 / vfvf;
      for (int i = 0; i < b->nb; ++i) lamfull[i] -= d * vf[i];
      lam1 = lamfull[piv];
      int q = 0;
      for (int i = 0; i < b->nb; ++i)
        if (i != piv) lam[q++] = lamfull[i];
    } else {
      memcpy(lam, lamfull, sizeof(double) * (size_t)nb);
    }
    solve_rt(M, nb, P, lam, y);
    for (int i = 0; i < M; ++i) z[i] = (i < nb) ? y[i] : 0.0;
    apply_q(M, nb, P, tau, z);
    double* w = out_w + (size_t)r * M;
    for (int i = 0; i < M; ++i) w[i] = sw[i] * z[i];
    if (out_beta) {
      if (nrm) {
        /* beta = (lambda~_1 - w^T p~_1) / rho, p~_1 unscaled = pt / sqrt(W) */
        double s = 0.0;
        for (int i = 0; i < M; ++i) s += z[i] * pt[i]; /* (sqrtW z)^T (pt/sqrtW) */
        out_beta[r] = (lam1 - s) / rho;
      } else {
        out_beta[r] = 0.0;
      }
    }
  }
  free(lamfull);
  free(vf);
  free(P);
  free(sw);
  free(lam);
  free(tau);
  free(y);
  free(z);
  free(pt);
  return ORC_OK;
}

/*
 * Many targets (OpenMP over targets).  Neighbour lists are CSR: target q uses
 * nbr_idx[nbr_off[q] .. nbr_off[q+1]).  Weights for target q start at
 * out_w + w_off[q] and hold nrows * (k_q * nc) values.  nrm_all is NULL or
 * n_tgt*dim normals; a target with bflag[q] != 0 takes the Neumann
 * constraint with its normal.
 */
int orc_stencils(int dim, int64_t n, const double* x, int64_t n_tgt, const int32_t* tgt, const int64_t* nbr_off,
                 const int32_t* nbr_idx, const double* eps, double wpow, int nb, int nc, const int* b_off,
                 const double* b_coef, const int* b_expo, int nrows, const int* f_off, const double* f_coef,
                 const int* f_comp, const int* f_beta, const uint8_t* bflag, const double* nrm_all,
                 const int64_t* w_off, double* out_w, double* out_beta, double* out_diag) {
  orc_basis b = {nb, nc, b_off, b_coef, b_expo};
  orc_functional f = {nrows, f_off, f_coef, f_comp, f_beta};
  int err = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : err)
  for (int64_t q = 0; q < n_tgt; ++q) {
    int k = (int)(nbr_off[q + 1] - nbr_off[q]);
    const double* nrm = (bflag && bflag[q]) ? nrm_all + q * dim : NULL;
    int rc = orc_stencil_one(dim, n, x, tgt[q], nbr_idx + nbr_off[q], k, eps[q], wpow, &b, &f, nrm, out_w + w_off[q],
                             out_beta ? out_beta + q * nrows : NULL, out_diag + 2 * q);
    if (rc != ORC_OK) err |= 1;
  }
  return err ? ORC_EINVAL : ORC_OK;
}

/* Exposed for tests: Householder QR of a column-major matrix and Q application. */
void orc_qr(int M, int n, double* A, double* tau) { householder_qr(M, n, A, tau); }
void orc_apply_q(int M, int n, const double* A, const double* tau, double* z) { apply_q(M, n, A, tau, z); }
