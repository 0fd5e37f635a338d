/*
 * CPU ORACLE for smoothed-aggregation AMG with the classical and the
 * material-aware strength-of-connection measures.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, serial, FP64 C, written to be checked by
 * eye against the paper's definitions.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load this library; the CUDA
 * library never includes, links or calls it, and it shares no code, header
 * or table with the CUDA sources.
 *
 * Build: gcc -O2 -ffp-contract=off (no fused multiply-add, so every
 * floating-point expression below is evaluated exactly as written).
 *
 * Paper sections followed (arXiv 2602.05686):
 *   Sec. 2            multigrid V-cycle (Algorithm 1), Galerkin product,
 *                     aggregates as a disjoint cover, tentative prolongator
 *   Sec. 2.1          strength-of-connection S, dropping criterion C,
 *                     pointwise dropping C^pw, classical S^sa = D^-1/2 A D^-1/2,
 *                     distance Laplacian L_d and S^dlap
 *   Sec. 2.2          prolongator smoothing P = (I - w D^-1 A) P^,
 *                     w = (4/3)/lambda, filtered matrix A_F with lumped
 *                     diagonal, 1-norm diagonal D~_F
 *   Sec. 3            material distance d_sigma, S^dlap_sigma, Clement
 *                     averaging of elementwise tensors, coarse coordinate and
 *                     tensor transfer by aggregate means (Eq. auxiliary_transfer)
 *   Sec. 4            CG preconditioned by the V-cycle, residual reduced by
 *                     1e8, Chebyshev degree 2 smoothing, direct coarse solve,
 *                     coarsening to <= 5000 unknowns
 *
 * Readings where the paper is silent or garbled (listed again in the design
 * notes):
 *   - d_sigma(x,y) = max(d~(x,y), d~(y,x)): the printed max has two identical
 *     arguments; the low/high argument of Sec. 3 needs both nodes' tensors.
 *   - "A_ij != 0" in L_d means a stored entry of the structural pattern.
 *   - cut-drop: no gap in a row keeps the whole row; row decisions are
 *     symmetrised by keeping an edge only when both rows keep it.
 *   - pointwise dropping keeps |S_ij| >= theta; the diagonal is always kept
 *     and never enters the filtered graph; Dirichlet nodes never enter it.
 *   - the squared forms a_ij^2 >= theta^2 |a_ii a_jj| and
 *     w_ij^2 >= theta^2 D_i D_j are used (no square roots).
 *   - aggregation: greedy distance-2 maximal independent set in descending
 *     hash-priority order, root + its filtered neighbours (phase 1), leftover
 *     nodes join the phase-1 aggregate they share most filtered edges with,
 *     ties to the smallest aggregate id (phase 2).
 *   - w uses rho(D~_F^-1 A_F) from 10 power steps on D~^-1/2 A_F D~^-1/2
 *     started from a hash-uniform vector; lambda = ||M v|| / ||v|| at the
 *     last step (a spectral-radius estimate that stays positive when the
 *     lumped filtered matrix is indefinite).
 *   - a row of A_F with every off-diagonal dropped (lumped row sum ~ 0) is
 *     not smoothed: D~_i^-1 := 0 when D~_i <= 1e-12 sum_j |a_ij|.
 *   - Chebyshev: lambda_max = 1.1 x (10 power steps on D^-1/2 A D^-1/2),
 *     lambda_min = lambda_max / 30, D = diag(A).
 *   - coarse operators are stored exactly symmetric: the lower triangle of
 *     R (A P) takes the value of the mirrored upper-triangle entry.
 *   - stop: n_l <= max_coarse or max_levels reached; stagnation
 *     n_{l+1} > 0.9 n_l makes level l the coarsest; a coarsest level above
 *     16384 unknowns is an error.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { OR_OK = 0, OR_ERR_INVALID_ARG = -1, OR_ERR_OOM = -2, OR_ERR_NOT_SPD = -4,
       OR_ERR_STAGNATION = -5, OR_ERR_NO_CONVERGENCE = -6, OR_ERR_BREAKDOWN = -7 };

typedef struct {
  int64_t nrows, ncols;
  int64_t* rp;
  int32_t* ci;
  double* v;
} csr_t;

static csr_t csr_new(int64_t nrows, int64_t ncols, int64_t nnz) {
  csr_t m;
  m.nrows = nrows;
  m.ncols = ncols;
  m.rp = (int64_t*)calloc((size_t)nrows + 1, sizeof(int64_t));
  m.ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  m.v = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  return m;
}

static void csr_del(csr_t* m) {
  free(m->rp); free(m->ci); free(m->v);
  m->rp = NULL; m->ci = NULL; m->v = NULL;
}

static int64_t csr_nnz(const csr_t* m) { return m->rp[m->nrows]; }

/* ------------------------------------------------------------------------ */
/* counter-based hashing: MurmurHash3 32-bit finaliser (Appleby, public
 * domain), used for the MIS-2 priorities and the power-method start vectors */
/* ------------------------------------------------------------------------ */
static uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

/* MIS-2 priority of node i on level l (0 = finest): hash in the high word,
 * index in the low word, so keys are distinct. */
uint64_t or_mis_key(int64_t i, int level, uint32_t seed) {
  uint32_t h = fmix32((uint32_t)i ^ (0x9E3779B9u * (uint32_t)(level + 1)) ^ seed);
  return ((uint64_t)h << 32) | (uint64_t)(uint32_t)i;
}

/* entry i of a hash-uniform start vector in [-1, 1) */
double or_start_value(int64_t i, uint32_t tag, uint32_t seed) {
  uint32_t h = fmix32((uint32_t)i ^ (0x7F4A7C15u * tag) ^ (seed * 0x2545F491u));
  double u = (double)h * (1.0 / 4294967296.0);
  return 2.0 * u - 1.0;
}

/* ------------------------------------------------------------------------ */
/* a1. Dirichlet detection (Sec. 3, Fig. 4 caption: Dirichlet nodes are
 * isolated in the filtered graph): row i is Dirichlet iff every stored
 * off-diagonal value is exactly zero. */
/* ------------------------------------------------------------------------ */
void or_dirichlet(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, uint8_t* dir) {
  for (int64_t i = 0; i < n; ++i) {
    int d = 1;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] != i && v[p] != 0.0) d = 0;
    dir[i] = (uint8_t)d;
  }
}

/* ------------------------------------------------------------------------ */
/* a2. Nodal tensors from elementwise-constant tensors (Sec. 3, Clement
 * interpolant): sigma_i = sum_{e contains i} |e| sigma_e / sum |e|, summed in
 * ascending element index. */
/* ------------------------------------------------------------------------ */
int or_nodal_from_elements(int dim, int64_t n, int64_t ne, int npe, const int32_t* en,
                           const double* meas, const double* et, double* sigma) {
  const int kp = dim == 3 ? 6 : 3;
  double* den = (double*)calloc((size_t)n, sizeof(double));
  if (!den) return OR_ERR_OOM;
  memset(sigma, 0, sizeof(double) * (size_t)n * kp);
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < npe; ++a) {
      int64_t i = en[e * npe + a];
      for (int c = 0; c < kp; ++c) sigma[i * kp + c] += meas[e] * et[e * kp + c];
      den[i] += meas[e];
    }
  int st = OR_OK;
  for (int64_t i = 0; i < n; ++i) {
    if (den[i] == 0.0) { st = OR_ERR_INVALID_ARG; continue; }
    for (int c = 0; c < kp; ++c) sigma[i * kp + c] = sigma[i * kp + c] / den[i];
  }
  free(den);
  return st;
}

/* inverse of a packed symmetric tensor by adjugate / determinant
 * 2D (xx,yy,xy), 3D (xx,yy,zz,xy,xz,yz) */
void or_invert_tensors(int dim, int64_t n, const double* s, double* si) {
  for (int64_t i = 0; i < n; ++i) {
    if (dim == 2) {
      const double* t = s + 3 * i;
      double det = t[0] * t[1] - t[2] * t[2];
      si[3 * i + 0] = t[1] / det;
      si[3 * i + 1] = t[0] / det;
      si[3 * i + 2] = -t[2] / det;
    } else {
      const double* t = s + 6 * i;
      double a = t[0], b = t[1], c = t[2], d = t[3], e = t[4], f = t[5];
      double c00 = b * c - f * f;
      double c11 = a * c - e * e;
      double c22 = a * b - d * d;
      double c01 = e * f - d * c;
      double c02 = d * f - b * e;
      double c12 = d * e - a * f;
      double det = a * c00 + d * c01 + e * c02;
      si[6 * i + 0] = c00 / det;
      si[6 * i + 1] = c11 / det;
      si[6 * i + 2] = c22 / det;
      si[6 * i + 3] = c01 / det;
      si[6 * i + 4] = c02 / det;
      si[6 * i + 5] = c12 / det;
    }
  }
}

static double diag_of(const int64_t* rp, const int32_t* ci, const double* v, int64_t i) {
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) return v[p];
  return 0.0;
}

/* ------------------------------------------------------------------------ */
/* a3. Classical measure with pointwise dropping (Sec. 2.1):
 * |a_ij| / sqrt(|a_ii| |a_jj|) >= theta, evaluated as
 * a_ij*a_ij >= (theta*theta) * |a_ii*a_jj|.  Diagonal kept. */
/* ------------------------------------------------------------------------ */
void or_strength_classical(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                           const uint8_t* dir, double theta, uint8_t* keep) {
  double* dg = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) dg[i] = diag_of(rp, ci, v, i);
  const double t2 = theta * theta;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (j == i) { keep[p] = 1; continue; }
      if ((dir && (dir[i] || dir[j]))) { keep[p] = 0; continue; }
      double a = v[p];
      keep[p] = (uint8_t)(a * a >= t2 * fabs(dg[i] * dg[j]));
    }
  free(dg);
}

/* squared material distance d~(x_i, x_j)^2 = d^T sigma_i^-1 d, d = x_i - x_j:
 * t = sigma_i^-1 d, then d . t, each a running sum of fused multiply-adds
 * (one rounding per term) in index order.  The value is even in d bit for
 * bit (negating d negates t exactly), so d~ is the same from either end. */
static double quad_form(int dim, const double* si, const double* d) {
  if (dim == 2) {
    const double t0 = fma(si[2], d[1], si[0] * d[0]);
    const double t1 = fma(si[1], d[1], si[2] * d[0]);
    return fma(d[1], t1, d[0] * t0);
  }
  const double t0 = fma(si[4], d[2], fma(si[3], d[1], si[0] * d[0]));
  const double t1 = fma(si[5], d[2], fma(si[1], d[1], si[3] * d[0]));
  const double t2 = fma(si[2], d[2], fma(si[5], d[1], si[4] * d[0]));
  return fma(d[2], t2, fma(d[1], t1, d[0] * t0));
}

/* ------------------------------------------------------------------------ */
/* a4. Material-aware distance Laplacian with pointwise dropping (Sec. 2.1
 * distance Laplacian; Sec. 3 material distance):
 *   w_ij = -(L_sigma)_ij = 1 / d_sigma(x_i,x_j)^2
 *        = 1 / max(d~(x_i,x_j)^2, d~(x_j,x_i)^2)      for stored j != i
 *   D_i  = (L_sigma)_ii = sum_{j != i} w_ij  (ascending column order)
 *   keep ⇔ |S_ij| = w_ij / sqrt(D_i D_j) >= theta
 *        ⇔ w_ij*w_ij >= (theta*theta) * (D_i*D_j).
 * w[p] is written for off-diagonal entries (0 on the diagonal), D[i] per row.
 * With sigma == I this is the plain distance Laplacian S^dlap. */
/* ------------------------------------------------------------------------ */
void or_strength_material(int dim, int64_t n, const int64_t* rp, const int32_t* ci,
                          const uint8_t* dir, const double* x, const double* sinv, double theta,
                          double* w, double* D, uint8_t* keep) {
  const int kp = dim == 3 ? 6 : 3;
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (j == i) { w[p] = 0.0; continue; }
      double d[3];
      for (int c = 0; c < dim; ++c) d[c] = x[i * dim + c] - x[j * dim + c];
      double qij = quad_form(dim, sinv + i * kp, d);
      double qji = quad_form(dim, sinv + j * kp, d);
      double m = qij > qji ? qij : qji;
      w[p] = 1.0 / m;
      acc += w[p];
    }
    D[i] = acc;
  }
  const double t2 = theta * theta;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (j == i) { keep[p] = 1; continue; }
      if (dir && (dir[i] || dir[j])) { keep[p] = 0; continue; }
      keep[p] = (uint8_t)(w[p] * w[p] >= t2 * (D[i] * D[j]));
    }
}

/* ------------------------------------------------------------------------ */
/* Cut-drop criterion (Sec. 2.1, Eq. C^cut-drop) on squared strengths s2[p]
 * (off-diagonal entries; the diagonal and Dirichlet-incident entries are
 * ignored and never kept).  Per row: order the values descending,
 * s_1 >= s_2 >= ... >= s_m; k is the smallest index with
 * theta * s_k >= s_{k+1} (in squares: theta^2 s2_k >= s2_{k+1}); keep the
 * entries with s >= s_k.  Readings: if no such k exists every entry is kept;
 * the row-wise decisions are symmetrised by keeping an edge only when both
 * of its rows keep it (the filtered graph must be symmetric). */
/* ------------------------------------------------------------------------ */
static int cmp_dbl_desc(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x < y) - (x > y);
}

void or_cut_drop(int64_t n, const int64_t* rp, const int32_t* ci, const uint8_t* dir, const double* s2,
                 double theta, uint8_t* keep) {
  const double t2 = theta * theta;
  int64_t maxrow = 0;
  for (int64_t i = 0; i < n; ++i) if (rp[i + 1] - rp[i] > maxrow) maxrow = rp[i + 1] - rp[i];
  double* vals = (double*)malloc(sizeof(double) * (size_t)(maxrow > 0 ? maxrow : 1));
  uint8_t* rowkeep = (uint8_t*)calloc((size_t)(rp[n] > 0 ? rp[n] : 1), 1);
  for (int64_t i = 0; i < n; ++i) {
    int64_t m = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (j == i || (dir && (dir[i] || dir[j]))) continue;
      vals[m++] = s2[p];
    }
    if (m == 0) continue;
    qsort(vals, (size_t)m, sizeof(double), cmp_dbl_desc);
    double thr = vals[m - 1];
    for (int64_t k = 0; k + 1 < m; ++k)
      if (t2 * vals[k] >= vals[k + 1]) { thr = vals[k]; break; }
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (j == i || (dir && (dir[i] || dir[j]))) continue;
      rowkeep[p] = (uint8_t)(s2[p] >= thr);
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (j == i) { keep[p] = 1; continue; }
      int64_t q = -1;
      for (int64_t r = rp[j]; r < rp[j + 1]; ++r) if (ci[r] == i) { q = r; break; }
      keep[p] = (uint8_t)(rowkeep[p] && q >= 0 && rowkeep[q]);
    }
  free(vals);
  free(rowkeep);
}

/* squared strengths for cut-drop: classical a_ij^2 / |a_ii a_jj|, material
 * (or distance) w_ij^2 / (D_i D_j) */
void or_strength2_classical(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double* s2) {
  double* dg = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) dg[i] = diag_of(rp, ci, v, i);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      s2[p] = (j == i) ? 0.0 : (v[p] * v[p]) / fabs(dg[i] * dg[j]);
    }
  free(dg);
}

void or_strength2_material(int64_t n, const int64_t* rp, const int32_t* ci, const double* w, const double* D,
                           double* s2) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      s2[p] = (j == i) ? 0.0 : (w[p] * w[p]) / (D[i] * D[j]);
    }
}

/* ------------------------------------------------------------------------ */
/* a5. Filtered graph G_C (Sec. 2.1): kept off-diagonal entries between
 * non-Dirichlet nodes; returns nnz(G_C); gc_ci must hold nnz(A) entries. */
/* ------------------------------------------------------------------------ */
int64_t or_filtered_graph(int64_t n, const int64_t* rp, const int32_t* ci, const uint8_t* keep,
                          const uint8_t* dir, int64_t* gc_rp, int32_t* gc_ci) {
  int64_t w = 0;
  gc_rp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(dir && dir[i]))
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t j = ci[p];
        if (j != i && keep[p] && !(dir && dir[j])) gc_ci[w++] = (int32_t)j;
      }
    gc_rp[i + 1] = w;
  }
  return w;
}

/* ------------------------------------------------------------------------ */
/* a6. Distance-2 maximal independent set, greedy definition: visit the
 * non-Dirichlet nodes in descending key order; select a node iff no selected
 * node lies within G_C-distance <= 2.  (The paper's "simplest aggregation",
 * Sec. 2: a node that does not neighbour any existing aggregate starts one.) */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; int64_t i; } keyed_t;

static int cmp_key_desc(const void* a, const void* b) {
  uint64_t ka = ((const keyed_t*)a)->key, kb = ((const keyed_t*)b)->key;
  return ka < kb ? 1 : (ka > kb ? -1 : 0);
}

void or_mis2(int64_t n, const int64_t* gc_rp, const int32_t* gc_ci, const uint8_t* dir,
             int level, uint32_t seed, uint8_t* root) {
  keyed_t* order = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(n > 0 ? n : 1));
  uint8_t* blocked = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    root[i] = 0;
    if (dir && dir[i]) continue;
    order[m].key = or_mis_key(i, level, seed);
    order[m].i = i;
    ++m;
  }
  qsort(order, (size_t)m, sizeof(keyed_t), cmp_key_desc);
  for (int64_t t = 0; t < m; ++t) {
    int64_t i = order[t].i;
    if (blocked[i]) continue;
    root[i] = 1;
    blocked[i] = 1;
    for (int64_t p = gc_rp[i]; p < gc_rp[i + 1]; ++p) {
      int64_t j = gc_ci[p];
      blocked[j] = 1;
      for (int64_t q = gc_rp[j]; q < gc_rp[j + 1]; ++q) blocked[gc_ci[q]] = 1;
    }
  }
  free(order);
  free(blocked);
}

/* ------------------------------------------------------------------------ */
/* a7. Aggregates from the MIS-2 roots (Sec. 2: aggregates form a disjoint
 * cover of the non-Dirichlet nodes):
 *   id(root) = rank of the root among roots in ascending index;
 *   phase 1: root and its G_C neighbours get id(root);
 *   phase 2: every other non-Dirichlet node joins the phase-1 aggregate with
 *            which it shares the most G_C edges, ties to the smallest id.
 * Returns the number of aggregates; agg[i] = -1 for Dirichlet nodes. */
/* ------------------------------------------------------------------------ */
int64_t or_aggregate(int64_t n, const int64_t* gc_rp, const int32_t* gc_ci, const uint8_t* dir,
                     const uint8_t* root, int32_t* agg) {
  int64_t nc = 0;
  int32_t* p1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) p1[i] = -1;
  for (int64_t i = 0; i < n; ++i)
    if (root[i]) {
      p1[i] = (int32_t)nc;
      for (int64_t p = gc_rp[i]; p < gc_rp[i + 1]; ++p) p1[gc_ci[p]] = (int32_t)nc;
      ++nc;
    }
  for (int64_t i = 0; i < n; ++i) {
    agg[i] = p1[i];
    if (p1[i] >= 0 || (dir && dir[i])) continue;
    /* phase 2: count edges to each adjacent phase-1 aggregate */
    int32_t best = -1;
    int64_t bestc = 0;
    for (int64_t p = gc_rp[i]; p < gc_rp[i + 1]; ++p) {
      int32_t a = p1[gc_ci[p]];
      if (a < 0) continue;
      int64_t c = 0;
      for (int64_t q = gc_rp[i]; q < gc_rp[i + 1]; ++q)
        if (p1[gc_ci[q]] == a) ++c;
      if (c > bestc || (c == bestc && a < best)) { best = a; bestc = c; }
    }
    agg[i] = best; /* -1 would mean the MIS-2 was not maximal */
  }
  free(p1);
  return nc;
}

/* a8. Tentative prolongator on the constant near-nullspace (Sec. 2):
 * P^_{i,agg(i)} = 1; Dirichlet rows are empty. */
csr_t or_tentative(int64_t n, int64_t nc, const int32_t* agg) {
  int64_t nnz = 0;
  for (int64_t i = 0; i < n; ++i) nnz += agg[i] >= 0;
  csr_t P = csr_new(n, nc, nnz);
  int64_t w = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) { P.ci[w] = agg[i]; P.v[w] = 1.0; ++w; }
    P.rp[i + 1] = w;
  }
  return P;
}

/* a9. Coarse coordinates and tensors (Sec. 3, Eq. auxiliary_transfer): means
 * over the aggregate's members, summed in ascending fine index. */
void or_coarse_aux(int dim, int64_t n, int64_t nc, const int32_t* agg, const double* x,
                   const double* sigma, double* xc, double* sc) {
  const int kp = dim == 3 ? 6 : 3;
  double* cnt = (double*)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
  memset(xc, 0, sizeof(double) * (size_t)nc * dim);
  memset(sc, 0, sizeof(double) * (size_t)nc * kp);
  for (int64_t i = 0; i < n; ++i) {
    int32_t a = agg[i];
    if (a < 0) continue;
    for (int c = 0; c < dim; ++c) xc[a * dim + c] += x[i * dim + c];
    for (int c = 0; c < kp; ++c) sc[a * kp + c] += sigma[i * kp + c];
    cnt[a] += 1.0;
  }
  for (int64_t a = 0; a < nc; ++a) {
    for (int c = 0; c < dim; ++c) xc[a * dim + c] = xc[a * dim + c] / cnt[a];
    for (int c = 0; c < kp; ++c) sc[a * kp + c] = sc[a * kp + c] / cnt[a];
  }
  free(cnt);
}

/* ------------------------------------------------------------------------ */
/* a10. Filtered matrix and 1-norm diagonal (Sec. 2.2, Eqs. filtered_matrix
 * and 1_norm_diagonal): kept off-diagonals keep a_ij, dropped ones become 0
 * and are lumped into the diagonal (a_ii + sum of dropped a_ij, ascending
 * column order); the pattern keeps only the diagonal and the kept entries;
 * D~_i = sum_j |(A_F)_ij| in ascending column order.  Where D~_i <= 1e-12
 * sum_j |a_ij| (every off-diagonal dropped, lumped row sum ~ 0) the row is
 * not smoothed: D~_i := +inf, so w / D~_i = 0 and P keeps the tentative row.
 * The paper notes that excessive dropping can leave near-zero diagonals and
 * does not treat the fully dropped row; this is our reading. */
/* ------------------------------------------------------------------------ */
csr_t or_filter(const csr_t* A, const uint8_t* keep, double* Dt) {
  int64_t n = A->nrows, nnz = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) nnz += (A->ci[p] == i) || keep[p];
  csr_t F = csr_new(n, A->ncols, nnz);
  int64_t w = 0;
  for (int64_t i = 0; i < n; ++i) {
    double dg = 0.0;
    int64_t dpos = -1;
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (A->ci[p] == i) dg = A->v[p];
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (A->ci[p] != i && !keep[p]) dg += A->v[p];
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      if (A->ci[p] == i) { dpos = w; F.ci[w] = (int32_t)i; F.v[w] = dg; ++w; }
      else if (keep[p]) { F.ci[w] = A->ci[p]; F.v[w] = A->v[p]; ++w; }
    }
    (void)dpos;
    F.rp[i + 1] = w;
    double s = 0.0;
    for (int64_t p = F.rp[i]; p < F.rp[i + 1]; ++p) s += fabs(F.v[p]);
    double a1 = 0.0;
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) a1 += fabs(A->v[p]);
    /* a row whose off-diagonals were all dropped is left to its lumped row
     * sum, which vanishes on rows of zero row sum; such a row is not smoothed:
     * D~_i := +inf makes D~_i^-1 = 0 (and its scaling in the power method 0) */
    Dt[i] = (s <= 1e-12 * a1) ? INFINITY : s;
  }
  return F;
}

/* ------------------------------------------------------------------------ */
/* power method on the symmetrically scaled matrix M = S A S, S = diag(s):
 * `steps` products from the hash-uniform start v_0; each step forms
 * w = M v, lambda = ||w|| / ||v||, v = w / ||w||; returns the last lambda,
 * an estimate of the spectral radius rho(M) (Sec. 2.2: the damping uses an
 * approximation of the spectral radius from a few power iterations).  The
 * norm ratio is used rather than the Rayleigh quotient because the lumped
 * filtered matrix may be indefinite, where the Rayleigh quotient can be
 * negative while the spectral radius is not. */
/* ------------------------------------------------------------------------ */
static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static void spmv_scaled(const csr_t* A, const double* s, const double* v, double* y) {
  for (int64_t i = 0; i < A->nrows; ++i) {
    double acc = 0.0;
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int64_t j = A->ci[p];
      acc += A->v[p] * (s[j] * v[j]);
    }
    y[i] = s[i] * acc;
  }
}

double or_power_estimate(const csr_t* A, const double* s, int steps, uint32_t tag, uint32_t seed) {
  int64_t n = A->nrows;
  double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) v[i] = or_start_value(i, tag, seed);
  double lam = 0.0;
  for (int it = 0; it < steps; ++it) {
    spmv_scaled(A, s, v, w);
    double nrm = sqrt(dot(n, w, w));
    if (nrm == 0.0) { lam = 0.0; break; } /* M v = 0: no spectral information */
    lam = nrm / sqrt(dot(n, v, v));
    for (int64_t i = 0; i < n; ++i) v[i] = w[i] / nrm;
  }
  free(v);
  free(w);
  return lam;
}

/* ------------------------------------------------------------------------ */
/* a12. Smoothed prolongator with the filtered matrix (Sec. 2.2):
 *   P = P^ - w D~^-1 A_F P^,  T = A_F P^ by the row-wise (Gustavson) product,
 *   c_i = w / D~_i,  P_ij = [j == agg(i)] - c_i * T_ij.
 * The pattern is the structural product; columns ascending; Dirichlet rows
 * empty. */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* C = A * B, Gustavson row by row: for k in A_i ascending, for j in B_k
 * ascending, acc[j] += a_ik * b_kj; columns of each row sorted ascending. */
csr_t or_spgemm(const csr_t* A, const csr_t* B) {
  int64_t n = A->nrows, m = B->ncols;
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
  double* acc = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  int32_t* cols = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  for (int64_t j = 0; j < m; ++j) mark[j] = -1;
  int64_t cap = csr_nnz(A) + 16, nnz = 0;
  int64_t* rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  double* v = (double*)malloc(sizeof(double) * (size_t)cap);
  for (int64_t i = 0; i < n; ++i) {
    int64_t nc = 0;
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int64_t k = A->ci[p];
      double a = A->v[p];
      for (int64_t q = B->rp[k]; q < B->rp[k + 1]; ++q) {
        int32_t j = B->ci[q];
        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols[nc++] = j; }
        acc[j] += a * B->v[q];
      }
    }
    qsort(cols, (size_t)nc, sizeof(int32_t), cmp_i32);
    if (nnz + nc > cap) {
      while (nnz + nc > cap) cap *= 2;
      ci = (int32_t*)realloc(ci, sizeof(int32_t) * (size_t)cap);
      v = (double*)realloc(v, sizeof(double) * (size_t)cap);
    }
    for (int64_t t = 0; t < nc; ++t) { ci[nnz] = cols[t]; v[nnz] = acc[cols[t]]; ++nnz; }
    rp[i + 1] = nnz;
  }
  free(mark); free(acc); free(cols);
  csr_t C;
  C.nrows = n; C.ncols = m; C.rp = rp; C.ci = ci; C.v = v;
  return C;
}

csr_t or_smooth_prolongator(const csr_t* F, const double* Dt, const csr_t* Pt, double omega,
                            const int32_t* agg) {
  csr_t T = or_spgemm(F, Pt);
  int64_t n = F->nrows;
  csr_t P = csr_new(n, Pt->ncols, csr_nnz(&T));
  int64_t w = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) {
      double c = omega / Dt[i];
      for (int64_t p = T.rp[i]; p < T.rp[i + 1]; ++p) {
        int32_t j = T.ci[p];
        P.ci[w] = j;
        P.v[w] = (j == agg[i]) ? 1.0 - c * T.v[p] : -(c * T.v[p]);
        ++w;
      }
    }
    P.rp[i + 1] = w;
  }
  csr_del(&T);
  return P;
}

/* R = P^T; rows of R list their source rows in ascending order */
csr_t or_transpose(const csr_t* P) {
  int64_t nnz = csr_nnz(P);
  csr_t R = csr_new(P->ncols, P->nrows, nnz);
  for (int64_t p = 0; p < nnz; ++p) R.rp[P->ci[p] + 1]++;
  for (int64_t j = 0; j < P->ncols; ++j) R.rp[j + 1] += R.rp[j];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P->ncols > 0 ? P->ncols : 1));
  for (int64_t j = 0; j < P->ncols; ++j) fill[j] = R.rp[j];
  for (int64_t i = 0; i < P->nrows; ++i)
    for (int64_t p = P->rp[i]; p < P->rp[i + 1]; ++p) {
      int64_t j = P->ci[p];
      R.ci[fill[j]] = (int32_t)i;
      R.v[fill[j]] = P->v[p];
      fill[j]++;
    }
  free(fill);
  return R;
}

/* ------------------------------------------------------------------------ */
/* a13. Galerkin product A_c = P^T A P (Sec. 2): AP = A P, then R (AP) with
 * R = P^T, both by or_spgemm; the result is stored exactly symmetric (the
 * lower triangle takes the value of the mirrored upper-triangle entry). */
/* ------------------------------------------------------------------------ */
static int64_t find_col(const csr_t* A, int64_t i, int32_t j) {
  int64_t lo = A->rp[i], hi = A->rp[i + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (A->ci[mid] == j) return mid;
    if (A->ci[mid] < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

int or_symmetrize_lower(csr_t* A) {
  for (int64_t i = 0; i < A->nrows; ++i)
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int32_t j = A->ci[p];
      if (j < i) {
        int64_t q = find_col(A, j, (int32_t)i);
        if (q < 0) return OR_ERR_INVALID_ARG;
        A->v[p] = A->v[q];
      }
    }
  return OR_OK;
}

csr_t or_galerkin(const csr_t* A, const csr_t* P, const csr_t* R, int* st) {
  csr_t AP = or_spgemm(A, P);
  csr_t Ac = or_spgemm(R, &AP);
  csr_del(&AP);
  *st = or_symmetrize_lower(&Ac);
  return Ac;
}

/* ------------------------------------------------------------------------ */
/* hierarchy */
/* ------------------------------------------------------------------------ */
typedef struct {
  csr_t A;
  double* dinv;          /* 1 / a_ii */
  double cheb_lmax, cheb_lmin;
  /* coarsening data (levels l < L-1) */
  uint8_t* dir;          /* Dirichlet flags (level 0) or NULL */
  uint8_t* keep;         /* strength mask per stored entry of A */
  uint8_t* root;
  int32_t* agg;
  int64_t nnz_gc;
  double omega, lam_omega;
  csr_t P, R;
  double *x, *sigma, *sinv; /* auxiliary data (material measure) */
} or_level_t;

typedef struct {
  int nlev;
  int dim;
  or_level_t lev[32];
  double* chol;          /* dense Cholesky factor of the coarsest operator */
  int64_t nL;
  int status;
} or_hier_t;

typedef struct {
  double theta;
  int measure;      /* 0 classical, 1 material, 2 distance Laplacian (sigma = I) */
  int drop;         /* 0 pointwise, 1 cut-drop */
  int max_coarse, max_levels;
  int power_iters;
  double omega_sym;
  double cheb_boost, cheb_ratio;
  uint32_t seed;
} or_opts_t;

static void level_free(or_level_t* L) {
  csr_del(&L->A);
  free(L->dinv); free(L->dir); free(L->keep); free(L->root); free(L->agg);
  if (L->P.rp) csr_del(&L->P);
  if (L->R.rp) csr_del(&L->R);
  free(L->x); free(L->sigma); free(L->sinv);
}

void or_free(or_hier_t* h) {
  if (!h) return;
  for (int l = 0; l < h->nlev; ++l) level_free(&h->lev[l]);
  free(h->chol);
  free(h);
}

static csr_t csr_copy_in(int64_t n, const int64_t* rp, const int32_t* ci, const double* v) {
  csr_t A = csr_new(n, n, rp[n]);
  memcpy(A.rp, rp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(A.ci, ci, sizeof(int32_t) * (size_t)rp[n]);
  memcpy(A.v, v, sizeof(double) * (size_t)rp[n]);
  return A;
}

/* dense Cholesky A = L L^T of the coarsest operator (row-major, lower) */
static int dense_cholesky(const csr_t* A, double** out) {
  int64_t n = A->nrows;
  double* L = (double*)calloc((size_t)(n * n > 0 ? n * n : 1), sizeof(double));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) L[i * n + A->ci[p]] = A->v[p];
  for (int64_t j = 0; j < n; ++j) {
    double d = L[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) { free(L); return OR_ERR_NOT_SPD; }
    d = sqrt(d);
    L[j * n + j] = d;
    for (int64_t i = j + 1; i < n; ++i) {
      double s = L[i * n + j];
      for (int64_t k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / d;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) L[i * n + j] = 0.0;
  *out = L;
  return OR_OK;
}

static void dense_chol_solve(int64_t n, const double* L, const double* b, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
    x[i] = s / L[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int64_t k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

/*
 * Setup of the hierarchy (Sec. 2 and Sec. 4 settings).  Inputs are host
 * arrays: CSR A (symmetric, sorted columns, diagonal stored), coordinates
 * n*dim, and either nodal tensors (tloc 0: n*kp) or elementwise tensors with
 * connectivity (tloc 1).  Coordinates/tensors may be NULL for the classical
 * measure.
 */
or_hier_t* or_setup(int dim, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                    const double* coords, int tloc, const double* tensors, int64_t ne, int npe,
                    const int32_t* en, const double* emeas, const or_opts_t* o, int* status) {
  or_hier_t* h = (or_hier_t*)calloc(1, sizeof(or_hier_t));
  h->dim = dim;
  const int kp = dim == 3 ? 6 : 3;
  int st = OR_OK;
  or_level_t* L0 = &h->lev[0];
  L0->A = csr_copy_in(n, rp, ci, v);
  h->nlev = 1;
  int use_aux = (o->measure == 1 || o->measure == 2);
  if (use_aux) {
    L0->x = (double*)malloc(sizeof(double) * (size_t)n * dim);
    memcpy(L0->x, coords, sizeof(double) * (size_t)n * dim);
    L0->sigma = (double*)malloc(sizeof(double) * (size_t)n * kp);
    if (o->measure == 2) {
      for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < kp; ++c) L0->sigma[i * kp + c] = (c < dim) ? 1.0 : 0.0;
    } else if (tloc == 0) {
      memcpy(L0->sigma, tensors, sizeof(double) * (size_t)n * kp);
    } else {
      st = or_nodal_from_elements(dim, n, ne, npe, en, emeas, tensors, L0->sigma);
      if (st) { *status = st; or_free(h); return NULL; }
    }
    L0->sinv = (double*)malloc(sizeof(double) * (size_t)n * kp);
    or_invert_tensors(dim, n, L0->sigma, L0->sinv);
  }
  L0->dir = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  or_dirichlet(n, rp, ci, v, L0->dir);

  for (int l = 0;; ++l) {
    or_level_t* Lc = &h->lev[l];
    int64_t nl = Lc->A.nrows;
    if (nl <= o->max_coarse || l + 1 >= o->max_levels) break;
    int64_t nnz = csr_nnz(&Lc->A);
    Lc->keep = (uint8_t*)malloc((size_t)(nnz > 0 ? nnz : 1));
    double* s2 = o->drop ? (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1)) : NULL;
    if (o->measure == 0) {
      or_strength_classical(nl, Lc->A.rp, Lc->A.ci, Lc->A.v, Lc->dir, o->theta, Lc->keep);
      if (o->drop) or_strength2_classical(nl, Lc->A.rp, Lc->A.ci, Lc->A.v, s2);
    } else {
      double* w = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
      double* D = (double*)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
      or_strength_material(dim, nl, Lc->A.rp, Lc->A.ci, Lc->dir, Lc->x, Lc->sinv, o->theta, w, D,
                           Lc->keep);
      if (o->drop) or_strength2_material(nl, Lc->A.rp, Lc->A.ci, w, D, s2);
      free(w); free(D);
    }
    if (o->drop) {
      or_cut_drop(nl, Lc->A.rp, Lc->A.ci, Lc->dir, s2, o->theta, Lc->keep);
      free(s2);
    }
    int64_t* gc_rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nl + 1));
    int32_t* gc_ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    Lc->nnz_gc = or_filtered_graph(nl, Lc->A.rp, Lc->A.ci, Lc->keep, Lc->dir, gc_rp, gc_ci);
    Lc->root = (uint8_t*)malloc((size_t)(nl > 0 ? nl : 1));
    or_mis2(nl, gc_rp, gc_ci, Lc->dir, l, o->seed, Lc->root);
    Lc->agg = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    int64_t nc = or_aggregate(nl, gc_rp, gc_ci, Lc->dir, Lc->root, Lc->agg);
    free(gc_rp); free(gc_ci);
    if (nc == 0 || (double)nc > 0.9 * (double)nl) {
      /* stagnation (or nothing to coarsen): level l is the coarsest */
      free(Lc->keep); Lc->keep = NULL;
      free(Lc->root); Lc->root = NULL;
      free(Lc->agg); Lc->agg = NULL;
      break;
    }
    csr_t Pt = or_tentative(nl, nc, Lc->agg);
    double* Dt = (double*)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    csr_t F = or_filter(&Lc->A, Lc->keep, Dt);
    double* s = (double*)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    for (int64_t i = 0; i < nl; ++i) s[i] = 1.0 / sqrt(Dt[i]);
    Lc->lam_omega = or_power_estimate(&F, s, o->power_iters, (uint32_t)(2 * l + 1), o->seed);
    Lc->omega = Lc->lam_omega > 0.0 ? o->omega_sym / Lc->lam_omega : 0.0;
    free(s);
    Lc->P = or_smooth_prolongator(&F, Dt, &Pt, Lc->omega, Lc->agg);
    csr_del(&F); csr_del(&Pt); free(Dt);
    Lc->R = or_transpose(&Lc->P);
    or_level_t* Ln = &h->lev[l + 1];
    Ln->A = or_galerkin(&Lc->A, &Lc->P, &Lc->R, &st);
    if (st) { h->nlev = l + 2; *status = st; or_free(h); return NULL; }
    if (use_aux) {
      Ln->x = (double*)malloc(sizeof(double) * (size_t)nc * dim);
      Ln->sigma = (double*)malloc(sizeof(double) * (size_t)nc * kp);
      Ln->sinv = (double*)malloc(sizeof(double) * (size_t)nc * kp);
      or_coarse_aux(dim, nl, nc, Lc->agg, Lc->x, Lc->sigma, Ln->x, Ln->sigma);
      or_invert_tensors(dim, nc, Ln->sigma, Ln->sinv);
    }
    h->nlev = l + 2;
  }
  or_level_t* Lc = &h->lev[h->nlev - 1];
  if (Lc->A.nrows > 16384) { *status = OR_ERR_STAGNATION; or_free(h); return NULL; }
  /* smoother data for every level above the coarsest (Sec. 4: Chebyshev 2) */
  for (int l = 0; l < h->nlev; ++l) {
    or_level_t* Lv = &h->lev[l];
    int64_t nl = Lv->A.nrows;
    Lv->dinv = (double*)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    double* s = (double*)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    for (int64_t i = 0; i < nl; ++i) {
      double d = diag_of(Lv->A.rp, Lv->A.ci, Lv->A.v, i);
      Lv->dinv[i] = 1.0 / d;
      s[i] = 1.0 / sqrt(d);
    }
    if (l + 1 < h->nlev) {
      double lam = or_power_estimate(&Lv->A, s, o->power_iters, (uint32_t)(2 * l + 2), o->seed);
      Lv->cheb_lmax = o->cheb_boost * lam;
      Lv->cheb_lmin = Lv->cheb_lmax / o->cheb_ratio;
    }
    free(s);
  }
  h->nL = Lc->A.nrows;
  st = dense_cholesky(&Lc->A, &h->chol);
  if (st) { *status = st; or_free(h); return NULL; }
  *status = OR_OK;
  return h;
}

/* ------------------------------------------------------------------------ */
/* solve phase */
/* ------------------------------------------------------------------------ */
static void spmv(const csr_t* A, const double* x, double* y) {
  for (int64_t i = 0; i < A->nrows; ++i) {
    double acc = 0.0;
    for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) acc += A->v[p] * x[A->ci[p]];
    y[i] = acc;
  }
}

/* Chebyshev smoothing of degree `deg` (Sec. 4; the standard three-term
 * Chebyshev iteration on D^-1 A with eigenvalue interval [lmin, lmax]):
 *   theta = (lmax+lmin)/2, delta = (lmax-lmin)/2, sigma1 = theta/delta,
 *   rho_0 = 1/sigma1
 *   step 1: r = b - A x; d = D^-1 r / theta; x += d
 *   step k: rho_k = 1/(2 sigma1 - rho_{k-1});
 *           r = b - A x; d = rho_k rho_{k-1} d + (2 rho_k / delta) D^-1 r; x += d
 * x_is_zero skips the first product. */
void or_chebyshev(const csr_t* A, const double* dinv, double lmax, double lmin, int deg,
                  const double* b, double* x, int x_is_zero, double* r, double* d) {
  int64_t n = A->nrows;
  double th = 0.5 * (lmax + lmin), de = 0.5 * (lmax - lmin);
  double s1 = th / de, rho = 1.0 / s1;
  if (x_is_zero) { for (int64_t i = 0; i < n; ++i) { r[i] = b[i]; x[i] = 0.0; } }
  else { spmv(A, x, r); for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i]; }
  for (int64_t i = 0; i < n; ++i) { d[i] = dinv[i] * r[i] / th; x[i] += d[i]; }
  for (int k = 1; k < deg; ++k) {
    double rn = 1.0 / (2.0 * s1 - rho);
    double c1 = rn * rho, c2 = 2.0 * rn / de;
    spmv(A, x, r);
    for (int64_t i = 0; i < n; ++i) {
      r[i] = b[i] - r[i];
      d[i] = c1 * d[i] + c2 * (dinv[i] * r[i]);
      x[i] += d[i];
    }
    rho = rn;
  }
}

/* V-cycle of Algorithm 1 (Sec. 2) with Chebyshev pre/post smoothing and the
 * direct coarse solve; x starts from zero on every level. */
static void vcycle(const or_hier_t* h, int l, const double* b, double* x, int deg) {
  const or_level_t* L = &h->lev[l];
  int64_t n = L->A.nrows;
  if (l == h->nlev - 1) { dense_chol_solve(n, h->chol, b, x); return; }
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  or_chebyshev(&L->A, L->dinv, L->cheb_lmax, L->cheb_lmin, deg, b, x, 1, r, d);
  spmv(&L->A, x, r);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  int64_t nc = L->P.ncols;
  double* bc = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
  double* xc = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
  spmv(&L->R, r, bc);
  vcycle(h, l + 1, bc, xc, deg);
  spmv(&L->P, xc, r);
  for (int64_t i = 0; i < n; ++i) x[i] += r[i];
  or_chebyshev(&L->A, L->dinv, L->cheb_lmax, L->cheb_lmin, deg, b, x, 0, r, d);
  free(r); free(d); free(bc); free(xc);
}

void or_vcycle(const or_hier_t* h, const double* b, double* x) { vcycle(h, 0, b, x, 2); }

/*
 * CG preconditioned by z = M r (Sec. 4: one V-cycle per iteration).
 * Converged when ||b - A x_k|| <= tol ||b - A x_0||; the recursive residual is
 * confirmed by the true residual.  flexible = 1 uses the Polak-Ribiere form
 * beta = z_k^T (r_k - r_{k-1}) / z_{k-1}^T r_{k-1}, which stays a
 * conjugate-direction method when M changes between iterations; flexible = 0
 * uses the plain beta = z_k^T r_k / z_{k-1}^T r_{k-1}.  Returns a status;
 * *iters counts operator products with the search direction; *relres is the
 * final true relative residual; hist (may be NULL, maxit + 1 entries)
 * receives ||r_k|| / ||r_0|| of the recursive residual after each step.
 */
typedef void (*or_prec_fn)(void* ctx, int k, const double* r, double* z);

static int pcg_core(const csr_t* A, or_prec_fn prec, void* ctx, const double* b, double* x, double tol,
                    int maxit, int flexible, int* iters, double* relres, double* hist) {
  int64_t n = A->nrows;
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  double* rp = (double*)malloc(sizeof(double) * (size_t)n);
  spmv(A, x, r);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  double r0 = sqrt(dot(n, r, r));
  int st = OR_ERR_NO_CONVERGENCE, it = 0, napp = 0;
  double rel = 0.0;
  if (hist) hist[0] = 1.0;
  if (r0 == 0.0) { st = OR_OK; goto done; }
  prec(ctx, napp++, r, z);
  memcpy(p, z, sizeof(double) * (size_t)n);
  double rz = dot(n, r, z);
  for (it = 1; it <= maxit; ++it) {
    spmv(A, p, q);
    double pq = dot(n, p, q);
    if (!(pq > 0.0)) { st = OR_ERR_BREAKDOWN; break; }
    double alpha = rz / pq;
    if (flexible) memcpy(rp, r, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
    double rn = sqrt(dot(n, r, r));
    if (hist) hist[it] = rn / r0;
    if (rn <= tol * r0) {
      spmv(A, x, q);
      for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
      double tn = sqrt(dot(n, q, q));
      if (tn <= tol * r0) { st = OR_OK; break; }
      memcpy(r, q, sizeof(double) * (size_t)n);
    }
    prec(ctx, napp++, r, z);
    double rzn = dot(n, r, z), beta;
    if (flexible) {
      double s = 0.0;
      for (int64_t i = 0; i < n; ++i) s += z[i] * (r[i] - rp[i]);
      beta = s / rz;
    } else {
      beta = rzn / rz;
    }
    rz = rzn;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  if (it > maxit) it = maxit;
done:
  spmv(A, x, q);
  for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
  rel = r0 > 0.0 ? sqrt(dot(n, q, q)) / r0 : 0.0;
  *iters = it;
  *relres = rel;
  free(r); free(z); free(p); free(q); free(rp);
  return st;
}

static void prec_vcycle(void* ctx, int k, const double* r, double* z) {
  (void)k;
  or_vcycle((const or_hier_t*)ctx, r, z);
}

int or_pcg(const or_hier_t* h, const double* b, double* x, double tol, int maxit, int flexible,
           int* iters, double* relres) {
  return pcg_core(&h->lev[0].A, prec_vcycle, (void*)h, b, x, tol, maxit, flexible, iters, relres, NULL);
}

/* or_pcg with the residual history (hist: maxit + 1 entries) */
int or_pcg_hist(const or_hier_t* h, const double* b, double* x, double tol, int maxit, int flexible,
                int* iters, double* relres, double* hist) {
  return pcg_core(&h->lev[0].A, prec_vcycle, (void*)h, b, x, tol, maxit, flexible, iters, relres, hist);
}

/* CG with a preconditioner that changes between applications: the k-th
 * application (k = 0, 1, ...) is z = diag(dinv[k mod ndiag]) r, dinv holding
 * ndiag vectors of n entries.  A test device for the flexible beta: with
 * ndiag > 1 only the Polak-Ribiere form keeps the search directions
 * A-conjugate. */
typedef struct { int64_t n; int ndiag; const double* dinv; } diag_cycle_t;

static void prec_diag_cycle(void* ctx, int k, const double* r, double* z) {
  const diag_cycle_t* c = (const diag_cycle_t*)ctx;
  const double* d = c->dinv + (size_t)(k % c->ndiag) * (size_t)c->n;
  for (int64_t i = 0; i < c->n; ++i) z[i] = d[i] * r[i];
}

int or_pcg_diag_cycle(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, int ndiag,
                      const double* dinv, const double* b, double* x, double tol, int maxit, int flexible,
                      int* iters, double* relres, double* hist) {
  csr_t A;
  A.nrows = n; A.ncols = n; A.rp = (int64_t*)rp; A.ci = (int32_t*)ci; A.v = (double*)v;
  diag_cycle_t c = {n, ndiag, dinv};
  return pcg_core(&A, prec_diag_cycle, &c, b, x, tol, maxit, flexible, iters, relres, hist);
}

/* ------------------------------------------------------------------------ */
/* export helpers for the tests */
/* ------------------------------------------------------------------------ */
int or_num_levels(const or_hier_t* h) { return h->nlev; }

void or_level_sizes(const or_hier_t* h, int l, int64_t* out) {
  const or_level_t* L = &h->lev[l];
  out[0] = L->A.nrows;
  out[1] = csr_nnz(&L->A);
  out[2] = L->P.rp ? csr_nnz(&L->P) : 0;
  out[3] = L->P.rp ? L->P.ncols : 0;
  out[4] = L->nnz_gc;
}

/* any pointer may be NULL; arrays sized by or_level_sizes */
void or_level_export(const or_hier_t* h, int l, int64_t* A_rp, int32_t* A_ci, double* A_v,
                     int32_t* agg, uint8_t* root, uint8_t* keep, uint8_t* dir, int64_t* P_rp,
                     int32_t* P_ci, double* P_v, double* x, double* sinv, double* scalars) {
  const or_level_t* L = &h->lev[l];
  int64_t n = L->A.nrows, nnz = csr_nnz(&L->A);
  const int kp = h->dim == 3 ? 6 : 3;
  if (A_rp) memcpy(A_rp, L->A.rp, sizeof(int64_t) * (size_t)(n + 1));
  if (A_ci) memcpy(A_ci, L->A.ci, sizeof(int32_t) * (size_t)nnz);
  if (A_v) memcpy(A_v, L->A.v, sizeof(double) * (size_t)nnz);
  if (agg && L->agg) memcpy(agg, L->agg, sizeof(int32_t) * (size_t)n);
  if (root && L->root) memcpy(root, L->root, (size_t)n);
  if (keep && L->keep) memcpy(keep, L->keep, (size_t)nnz);
  if (dir) { if (L->dir) memcpy(dir, L->dir, (size_t)n); else memset(dir, 0, (size_t)n); }
  if (L->P.rp) {
    int64_t pn = csr_nnz(&L->P);
    if (P_rp) memcpy(P_rp, L->P.rp, sizeof(int64_t) * (size_t)(n + 1));
    if (P_ci) memcpy(P_ci, L->P.ci, sizeof(int32_t) * (size_t)pn);
    if (P_v) memcpy(P_v, L->P.v, sizeof(double) * (size_t)pn);
  }
  if (x && L->x) memcpy(x, L->x, sizeof(double) * (size_t)n * h->dim);
  if (sinv && L->sinv) memcpy(sinv, L->sinv, sizeof(double) * (size_t)n * kp);
  if (scalars) {
    scalars[0] = L->omega;
    scalars[1] = L->lam_omega;
    scalars[2] = L->cheb_lmax;
    scalars[3] = L->cheb_lmin;
  }
}

/* overrides the Chebyshev interval of level l (for experiments on the
 * eigenvalue estimate; not part of the method) */
void or_set_cheb(or_hier_t* h, int l, double lmax, double lmin) {
  h->lev[l].cheb_lmax = lmax;
  h->lev[l].cheb_lmin = lmin;
}

double or_operator_complexity(const or_hier_t* h) {
  double s = 0.0;
  for (int l = 0; l < h->nlev; ++l) s += (double)csr_nnz(&h->lev[l].A);
  return s / (double)csr_nnz(&h->lev[0].A);
}

/* ------------------------------------------------------------------------ */
/* thin wrappers over single steps, for the pins */
/* ------------------------------------------------------------------------ */
typedef struct { csr_t m; } or_csr_box;

static or_csr_box* box(csr_t m) {
  or_csr_box* b = (or_csr_box*)malloc(sizeof(or_csr_box));
  b->m = m;
  return b;
}

void or_csr_info(const or_csr_box* b, int64_t* out) {
  out[0] = b->m.nrows; out[1] = b->m.ncols; out[2] = csr_nnz(&b->m);
}

void or_csr_copy(const or_csr_box* b, int64_t* rp, int32_t* ci, double* v) {
  int64_t nnz = csr_nnz(&b->m);
  memcpy(rp, b->m.rp, sizeof(int64_t) * (size_t)(b->m.nrows + 1));
  memcpy(ci, b->m.ci, sizeof(int32_t) * (size_t)nnz);
  memcpy(v, b->m.v, sizeof(double) * (size_t)nnz);
}

void or_csr_free(or_csr_box* b) { if (b) { csr_del(&b->m); free(b); } }

static csr_t view(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ci, const double* v) {
  csr_t m;
  m.nrows = nrows; m.ncols = ncols;
  m.rp = (int64_t*)rp; m.ci = (int32_t*)ci; m.v = (double*)v;
  return m;
}

or_csr_box* or_step_spgemm(int64_t n, int64_t k, int64_t m, const int64_t* arp, const int32_t* aci,
                           const double* av, const int64_t* brp, const int32_t* bci, const double* bv) {
  csr_t A = view(n, k, arp, aci, av), B = view(k, m, brp, bci, bv);
  return box(or_spgemm(&A, &B));
}

or_csr_box* or_step_transpose(int64_t n, int64_t m, const int64_t* rp, const int32_t* ci, const double* v) {
  csr_t A = view(n, m, rp, ci, v);
  return box(or_transpose(&A));
}

or_csr_box* or_step_filter(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                           const uint8_t* keep, double* Dt) {
  csr_t A = view(n, n, rp, ci, v);
  return box(or_filter(&A, keep, Dt));
}

or_csr_box* or_step_tentative(int64_t n, int64_t nc, const int32_t* agg) {
  return box(or_tentative(n, nc, agg));
}

or_csr_box* or_step_smooth_prolongator(int64_t n, int64_t nc, const int64_t* frp, const int32_t* fci,
                                       const double* fv, const double* Dt, double omega,
                                       const int32_t* agg) {
  csr_t F = view(n, n, frp, fci, fv);
  csr_t Pt = or_tentative(n, nc, agg);
  csr_t P = or_smooth_prolongator(&F, Dt, &Pt, omega, agg);
  csr_del(&Pt);
  return box(P);
}

or_csr_box* or_step_galerkin(int64_t n, int64_t nc, const int64_t* arp, const int32_t* aci,
                             const double* av, const int64_t* prp, const int32_t* pci,
                             const double* pv, int* status) {
  csr_t A = view(n, n, arp, aci, av), P = view(n, nc, prp, pci, pv);
  csr_t R = or_transpose(&P);
  csr_t Ac = or_galerkin(&A, &P, &R, status);
  csr_del(&R);
  return box(Ac);
}

double or_step_power(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                     const double* s, int steps, uint32_t tag, uint32_t seed) {
  csr_t A = view(n, n, rp, ci, v);
  return or_power_estimate(&A, s, steps, tag, seed);
}

void or_step_chebyshev(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                       const double* dinv, double lmax, double lmin, int deg, const double* b,
                       double* x, int x_is_zero) {
  csr_t A = view(n, n, rp, ci, v);
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  or_chebyshev(&A, dinv, lmax, lmin, deg, b, x, x_is_zero, r, d);
  free(r); free(d);
}

int or_dense_cholesky_factor(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double* Lout) {
  csr_t A = view(n, n, rp, ci, v);
  double* L = NULL;
  int st = dense_cholesky(&A, &L);
  if (st == OR_OK) { memcpy(Lout, L, sizeof(double) * (size_t)(n * n)); free(L); }
  return st;
}

void or_coarsest_solve(const or_hier_t* h, const double* b, double* x) {
  dense_chol_solve(h->nL, h->chol, b, x);
}
