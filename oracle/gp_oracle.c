/*
 * gp_oracle.c -- the oracle: a plain, slow, FP64 CPU statement of what the exact sparse GP computes.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls this file; only the tests,
 * the package's smoke check and the benchmark's CPU-baseline leg do. It shares no code, header, table or
 * helper with the CUDA library. Compile with -ffp-contract=off so every product/sum below is a separately
 * rounded IEEE operation in the order written.
 *
 * Contents, each with the passage it follows (arXiv 2411.05869):
 *   or_wendland          Wendland f0, Sec. 2.1 Eq. compSupp (coefficient 35 as printed)
 *   or_bump              bump function g, Sec. 2.1 Eq. bumpFcn
 *   or_features          f_i(x) = sum_j g_ij(x), Sec. 2.1 (sum of bumps below Eq. C_sparse)
 *   or_csparse / or_cy   C_sparse (Eq. C_sparse), C_y = C_core * C_sparse (Sec. 2, Eq. sparseCov)
 *   or_dense_cov         C_z = C_y + tau^2 I{x = x'} (Sec. 3.1, Eq. Zcov), all pairs
 *   or_pattern_*         brute-force O(n^2) support pattern (pairs with q^2 < 1 of the compact core)
 *   or_nd_order          geometric nested-dissection ordering (the paper is silent; the build's rule)
 *   or_etree_postorder   fill-preserving relabelling of an order by a postorder of its elimination tree
 *   or_symbolic          etree, column counts, supernodes from explicit column structures
 *   or_dense_chol, or_dense_loglik, or_sample_dense   dense Cholesky, log-likelihood of Sec. 3.3
 *   or_sparse_chol, or_sparse_loglik                  left-looking sparse Cholesky, same log-likelihood
 *   or_predict           predictive mean m = mu* + C_{y,z} C_z^{-1} r (Sec. 3.2)
 *   or_csr_values        C_z on a given pattern (the matrix of the iterative path of Sec. 3.3)
 *   core_paciorek        the parametric nonstationary Matern core of App. B (Eq. PScov), a non-compact core
 *   or_pattern_*_sparse  brute-force support of C_sparse (the pattern with a non-compact core)
 *
 * Hyperparameter block (theta, doubles), used by every kernel function:
 *   [0] core_var, [1..d] core_radius, [1+d] s0, [2+d..1+2d] r0, [2+2d] noise_var,
 *   then h (n1*n2*bump_dims), a (n1*n2), b (n1*n2), r (n1*n2).
 *   With the non-compact core (kind 1) the block continues with sigma0, Sigma0, phi_sigma (d), phi_Sigma (d).
 * Integer block (dims): d, n1, n2, bump_dims, core kind (0 compact Wendland, 1 parametric nonstationary Matern).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_WENDLAND_C3 35.0   /* cubic coefficient exactly as printed in Eq. compSupp */

typedef struct {
  int d, n1, n2, bd;
  double core_var, s0, noise_var;
  const double *core_radius, *r0, *h, *a, *b, *r;
  int kind;                       /* 0: compact Wendland core; 1: parametric nonstationary Matern core (App. B) */
  double sigma0, Sigma0;
  const double *phi_sigma, *phi_Sigma;
} hyp_t;

static hyp_t unpack(const int* dims, const double* th) {
  hyp_t p;
  p.d = dims[0]; p.n1 = dims[1]; p.n2 = dims[2]; p.bd = dims[3];
  int d = p.d, nb = p.n1 * p.n2;
  p.core_var = th[0];
  p.core_radius = th + 1;
  p.s0 = th[1 + d];
  p.r0 = th + 2 + d;
  p.noise_var = th[2 + 2 * d];
  p.h = th + 3 + 2 * d;
  p.a = p.h + nb * p.bd;
  p.b = p.a + nb;
  p.r = p.b + nb;
  p.kind = dims[4];
  p.sigma0 = p.Sigma0 = 1.0;
  p.phi_sigma = p.phi_Sigma = NULL;
  if (p.kind == 1) {
    const double* c = p.r + nb;
    p.sigma0 = c[0];
    p.Sigma0 = c[1];
    p.phi_sigma = c + 2;
    p.phi_Sigma = c + 2 + d;
  }
  return p;
}

/* ---------------------------------------------------------------- kernel (Sec. 2.1) */

/* f0 as a function of q = |x - x'| / r0: (1-q)^8 (35 q^3 + 25 q^2 + 8 q + 1) for q < 1, else 0. */
double or_wendland(double q) {
  if (!(q < 1.0)) return 0.0;
  double t = 1.0 - q;
  double t2 = t * t, t4 = t2 * t2, t8 = t4 * t4;
  double poly = ((OR_WENDLAND_C3 * q + 25.0) * q + 8.0) * q + 1.0;
  return t8 * poly;
}

/* squared anisotropic distance: sum_k (x_k/rad_k - y_k/rad_k)^2, summed in coordinate order */
static double q2_scaled(const double* x, const double* y, const double* rad, int d) {
  double s = 0.0;
  for (int k = 0; k < d; k++) {
    double dk = x[k] / rad[k] - y[k] / rad[k];
    s = s + dk * dk;
  }
  return s;
}

/* g(x) = a exp{ b [1 - (1 - |x-h|^2/r^2)^(-1)] } if |x-h| < r, else 0 (Eq. bumpFcn). */
double or_bump(const double* x, int bump_dims, const double* h, double a, double b, double r) {
  double s = 0.0;
  for (int k = 0; k < bump_dims; k++) {
    double dk = x[k] - h[k];
    s = s + dk * dk;
  }
  double rr = r * r;
  if (!(s < rr)) return 0.0;
  double t = s / rr;
  double e = b * (1.0 - 1.0 / (1.0 - t));
  return a * exp(e);
}

static void features_one(const hyp_t* p, const double* x, double* f) {
  for (int i = 0; i < p->n1; i++) {
    double acc = 0.0;
    for (int j = 0; j < p->n2; j++) {
      int ij = i * p->n2 + j;
      acc = acc + or_bump(x, p->bd, p->h + (size_t)ij * p->bd, p->a[ij], p->b[ij], p->r[ij]);
    }
    f[i] = acc;
  }
}

/* F (n x n1, row-major): f_i(x_k) = sum_j g_ij(x_k). */
void or_features(int64_t n, const int* dims, const double* th, const double* X, double* F) {
  hyp_t p = unpack(dims, th);
  for (int64_t k = 0; k < n; k++) features_one(&p, X + k * p.d, F + k * p.n1);
}

static double csparse_f(const hyp_t* p, const double* xi, const double* xj, const double* fi, const double* fj) {
  double acc = p->s0 * or_wendland(sqrt(q2_scaled(xi, xj, p->r0, p->d)));
  for (int i = 0; i < p->n1; i++) acc = acc + fi[i] * fj[i];
  return acc;
}

/* Matern correlation of smoothness 3/2: M(t) = (1 + sqrt(3) t) exp(-sqrt(3) t). */
static double matern32(double t) {
  double st = sqrt(3.0) * t;
  return (1.0 + st) * exp(-st);
}

/* The parametric nonstationary core of App. B (Eq. PScov), locally isotropic, smoothness 3/2:
 *   C(x, x') = sigma(x) sigma(x') (Sigma(x) Sigma(x'))^(d/4) / ((Sigma(x) + Sigma(x')) / 2)^(d/2) M(sqrt(Q)),
 *   Q = |x - x'|^2 / ((Sigma(x) + Sigma(x')) / 2),
 * with log sigma(x) = log sigma0 + sum_k phi_sigma_k x_k and log Sigma(x) = log Sigma0 + sum_k phi_Sigma_k x_k.
 * (The printed denominator repeats Sigma(x'); the average of Sigma(x) and Sigma(x') is the Paciorek form it cites.) */
static double core_paciorek(const hyp_t* p, const double* x, const double* y) {
  double lsx = log(p->sigma0), lsy = log(p->sigma0), lSx = log(p->Sigma0), lSy = log(p->Sigma0);
  for (int k = 0; k < p->d; k++) {
    lsx = lsx + p->phi_sigma[k] * x[k];
    lsy = lsy + p->phi_sigma[k] * y[k];
    lSx = lSx + p->phi_Sigma[k] * x[k];
    lSy = lSy + p->phi_Sigma[k] * y[k];
  }
  double sx = exp(lsx), sy = exp(lsy), Sx = exp(lSx), Sy = exp(lSy);
  double avg = (Sx + Sy) / 2.0;
  double pref = sx * sy * pow(Sx * Sy, p->d / 4.0) / pow(avg, p->d / 2.0);
  double r2 = 0.0;
  for (int k = 0; k < p->d; k++) {
    double dk = x[k] - y[k];
    r2 = r2 + dk * dk;
  }
  return pref * matern32(sqrt(r2 / avg));
}

static double cy_f(const hyp_t* p, const double* xi, const double* xj, const double* fi, const double* fj) {
  if (p->kind == 1) {
    double cs = csparse_f(p, xi, xj, fi, fj);
    if (cs == 0.0) return 0.0;
    return core_paciorek(p, xi, xj) * cs;
  }
  double wc = or_wendland(sqrt(q2_scaled(xi, xj, p->core_radius, p->d)));
  if (wc == 0.0) return 0.0;
  return (p->core_var * wc) * csparse_f(p, xi, xj, fi, fj);
}

/* C_sparse(x, x') = s0 f0(x, x'; r0) + sum_i f_i(x) f_i(x') (Eq. C_sparse). */
double or_csparse(const int* dims, const double* th, const double* xi, const double* xj) {
  hyp_t p = unpack(dims, th);
  double fi[64], fj[64];
  if (p.n1 > 64) return NAN;
  features_one(&p, xi, fi);
  features_one(&p, xj, fj);
  return csparse_f(&p, xi, xj, fi, fj);
}

/* C_y(x, x') = C_core(x, x') C_sparse(x, x') with C_core = core_var * f0-shaped Wendland of radius core_radius. */
double or_cy(const int* dims, const double* th, const double* xi, const double* xj) {
  hyp_t p = unpack(dims, th);
  double fi[64], fj[64];
  if (p.n1 > 64) return NAN;
  features_one(&p, xi, fi);
  features_one(&p, xj, fj);
  return cy_f(&p, xi, xj, fi, fj);
}

/* Dense C_z (n x n, row-major): C_y over all pairs plus tau^2 on the observation diagonal (Eq. Zcov). */
void or_dense_cov(int64_t n, const int* dims, const double* th, const double* X, int add_noise, double* C) {
  hyp_t p = unpack(dims, th);
  double* F = (double*)malloc(sizeof(double) * (size_t)(n * (p.n1 > 0 ? p.n1 : 1)));
  or_features(n, dims, th, X, F);
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < n; j++) {
      double v = cy_f(&p, X + i * p.d, X + j * p.d, F + i * p.n1, F + j * p.n1);
      if (i == j && add_noise) v = v + p.noise_var;
      C[i * n + j] = v;
    }
  free(F);
}

/* ---------------------------------------------------------------- support pattern, brute force */

/* Pattern predicate on the compact core: u = x / rho per coordinate, q^2 = sum_k (u_ik - u_jk)^2 in
 * coordinate order, include iff q^2 < 1. */
static int in_support(const double* xi, const double* xj, const double* rho, int d) {
  double s = 0.0;
  for (int k = 0; k < d; k++) {
    double dk = xi[k] / rho[k] - xj[k] / rho[k];
    s = s + dk * dk;
  }
  return s < 1.0;
}

/* Row counts (rowcnt[n]) of the full symmetric pattern; returns total. Rows are independent, so they may be
 * spread over threads (OpenMP, when the oracle is built with it) without changing any result. */
int64_t or_pattern_count(int64_t n, int d, const double* X, const double* rho, int64_t* rowcnt) {
  int64_t tot = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : tot)
  for (int64_t i = 0; i < n; i++) {
    int64_t c = 0;
    for (int64_t j = 0; j < n; j++) c += in_support(X + i * d, X + j * d, rho, d);
    rowcnt[i] = c;
    tot += c;
  }
  return tot;
}

/* CSR fill: rowptr[n+1] must hold the prefix sums of or_pattern_count; columns ascending. */
void or_pattern_fill(int64_t n, int d, const double* X, const double* rho, const int64_t* rowptr, int32_t* col) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; i++) {
    int64_t o = rowptr[i];
    for (int64_t j = 0; j < n; j++)
      if (in_support(X + i * d, X + j * d, rho, d)) col[o++] = (int32_t)j;
  }
}

/* One row of the pattern by brute force (for sampled checks at large n). Returns the count written. */
int64_t or_pattern_row(int64_t n, int d, const double* X, const double* rho, int64_t i, int32_t* out, int64_t cap) {
  int64_t c = 0;
  for (int64_t j = 0; j < n; j++)
    if (in_support(X + i * d, X + j * d, rho, d)) {
      if (c < cap) out[c] = (int32_t)j;
      c++;
    }
  return c;
}

/* ---------------------------------------------------------------- nested dissection (build-defined rule) */
/*
 * ND(V): if |V| <= 64, order V by (cell key, index). Otherwise choose the coordinate k with the largest
 * extent max u_k - min u_k over V (ties: lowest k), sort V by (u_k, index), L = first floor(|V|/2), R = rest,
 * S = {v in L with a pattern neighbour in R}; emit ND(L \ S), ND(R), then S in (u_k, index) order.
 * u = x / rho per coordinate. Cell key: c_k = floor(u_k) - floor(min over all points u_k),
 * key = c_0 + nc_0 (c_1 + nc_1 c_2), nc_k = floor(max u_k) - floor(min u_k) + 1.
 */
#define ND_LEAF 64

typedef struct {
  int d;
  const double* U;       /* n x d scaled coordinates */
  const int64_t* key;    /* cell keys */
  const int64_t* rowptr;
  const int32_t* col;
  int32_t* side;         /* scratch marker per vertex */
  int32_t* out;          /* output order */
  int64_t pos;           /* next output slot */
  int32_t* node_lo;      /* optional ND tree record: [lo, hi) of each emitted separator/leaf */
  int32_t* node_hi;
  int32_t* node_kind;    /* 0 leaf, 1 separator */
  int64_t nnodes;
} nd_t;

typedef struct { double u; int32_t v; } uv_t;
typedef struct { int64_t key; int32_t v; } kv_t;

static int cmp_uv(const void* a, const void* b) {
  const uv_t* x = (const uv_t*)a; const uv_t* y = (const uv_t*)b;
  if (x->u < y->u) return -1;
  if (x->u > y->u) return 1;
  return (x->v > y->v) - (x->v < y->v);
}
static int cmp_kv(const void* a, const void* b) {
  const kv_t* x = (const kv_t*)a; const kv_t* y = (const kv_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->v > y->v) - (x->v < y->v);
}

static void nd_rec(nd_t* st, int32_t* V, int64_t m) {
  if (m == 0) return;
  if (m <= ND_LEAF) {
    kv_t* t = (kv_t*)malloc(sizeof(kv_t) * (size_t)m);
    for (int64_t i = 0; i < m; i++) { t[i].key = st->key[V[i]]; t[i].v = V[i]; }
    qsort(t, (size_t)m, sizeof(kv_t), cmp_kv);
    int64_t lo = st->pos;
    for (int64_t i = 0; i < m; i++) st->out[st->pos++] = t[i].v;
    if (st->node_lo) { st->node_lo[st->nnodes] = (int32_t)lo; st->node_hi[st->nnodes] = (int32_t)st->pos; st->node_kind[st->nnodes] = 0; }
    st->nnodes++;
    free(t);
    return;
  }
  int d = st->d, kbest = 0;
  double best = -1.0;
  for (int k = 0; k < d; k++) {
    double mn = st->U[(int64_t)V[0] * d + k], mx = mn;
    for (int64_t i = 1; i < m; i++) {
      double u = st->U[(int64_t)V[i] * d + k];
      if (u < mn) mn = u;
      if (u > mx) mx = u;
    }
    double ext = mx - mn;
    if (ext > best) { best = ext; kbest = k; }
  }
  uv_t* t = (uv_t*)malloc(sizeof(uv_t) * (size_t)m);
  for (int64_t i = 0; i < m; i++) { t[i].u = st->U[(int64_t)V[i] * d + kbest]; t[i].v = V[i]; }
  qsort(t, (size_t)m, sizeof(uv_t), cmp_uv);
  int64_t nl = m / 2;
  for (int64_t i = nl; i < m; i++) st->side[t[i].v] = 1;            /* mark R */
  int32_t* inS = (int32_t*)calloc((size_t)nl, sizeof(int32_t));
  int64_t ns = 0;
  for (int64_t i = 0; i < nl; i++) {
    int32_t v = t[i].v;
    for (int64_t e = st->rowptr[v]; e < st->rowptr[v + 1]; e++)
      if (st->side[st->col[e]] == 1) { inS[i] = 1; ns++; break; }
  }
  for (int64_t i = nl; i < m; i++) st->side[t[i].v] = 0;            /* clear marks before recursing */
  int32_t* Lrest = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nl - ns + 1));
  int32_t* R = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m - nl));
  int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ns + 1));
  int64_t a = 0, s = 0;
  for (int64_t i = 0; i < nl; i++) {
    if (inS[i]) S[s++] = t[i].v; else Lrest[a++] = t[i].v;
  }
  for (int64_t i = nl; i < m; i++) R[i - nl] = t[i].v;
  free(t);
  free(inS);
  nd_rec(st, Lrest, a);
  nd_rec(st, R, m - nl);
  int64_t lo = st->pos;
  for (int64_t i = 0; i < s; i++) st->out[st->pos++] = S[i];
  if (st->node_lo) { st->node_lo[st->nnodes] = (int32_t)lo; st->node_hi[st->nnodes] = (int32_t)st->pos; st->node_kind[st->nnodes] = 1; }
  st->nnodes++;
  free(Lrest); free(R); free(S);
}

/* Cell keys of the uniform grid with unit cells in u = x / rho. */
void or_cell_keys(int64_t n, int d, const double* X, const double* rho, int64_t* key) {
  double mn[3], mx[3];
  int64_t c0[3], nc[3];
  for (int k = 0; k < d; k++) { mn[k] = INFINITY; mx[k] = -INFINITY; }
  for (int64_t i = 0; i < n; i++)
    for (int k = 0; k < d; k++) {
      double u = X[i * d + k] / rho[k];
      if (u < mn[k]) mn[k] = u;
      if (u > mx[k]) mx[k] = u;
    }
  for (int k = 0; k < d; k++) { c0[k] = (int64_t)floor(mn[k]); nc[k] = (int64_t)floor(mx[k]) - c0[k] + 1; }
  for (int64_t i = 0; i < n; i++) {
    int64_t kk = 0;
    for (int k = d - 1; k >= 0; k--) {
      int64_t c = (int64_t)floor(X[i * d + k] / rho[k]) - c0[k];
      kk = kk * nc[k] + c;
    }
    key[i] = kk;
  }
}

/* perm[new] = old. Optional node arrays (capacity n) receive the emitted ND pieces; returns their count. */
int64_t or_nd_order(int64_t n, int d, const double* X, const double* rho, const int64_t* rowptr,
                    const int32_t* col, int32_t* perm, int32_t* node_lo, int32_t* node_hi, int32_t* node_kind) {
  double* U = (double*)malloc(sizeof(double) * (size_t)(n * d));
  for (int64_t i = 0; i < n * d; i++) U[i] = X[i] / rho[i % d];
  int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  or_cell_keys(n, d, X, rho, key);
  nd_t st;
  st.d = d; st.U = U; st.key = key; st.rowptr = rowptr; st.col = col;
  st.side = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  st.out = perm; st.pos = 0;
  st.node_lo = node_lo; st.node_hi = node_hi; st.node_kind = node_kind; st.nnodes = 0;
  int32_t* V = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < n; i++) V[i] = (int32_t)i;
  nd_rec(&st, V, n);
  free(V); free(st.side); free(key); free(U);
  return st.nnodes;
}

/* ---------------------------------------------------------------- symbolic analysis */
/*
 * Column structures of L for A = P C P^T by the textbook union rule, processing columns in order:
 *   struct(j) = {i > j : A_ij != 0}  U  union over children k of j of (struct(k) \ {j}),
 * parent(j) = min struct(j) (or -1), eta_j = |struct(j)| + 1 (diagonal included).
 * Structures are kept as sorted arrays (memory ~ nnz(L)).
 */
typedef struct {
  int64_t n;
  int32_t** s;    /* s[j]: sorted strictly-below-diagonal rows of column j */
  int32_t* len;
  int32_t* parent;
} colstruct_t;

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static void colstruct_build(colstruct_t* cs, int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm) {
  int32_t* pinv = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) pinv[perm[i]] = (int32_t)i;
  cs->n = n;
  cs->s = (int32_t**)calloc((size_t)n, sizeof(int32_t*));
  cs->len = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  cs->parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  /* children lists as linked lists */
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) head[i] = -1;
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) mark[i] = -1;
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t j = 0; j < n; j++) {
    int64_t cnt = 0;
    int32_t oj = perm[j];
    for (int64_t e = rowptr[oj]; e < rowptr[oj + 1]; e++) {
      int32_t i = pinv[col[e]];
      if (i > j && mark[i] != j) { mark[i] = (int32_t)j; buf[cnt++] = i; }
    }
    for (int32_t k = head[j]; k != -1; k = next[k])
      for (int32_t t = 0; t < cs->len[k]; t++) {
        int32_t i = cs->s[k][t];
        if (i > j && mark[i] != j) { mark[i] = (int32_t)j; buf[cnt++] = i; }
      }
    qsort(buf, (size_t)cnt, sizeof(int32_t), cmp_i32);
    cs->len[j] = (int32_t)cnt;
    cs->s[j] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
    memcpy(cs->s[j], buf, sizeof(int32_t) * (size_t)cnt);
    cs->parent[j] = cnt > 0 ? buf[0] : -1;
    if (cnt > 0) { next[j] = head[buf[0]]; head[buf[0]] = (int32_t)j; }
  }
  free(buf); free(mark); free(head); free(next); free(pinv);
}

static void colstruct_free(colstruct_t* cs) {
  for (int64_t j = 0; j < cs->n; j++) free(cs->s[j]);
  free(cs->s); free(cs->len); free(cs->parent);
}

/*
 * Supernodes.
 * Fundamental: j and j+1 share a supernode iff parent(j) = j+1, eta_j = eta_{j+1} + 1 and j is the only
 * child of j+1.
 * Relaxed amalgamation, supernodes taken in increasing column order: while the supernode c that ends at
 * first(p)-1 has its supernodal parent equal to p, merge c into p if the merged width is <= 16 or if the
 * explicit zeros of the merged panel are at most 10 % of its entries (10 * zeros <= entries). Bounding the
 * total, not only the zeros one merge adds, keeps chains of separators from compounding into wide, mostly
 * empty supernodes.
 * A panel of columns [f, l] with r rows below l holds sum_{j=f..l} (l - j + 1 + r) entries; r = eta_l - 1.
 * Returns the supernode count; sn_first[ns+1] are the first columns (sn_first[ns] = n).
 */
#define SN_RELAX_WIDTH 16

static int64_t panel_entries(int64_t f, int64_t l, int64_t r) {
  int64_t w = l - f + 1;
  return w * (w + 1) / 2 + w * r;
}

int64_t or_supernodes(int64_t n, const int32_t* parent, const int32_t* eta, int32_t* sn_first) {
  int32_t* nchild = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  for (int64_t j = 0; j < n; j++) if (parent[j] >= 0) nchild[parent[j]]++;
  /* fundamental supernodes as [first, last] */
  int64_t* f = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t ns = 0;
  f[ns++] = 0;
  for (int64_t j = 0; j + 1 < n; j++) {
    int same = parent[j] == j + 1 && eta[j] == eta[j + 1] + 1 && nchild[j + 1] == 1;
    if (!same) f[ns++] = j + 1;
  }
  f[ns] = n;
  /* column -> fundamental supernode */
  int64_t* zeros = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  int64_t* first = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  int64_t* last = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  int64_t* exact = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  int32_t* snof = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t s = 0; s < ns; s++) {
    first[s] = f[s]; last[s] = f[s + 1] - 1;
    int64_t ex = 0;
    for (int64_t j = first[s]; j <= last[s]; j++) { ex += eta[j]; snof[j] = (int32_t)s; }
    exact[s] = ex;
    zeros[s] = panel_entries(first[s], last[s], eta[last[s]] - 1) - ex;
  }
  /* merged supernodes kept on a stack in increasing order; top is the latest */
  int64_t* st_first = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  int64_t* st_last = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  int64_t* st_exact = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  int64_t* st_zeros = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  int64_t top = 0;
  for (int64_t s = 0; s < ns; s++) {
    int64_t pf = first[s], pl = last[s], pex = exact[s], pz = zeros[s];
    while (top > 0) {
      int64_t cf = st_first[top - 1], cl = st_last[top - 1];
      if (cl != pf - 1) break;
      int32_t par = parent[cl];
      if (!(par >= pf && par <= pl)) break;
      int64_t r = eta[pl] - 1;
      int64_t ent = panel_entries(cf, pl, r);
      int64_t ex = st_exact[top - 1] + pex;
      int64_t mz = ent - ex;
      int64_t width = pl - cf + 1;
      if (width <= SN_RELAX_WIDTH || 10 * mz <= ent) {
        pf = cf; pex = ex; pz = mz;
        top--;
      } else {
        break;
      }
    }
    st_first[top] = pf; st_last[top] = pl; st_exact[top] = pex; st_zeros[top] = pz;
    top++;
  }
  for (int64_t s = 0; s < top; s++) sn_first[s] = (int32_t)st_first[s];
  sn_first[top] = (int32_t)n;
  free(nchild); free(f); free(zeros); free(first); free(last); free(exact); free(snof);
  free(st_first); free(st_last); free(st_exact); free(st_zeros);
  return top;
}

/*
 * Full symbolic analysis of P C P^T (perm[new] = old):
 *   parent[n], eta[n]; supernodes sn_first[ns+1] (capacity n+1); returns ns.
 *   If sn_rows != NULL (capacity given by sn_rows_cap) it receives, per supernode in order, the sorted rows
 *   below the supernode (struct of its last column), with sn_rowptr[ns+1] offsets; sn_level[ns] the height
 *   of each supernode in the supernodal tree (0 for leaves); sn_parent[ns].
 */
int64_t or_symbolic(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm,
                    int32_t* parent, int32_t* eta, int32_t* sn_first, int64_t* sn_rowptr, int32_t* sn_rows,
                    int64_t sn_rows_cap, int32_t* sn_parent, int32_t* sn_level, int64_t* nnzL_out) {
  colstruct_t cs;
  colstruct_build(&cs, n, rowptr, col, perm);
  int64_t nnzL = 0;
  for (int64_t j = 0; j < n; j++) {
    parent[j] = cs.parent[j];
    eta[j] = cs.len[j] + 1;
    nnzL += eta[j];
  }
  if (nnzL_out) *nnzL_out = nnzL;
  int64_t ns = or_supernodes(n, parent, eta, sn_first);
  int32_t* snof = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t s = 0; s < ns; s++)
    for (int64_t j = sn_first[s]; j < sn_first[s + 1]; j++) snof[j] = (int32_t)s;
  if (sn_rowptr) {
    int64_t o = 0;
    sn_rowptr[0] = 0;
    for (int64_t s = 0; s < ns; s++) {
      int64_t l = sn_first[s + 1] - 1;
      for (int32_t t = 0; t < cs.len[l]; t++) {
        if (sn_rows && o < sn_rows_cap) sn_rows[o] = cs.s[l][t];
        o++;
      }
      sn_rowptr[s + 1] = o;
    }
  }
  if (sn_parent || sn_level) {
    int32_t* sp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ns + 1));
    int32_t* lv = (int32_t*)calloc((size_t)(ns + 1), sizeof(int32_t));
    for (int64_t s = 0; s < ns; s++) {
      int64_t l = sn_first[s + 1] - 1;
      sp[s] = parent[l] >= 0 ? snof[parent[l]] : -1;
    }
    for (int64_t s = 0; s < ns; s++)           /* children precede parents */
      if (sp[s] >= 0 && lv[sp[s]] < lv[s] + 1) lv[sp[s]] = lv[s] + 1;
    for (int64_t s = 0; s < ns; s++) {
      if (sn_parent) sn_parent[s] = sp[s];
      if (sn_level) sn_level[s] = lv[s];
    }
    free(sp); free(lv);
  }
  free(snof);
  colstruct_free(&cs);
  return ns;
}

/*
 * Fill-preserving relabelling of an ordering by a postorder of its elimination tree (children visited in
 * increasing index order, roots in increasing order). The factor of the relabelled matrix has the same
 * column counts (permuted) and the same fill; each subtree becomes a contiguous range of columns, so chains
 * of the tree become runs j, j+1, ... . out_perm[new] = perm[post[new]].
 */
void or_etree_postorder(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm, int32_t* out_perm) {
  colstruct_t cs;
  colstruct_build(&cs, n, rowptr, col, perm);
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t j = 0; j < n; j++) head[j] = -1;
  for (int64_t j = n - 1; j >= 0; j--) {            /* prepend in decreasing order: lists ascend */
    int32_t p = cs.parent[j];
    if (p >= 0) { next[j] = head[p]; head[p] = (int32_t)j; }
  }
  int64_t k = 0;
  for (int64_t root = 0; root < n; root++) {
    if (cs.parent[root] != -1) continue;
    int64_t top = 0;
    stack[top++] = (int32_t)root;
    while (top > 0) {
      int32_t v = stack[top - 1];
      int32_t c = head[v];
      if (c != -1) {                                 /* descend into the next unvisited child */
        head[v] = next[c];
        stack[top++] = c;
      } else {
        top--;
        out_perm[k++] = perm[v];
      }
    }
  }
  free(head); free(next); free(stack);
  colstruct_free(&cs);
}

/* ---------------------------------------------------------------- dense path (n up to a few thousand) */

/* Kahan-compensated sum accumulator */
typedef struct { double s, c; } kahan_t;
static void kadd(kahan_t* k, double x) {
  double y = x - k->c;
  double t = k->s + y;
  k->c = (t - k->s) - y;
  k->s = t;
}

/* In-place lower Cholesky of a row-major n x n SPD matrix (upper part left untouched).
 * Returns -1 on success or the failing column index. */
int64_t or_dense_chol(int64_t n, double* A) {
  for (int64_t j = 0; j < n; j++) {
    double s = A[j * n + j];
    for (int64_t k = 0; k < j; k++) s = s - A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return j;
    double ljj = sqrt(s);
    A[j * n + j] = ljj;
    for (int64_t i = j + 1; i < n; i++) {
      double t = A[i * n + j];
      for (int64_t k = 0; k < j; k++) t = t - A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / ljj;
    }
  }
  return -1;
}

static void dense_fwd(int64_t n, const double* L, double* x) {      /* L x = b in place */
  for (int64_t i = 0; i < n; i++) {
    double t = x[i];
    for (int64_t k = 0; k < i; k++) t = t - L[i * n + k] * x[k];
    x[i] = t / L[i * n + i];
  }
}
static void dense_bwd(int64_t n, const double* L, double* x) {      /* L^T x = b in place */
  for (int64_t i = n - 1; i >= 0; i--) {
    double t = x[i];
    for (int64_t k = i + 1; k < n; k++) t = t - L[k * n + i] * x[k];
    x[i] = t / L[i * n + i];
  }
}

/*
 * log p(z | beta, theta) = -1/2 log det C_z - 1/2 r^T C_z^{-1} r - n/2 log(2 pi) (Sec. 3.3), dense.
 * out[0] = loglik, out[1] = logdet, out[2] = quadratic form. alpha (n, nullable) receives C_z^{-1} r.
 * Returns -1 or the failing pivot.
 */
int64_t or_dense_loglik(int64_t n, const int* dims, const double* th, const double* X, const double* resid,
                        double* out, double* alpha) {
  double* C = (double*)malloc(sizeof(double) * (size_t)(n * n));
  or_dense_cov(n, dims, th, X, 1, C);
  int64_t fail = or_dense_chol(n, C);
  if (fail >= 0) { free(C); return fail; }
  kahan_t ld = {0, 0};
  for (int64_t j = 0; j < n; j++) kadd(&ld, log(C[j * n + j]));
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(w, resid, sizeof(double) * (size_t)n);
  dense_fwd(n, C, w);
  kahan_t q = {0, 0};
  for (int64_t j = 0; j < n; j++) kadd(&q, w[j] * w[j]);
  if (alpha) {
    memcpy(alpha, w, sizeof(double) * (size_t)n);
    dense_bwd(n, C, alpha);
  }
  double logdet = 2.0 * ld.s;
  out[1] = logdet;
  out[2] = q.s;
  out[0] = -0.5 * logdet - 0.5 * q.s - 0.5 * (double)n * log(2.0 * M_PI);
  free(w); free(C);
  return -1;
}

/* y = L_y o with L_y the dense Cholesky factor of C_y (no noise): a GP draw (Sec. 3.2, unconditional
 * simulation). Returns -1 or the failing pivot. */
int64_t or_sample_dense(int64_t n, const int* dims, const double* th, const double* X, const double* o, double* y) {
  double* C = (double*)malloc(sizeof(double) * (size_t)(n * n));
  or_dense_cov(n, dims, th, X, 0, C);
  int64_t fail = or_dense_chol(n, C);
  if (fail < 0)
    for (int64_t i = 0; i < n; i++) {
      double t = 0.0;
      for (int64_t k = 0; k <= i; k++) t = t + C[i * n + k] * o[k];
      y[i] = t;
    }
  free(C);
  return fail;
}

/* ---------------------------------------------------------------- sparse left-looking Cholesky */
/*
 * Column-by-column left-looking Cholesky of A = P C_z P^T on the symbolic structure (George & Liu):
 * for column j, gather A(j:n, j) into a dense work vector, subtract L(j:n, k) L(j, k) for every k < j with
 * L(j, k) != 0, then L(j, j) = sqrt(w_j), L(i, j) = w_i / L(j, j). Entries A(i, j) come straight from the
 * kernel definition, C_z(perm[i], perm[j]). L is stored column-wise on the structure (diagonal first).
 */
typedef struct {
  int64_t n;
  int64_t* cp;     /* column pointers, n+1 */
  int32_t* ri;     /* row indices (diagonal first) */
  double* v;
} spL_t;

static int64_t sparse_chol(const colstruct_t* cs, const int* dims, const double* th, const double* X,
                           const int32_t* perm, spL_t* L) {
  hyp_t p = unpack(dims, th);
  int64_t n = cs->n;
  L->n = n;
  L->cp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  L->cp[0] = 0;
  for (int64_t j = 0; j < n; j++) L->cp[j + 1] = L->cp[j] + cs->len[j] + 1;
  L->ri = (int32_t*)malloc(sizeof(int32_t) * (size_t)L->cp[n]);
  L->v = (double*)malloc(sizeof(double) * (size_t)L->cp[n]);
  for (int64_t j = 0; j < n; j++) {
    L->ri[L->cp[j]] = (int32_t)j;
    memcpy(L->ri + L->cp[j] + 1, cs->s[j], sizeof(int32_t) * (size_t)cs->len[j]);
  }
  double* F = (double*)malloc(sizeof(double) * (size_t)(n * (p.n1 > 0 ? p.n1 : 1)));
  or_features(n, dims, th, X, F);
  double* w = (double*)calloc((size_t)n, sizeof(double));
  int64_t* nxt = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);   /* next pending entry of column k */
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);  /* columns waiting on row i */
  int32_t* link = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) head[i] = -1;
  int64_t fail = -1;
  for (int64_t j = 0; j < n && fail < 0; j++) {
    int32_t oj = perm[j];
    for (int64_t e = L->cp[j]; e < L->cp[j + 1]; e++) {
      int32_t i = L->ri[e], oi = perm[i];
      double v = cy_f(&p, X + (int64_t)oi * p.d, X + (int64_t)oj * p.d, F + (int64_t)oi * p.n1, F + (int64_t)oj * p.n1);
      if (i == j) v = v + p.noise_var;
      w[i] = v;
    }
    int32_t k = head[j];
    head[j] = -1;
    while (k != -1) {
      int32_t knext = link[k];
      int64_t e0 = nxt[k];                 /* entry of row j in column k */
      double ljk = L->v[e0];
      for (int64_t e = e0; e < L->cp[k + 1]; e++) w[L->ri[e]] = w[L->ri[e]] - L->v[e] * ljk;
      if (e0 + 1 < L->cp[k + 1]) {
        nxt[k] = e0 + 1;
        int32_t r = L->ri[e0 + 1];
        link[k] = head[r];
        head[r] = k;
      }
      k = knext;
    }
    double d = w[j];
    if (!(d > 0.0)) { fail = j; break; }
    double ljj = sqrt(d);
    L->v[L->cp[j]] = ljj;
    w[j] = 0.0;
    for (int64_t e = L->cp[j] + 1; e < L->cp[j + 1]; e++) {
      int32_t i = L->ri[e];
      L->v[e] = w[i] / ljj;
      w[i] = 0.0;
    }
    if (L->cp[j] + 1 < L->cp[j + 1]) {
      nxt[j] = L->cp[j] + 1;
      int32_t r = L->ri[L->cp[j] + 1];
      link[j] = head[r];
      head[r] = (int32_t)j;
    }
  }
  free(F); free(w); free(nxt); free(head); free(link);
  return fail;
}

/*
 * Sparse exact log-likelihood (same quantity as or_dense_loglik) through the sparse factor.
 * out[0..2] as in the dense version; out[3] = nnz(L); alpha (nullable) = C_z^{-1} r in original order.
 * Optional Ldiag[n] (nullable) receives L(j, j) in permuted order. Returns -1 or failing permuted column.
 */
int64_t or_sparse_loglik(int64_t n, const int* dims, const double* th, const double* X, const int64_t* rowptr,
                         const int32_t* col, const int32_t* perm, const double* resid, double* out,
                         double* alpha, double* Ldiag) {
  colstruct_t cs;
  colstruct_build(&cs, n, rowptr, col, perm);
  spL_t L;
  int64_t fail = sparse_chol(&cs, dims, th, X, perm, &L);
  colstruct_free(&cs);
  if (fail < 0) {
    kahan_t ld = {0, 0};
    for (int64_t j = 0; j < n; j++) {
      kadd(&ld, log(L.v[L.cp[j]]));
      if (Ldiag) Ldiag[j] = L.v[L.cp[j]];
    }
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; i++) w[i] = resid[perm[i]];
    for (int64_t j = 0; j < n; j++) {                       /* L w = P r, column oriented */
      w[j] = w[j] / L.v[L.cp[j]];
      for (int64_t e = L.cp[j] + 1; e < L.cp[j + 1]; e++) w[L.ri[e]] = w[L.ri[e]] - L.v[e] * w[j];
    }
    kahan_t q = {0, 0};
    for (int64_t j = 0; j < n; j++) kadd(&q, w[j] * w[j]);
    if (alpha) {
      for (int64_t j = n - 1; j >= 0; j--) {                /* L^T a = w */
        double t = w[j];
        for (int64_t e = L.cp[j] + 1; e < L.cp[j + 1]; e++) t = t - L.v[e] * w[L.ri[e]];
        w[j] = t / L.v[L.cp[j]];
      }
      for (int64_t i = 0; i < n; i++) alpha[perm[i]] = w[i];
    }
    double logdet = 2.0 * ld.s;
    out[1] = logdet;
    out[2] = q.s;
    out[0] = -0.5 * logdet - 0.5 * q.s - 0.5 * (double)n * log(2.0 * M_PI);
    out[3] = (double)L.cp[n];
    free(w);
  }
  free(L.cp); free(L.ri); free(L.v);
  return fail;
}

/* Sparse factor entries as a COO list in permuted coordinates (for reconstruction checks at small n).
 * Returns nnz(L); writes up to cap entries. */
int64_t or_sparse_factor(int64_t n, const int* dims, const double* th, const double* X, const int64_t* rowptr,
                         const int32_t* col, const int32_t* perm, int32_t* ri, int32_t* ci, double* v, int64_t cap) {
  colstruct_t cs;
  colstruct_build(&cs, n, rowptr, col, perm);
  spL_t L;
  int64_t fail = sparse_chol(&cs, dims, th, X, perm, &L);
  colstruct_free(&cs);
  int64_t nnz = -1;
  if (fail < 0) {
    nnz = L.cp[n];
    for (int64_t j = 0, o = 0; j < n; j++)
      for (int64_t e = L.cp[j]; e < L.cp[j + 1]; e++, o++)
        if (o < cap) { ri[o] = L.ri[e]; ci[o] = (int32_t)j; v[o] = L.v[e]; }
  }
  free(L.cp); free(L.ri); free(L.v);
  return nnz;
}

/* ---------------------------------------------------------------- prediction (Sec. 3.2) */
/* mean[k] = mu*[k] + sum_j C_y(x*_k, x_j) alpha_j over all training points j (in index order); no noise term. */
void or_predict(int64_t n, int64_t m, const int* dims, const double* th, const double* X, const double* alpha,
                const double* Xt, const double* mu_t, double* mean) {
  hyp_t p = unpack(dims, th);
  double* F = (double*)malloc(sizeof(double) * (size_t)(n * (p.n1 > 0 ? p.n1 : 1)));
  or_features(n, dims, th, X, F);
  double ft[64];
  for (int64_t k = 0; k < m; k++) {
    features_one(&p, Xt + k * p.d, ft);
    double acc = 0.0;
    for (int64_t j = 0; j < n; j++) {
      double c = cy_f(&p, Xt + k * p.d, X + j * p.d, ft, F + j * p.n1);
      if (c != 0.0) acc = acc + c * alpha[j];
    }
    mean[k] = (mu_t ? mu_t[k] : 0.0) + acc;
  }
  free(F);
}

/* ---------------------------------------------------------------- C_z on a given pattern (Sec. 3.1, Eq. Zcov) */
/* val[e] = C_y(x_i, x_col[e]) + tau^2 [i = col[e]] for every entry e of row i of a CSR pattern: the matrix the
 * iterative path (stochastic Lanczos log-determinant, MINRES) multiplies by. */
void or_csr_values(int64_t n, const int* dims, const double* th, const double* X, const int64_t* rowptr,
                   const int32_t* col, double* val) {
  hyp_t p = unpack(dims, th);
  double* F = (double*)malloc(sizeof(double) * (size_t)(n * (p.n1 > 0 ? p.n1 : 1)));
  or_features(n, dims, th, X, F);
  for (int64_t i = 0; i < n; i++)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
      int64_t j = col[e];
      double v = cy_f(&p, X + i * p.d, X + j * p.d, F + i * p.n1, F + j * p.n1);
      if (i == j) v = v + p.noise_var;
      val[e] = v;
    }
  free(F);
}


/* ---------------------------------------------------------------- support of C_sparse (non-compact core) */
/* With a non-compact core (App. B) C_y(x, x') != 0 only where C_sparse(x, x') can be: q0 < 1 for the Wendland
 * radii r0 (u = x / r0 per coordinate, q0^2 as in the compact pattern), or x and x' both inside the support of one
 * bump family i (|x - h_ij|^2 < r_ij^2 for some j, and the same for x' and some j'; Eq. bumpFcn, Eq. C_sparse).
 * Structural: bumps count by their radii whatever their amplitudes. */
static int in_family(const hyp_t* p, const double* x, int i) {
  for (int j = 0; j < p->n2; j++) {
    const double* h = p->h + (size_t)(i * p->n2 + j) * p->bd;
    double s = 0.0;
    for (int k = 0; k < p->bd; k++) {
      double dk = x[k] - h[k];
      s = s + dk * dk;
    }
    double r = p->r[i * p->n2 + j];
    if (s < r * r) return 1;
  }
  return 0;
}

static int in_sparse_support(const hyp_t* p, const double* xi, const double* xj) {
  if (in_support(xi, xj, p->r0, p->d)) return 1;
  for (int i = 0; i < p->n1; i++)
    if (in_family(p, xi, i) && in_family(p, xj, i)) return 1;
  return 0;
}

int64_t or_pattern_count_sparse(int64_t n, const int* dims, const double* th, const double* X, int64_t* rowcnt) {
  hyp_t p = unpack(dims, th);
  int64_t tot = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : tot)
  for (int64_t i = 0; i < n; i++) {
    int64_t c = 0;
    for (int64_t j = 0; j < n; j++) c += in_sparse_support(&p, X + i * p.d, X + j * p.d);
    rowcnt[i] = c;
    tot += c;
  }
  return tot;
}

void or_pattern_fill_sparse(int64_t n, const int* dims, const double* th, const double* X, const int64_t* rowptr,
                            int32_t* col) {
  hyp_t p = unpack(dims, th);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; i++) {
    int64_t o = rowptr[i];
    for (int64_t j = 0; j < n; j++)
      if (in_sparse_support(&p, X + i * p.d, X + j * p.d)) col[o++] = (int32_t)j;
  }
}
