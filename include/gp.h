/*
 * gp.h -- C-ABI of libgp.so, the GB300 (sm_103a) exact Gaussian-process engine for the compactly supported
 * nonstationary kernel of arXiv 2411.05869 ("Compactly-supported nonstationary kernels for computing exact
 * Gaussian processes on big data").
 *
 * The library evaluates, for one or many hyperparameter settings theta on a fixed point set X,
 *   log p(z | beta, theta) = -1/2 log det C_z - 1/2 r^T C_z^{-1} r - n/2 log(2 pi),   r = z - W beta
 * (Sec. 3.3, first display; C_z from Eq. Zcov) and the predictive mean
 *   m* = mu* + C_{y,z} C_z^{-1} r   (Sec. 3.2, first display of m_{y|z}),
 * exactly, through a sparse supernodal Cholesky factorization of C_z. C_z = C_core * C_sparse + tau^2 I:
 *   C_sparse(x, x') = s0 f0(x, x'; r0) + sum_{i=1..n1} f_i(x) f_i(x')          (Sec. 2.1, Eq. C_sparse)
 *   f_i(x) = sum_{j=1..n2} g_ij(x),  g(x) = a exp{b [1 - (1 - |x-h|^2/r^2)^{-1}]} for |x-h| < r  (Eq. bumpFcn)
 *   f0(x, x'; r0) = (1-q)^8 (35 q^3 + 25 q^2 + 8 q + 1), q = |x-x'|/r0 < 1                     (Eq. compSupp)
 *   C_core(x, x') = core_var * f0(x, x'; core_radius): a compactly supported Wendland-type core, so the
 *   support of C_core bounds the sparsity pattern of C_z (Sec. 2, product kernel C_y = C_core x C_sparse).
 * Distances are anisotropic: q^2 = sum_k ((x_k - x'_k)/rad_k)^2 with one radius per coordinate (Sec. 5.1, 5.2).
 *
 * Conventions (all entry points):
 *   - "d_" pointers are DEVICE memory on the context's device; every other pointer is host memory.
 *   - The caller owns every buffer it passes; the library owns the opaque handles and frees them only in
 *     the matching *_free / gp_destroy. Handles are not thread-safe; use one context per host thread.
 *   - Every call is ordered on the context's CUDA stream. gp_assemble and gp_create synchronise that stream
 *     (they build host-side plans); gp_factor, gp_factor_update, gp_loglik and gp_predict are asynchronous
 *     unless documented otherwise, and their device outputs are valid once the stream reaches them.
 *   - A status is returned and never aborts; gp_last_error gives the message of the last failure.
 *   - Row-major layouts: X is n x d (point k at X[k*d .. k*d+d-1]); batched vectors are B x n.
 */
#ifndef GP_H_
#define GP_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GP_API __attribute__((visibility("default")))
#else
#define GP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GP_OK = 0,
  GP_ERR_ARG = 1,      /* bad argument (null, size, dimension, mismatched handles) */
  GP_ERR_NOMEM = 2,    /* device memory allocation failed or would exceed the context budget */
  GP_ERR_NOT_PD = 3,   /* a pivot was not positive (reported per proposal by gp_factor_info) */
  GP_ERR_CUDA = 4,     /* a CUDA runtime error */
  GP_ERR_TIMEOUT = 5,  /* a bounded device wait ran out (no kernel here spins on another) */
  GP_ERR_STATE = 6     /* call out of order (e.g. predict before loglik) */
} gp_status;

typedef enum {
  GP_FP64 = 0,         /* every step in FP64 */
  GP_MIXED = 1         /* off-diagonal supernode updates on tensor cores with FP32 accumulation, each FP32 operand
                          split into an FP16 pair (or a TF32 pair: GP_OPT_SPLIT_F16), and FP32 off-diagonal
                          storage; diagonal-block factorization, log-det and refinement residuals in FP64 (the
                          diagonal blocks optionally factored in FP32: GP_OPT_DIAG_FP32) */
} gp_precision;

typedef struct gp_ctx gp_ctx;
typedef struct gp_pointset gp_pointset;
typedef struct gp_factor_s gp_factor_t;   /* a numeric factorization (B proposals) */
typedef struct gp_symbolic gp_symbolic;   /* a host-side symbolic analysis (step A6 alone) */

/* One hyperparameter setting (host memory, FP64). Sec. 2.1 lists theta_sparse = (s0, r0, {h, a, b, r});
 * core_var / core_radius parameterise the compact core, noise_var is tau^2 of Eq. Zcov (constant).
 * h is n1*n2*bump_dims (bump (i,j) at h[(i*n2+j)*bump_dims ...]); a, b, r are n1*n2, row-major over (i,j).
 * Bumps act on the leading bump_dims coordinates (space-time: the spatial ones, Sec. 5.2). */
typedef struct {
  int d, n1, n2, bump_dims;
  double core_var;
  const double* core_radius;  /* [d] must equal the radii the point set was assembled with */
  double s0;
  const double* r0;           /* [d] Wendland radii of C_sparse; entries of C_z outside the core support are 0 */
  const double* h;
  const double* a;
  const double* b;
  const double* r;
  double noise_var;
} gp_hyper;

typedef struct {
  int64_t n;            /* points */
  int d;
  int64_t nnz;          /* nonzeros of the full symmetric pattern of C_z */
  int64_t ncells;       /* cells of the unit grid in u = x / core_radius */
  int64_t nnzL;         /* exact nonzeros of the Cholesky factor (sum of column counts) */
  int64_t nsuper;       /* relaxed supernodes */
  int64_t panel_entries;/* stored panel entries (supernodal storage incl. explicit zeros) */
  int64_t update_entries;/* peak update-matrix workspace entries (per proposal) */
  int32_t nlevels;      /* levels of the supernodal elimination tree */
  int32_t max_front;    /* largest frontal matrix order */
  double flops;         /* algorithmic factorization flops: sum over columns of eta_j^2 */
} gp_pointset_info_t;

typedef struct {
  int B;
  int precision;              /* gp_precision */
  int64_t bytes;              /* device bytes held by the factor */
  int32_t not_pd_count;       /* proposals whose factorization met a non-positive pivot */
  int32_t diag_fp32;          /* GP_MIXED: 1 if its 64 x 64 diagonal blocks are factored in FP32 (GP_OPT_DIAG_FP32) */
  int32_t timed_out;          /* 1 if a bounded wait of the last factorization or of a later solve ran out
                                 (GP_ERR_TIMEOUT) */
  int32_t split_f16;          /* GP_MIXED: 1 if its tensor-core updates take FP16 operand pairs (GP_OPT_SPLIT_F16),
                                 0 for TF32 pairs */
} gp_factor_info_t;

/* Context options (gp_set_option). They apply to the factors created on the context afterwards.
 *   GP_OPT_DIAG_FP32: 0 (default) or 1. With 1, GP_MIXED factors factor their 64 x 64 diagonal blocks in FP32
 *     from the FP64-accumulated block instead of in FP64. The blocks are accumulated in FP64 either way and the
 *     log-determinant is summed in FP64 from their diagonals; FP32 is faster on GB300 (its FP64 pipe is slow) at
 *     the cost of an FP32-accurate diagonal of L in the log-determinant.
 *   GP_OPT_WAIT_POLLS (default 2^26, 1..2^32-1) and GP_OPT_WAIT_NS (default 1e9, >= 0): the limits of every
 *     bounded wait of the GP_MIXED tensor-core kernels (an mbarrier phase awaited by one warp role from another:
 *     operand copies landed, MMAs done, accumulator drained) and of the solves' tasks in both precisions (a task
 *     awaiting a block another task of the same launch publishes). A wait that runs out after that many polls or
 *     nanoseconds records the failure in the factor and ends its wait: a tensor-core kernel winds down (after
 *     waiting, with the default limits, for the copies and MMAs it already issued) and every later tensor-core
 *     launch of that factorization skips its tiles; a solve task goes on with what it has. The factor then
 *     reports GP_ERR_TIMEOUT: gp_factor_info (timed_out = 1) and gp_loglik return it, and the log-likelihoods are
 *     NaN. No legitimate wait comes near the defaults; tiny limits make waits run out on purpose (a test of this
 *     path). The next gp_factor_update of the factor starts clean.
 *   GP_OPT_REFINE_EXP (default 10, 6..15): gp_loglik's GP_MIXED refinement stops once every proposal's FP64
 *     relative residual |r - C alpha| / |r| is at most 10^-value (or after 10 corrections). Its quadratic form is
 *     second order in that residual, so the log-likelihood does not need more; gp_predict refines alpha to 1e-12
 *     first.
 *   GP_OPT_SPLIT_F16: 1 (default) or 0: how GP_MIXED factors split each FP32 entry of L into the two parts their
 *     tensor-core updates multiply (three products per step: hi hi, hi lo, lo hi, accumulated in FP32, emulating
 *     FP32 products). 1: FP16 parts of the entry times 2^k, kind::f16 MMAs at twice the TF32 rate on half the
 *     operand bytes (hi = the scaled entry rounded to FP16, lo = the remainder rounded to FP16; k per setting from
 *     max_i C_ii, so that every scaled entry is below 2^13 -- |L_ij| <= sqrt(C_ii)); the pair holds the scaled
 *     entry to within 2^-22 of it, or 2^-25 absolute below 2^-3, and the dropped lo lo term is at most 2^-22 of a
 *     product; the products are scaled back by 2^-2k, exactly. 0: TF32 parts, kind::tf32 MMAs (hi = the entry
 *     truncated to TF32, lo = the remainder rounded to TF32): the pair holds the entry to within 2^-22 of it, the
 *     dropped lo lo term is at most 2^-20 of a product. */
typedef enum {
  GP_OPT_DIAG_FP32 = 0,
  GP_OPT_WAIT_POLLS = 1,
  GP_OPT_WAIT_NS = 2,
  GP_OPT_REFINE_EXP = 3,
  GP_OPT_SPLIT_F16 = 4
} gp_option;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream` (a cudaStream_t; NULL = the legacy
 * default stream). mem_budget_bytes caps the device memory the context's handles may hold (0 = no cap).
 * With an explicit stream the context also creates two non-blocking streams of its own; GP_MIXED
 * factorizations fork work off their chain of dependent launches onto them and join it back into the context
 * stream, so later work on that stream waits for it and the calls can be captured in a CUDA graph. The results
 * are bitwise those of the legacy default stream, where everything runs in order.
 * Errors: GP_ERR_ARG (bad device), GP_ERR_CUDA. */
GP_API gp_status gp_create(gp_ctx** ctx, int device, void* cuda_stream, size_t mem_budget_bytes);
GP_API void gp_destroy(gp_ctx* ctx);
/* Message of the last failure on this context (static storage owned by the context; "" if none). */
GP_API const char* gp_last_error(const gp_ctx* ctx);
/* Set / read a context option (gp_option). Host-only. Errors: GP_ERR_ARG (unknown option or value). */
GP_API gp_status gp_set_option(gp_ctx* ctx, int option, int64_t value);
GP_API gp_status gp_get_option(const gp_ctx* ctx, int option, int64_t* value);

/* Steps A1, A2, A5, A6: cell list of the unit grid in u = x / core_radius, exact support pattern of C_z
 * (all pairs with q^2 = sum_k (u_ik - u_jk)^2 < 1, FP64 without contraction), nested-dissection ordering and
 * symbolic analysis (etree, column counts, relaxed supernodes, frontal plan). Depends only on X and the core
 * radii, so one point set serves every theta with the same core radii (Sec. 3.3 notes the pattern of C_z
 * is otherwise theta dependent; a compact core fixes it).
 *   d_X: n x d FP64 (device), d in {1,2,3}; core_radius: host [d] > 0.
 * Synchronous. Errors: GP_ERR_ARG (n < 1, d outside 1..3, radius <= 0, grid of more than max(2^24, 8n) cells),
 * GP_ERR_NOMEM, GP_ERR_CUDA. */
GP_API gp_status gp_assemble(gp_ctx* ctx, const double* d_X, int64_t n, int d, const double* core_radius,
                      gp_pointset** ps);
GP_API void gp_pointset_free(gp_pointset* ps);
GP_API gp_status gp_pointset_info(const gp_pointset* ps, gp_pointset_info_t* info);

/* Export a structural array of the point set to host memory (for bit-exact checks):
 *   what = 0 perm[n] int32 (new -> old), 1 parent[n] int32 (etree, -1 root), 2 eta[n] int32 (column counts),
 *   3 rowptr[n+1] int64, 4 col[nnz] int32 (pattern, columns ascending), 5 sn_first[nsuper+1] int32,
 *   6 sn_rowptr[nsuper+1] int64, 7 sn_rows int32 (rows below each supernode, ascending),
 *   8 sn_parent[nsuper] int32, 9 sn_level[nsuper] int32, 10 cell_perm[n] int32 (points by (cell, index)).
 * `bytes` must equal the array size. Synchronous. Errors: GP_ERR_ARG. */
GP_API gp_status gp_pointset_export(const gp_pointset* ps, int what, void* host_dst, size_t bytes);

/* Step A6 alone, on the host: the symbolic analysis gp_assemble runs on the device pattern (postorder
 * relabelling of the elimination tree, etree by Liu's algorithm, exact column counts, fundamental and relaxed
 * supernodes, supernodal row structures and levels, and the frontal plan), here from a caller's host pattern
 * and nested-dissection order, with no device call. The analysis of the paper's exact sparse Cholesky, named in
 * its Discussion; the structure rules are those of gp_assemble.
 *   rowptr[n+1] int64 (rowptr[0] = 0, non-decreasing), col[rowptr[n]] int32: the symmetric pattern of C_z, both
 *   triangles and the diagonal, columns strictly ascending in each row, all in 0..n-1;
 *   nd_perm[n] int32: a permutation (new -> old), the order before the postorder relabelling.
 * The caller keeps ownership of its arrays (read during the call only); *out is freed with gp_symbolic_free.
 * Synchronous. Errors: GP_ERR_ARG (n outside 1..2^31-2, a malformed pattern or permutation, null pointers),
 * GP_ERR_NOMEM, GP_ERR_STATE (inconsistent analysis, e.g. an unsymmetric pattern). */
GP_API gp_status gp_symbolic_host(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* nd_perm,
                                  gp_symbolic** out);
/* The analysis' sizes in a gp_pointset_info_t (d = 0, ncells = 0; nnz = rowptr[n]). Errors: GP_ERR_ARG. */
GP_API gp_status gp_symbolic_info(const gp_symbolic* sym, gp_pointset_info_t* info);
/* Export one of its arrays to host memory; `what` as for gp_pointset_export, the analysis' arrays only (0, 1, 2,
 * 5, 6, 7, 8, 9); `bytes` must equal the array size. Errors: GP_ERR_ARG. */
GP_API gp_status gp_symbolic_export(const gp_symbolic* sym, int what, void* host_dst, size_t bytes);
GP_API void gp_symbolic_free(gp_symbolic* sym);

/* ----------------------------------------------------------------------------- non-compact core (App. B)
 * The core kernel of a setting (Sec. 2.2: any PSD kernel may serve as C_core). gp_hyper alone describes the compact
 * Wendland-type core core_var f0(q; core_radius), whose support bounds the pattern. GP_CORE_PACIOREK selects the
 * parametric nonstationary Matern core of App. B (Eq. PScov), locally isotropic with smoothness 3/2:
 *   C_core(x, x') = sigma(x) sigma(x') (Sigma(x) Sigma(x'))^(d/4) / ((Sigma(x) + Sigma(x')) / 2)^(d/2) M(sqrt(Q)),
 *   Q = |x - x'|^2 / ((Sigma(x) + Sigma(x')) / 2), M(t) = (1 + sqrt(3) t) exp(-sqrt(3) t),
 *   log sigma(x) = log sigma0 + sum_k phi_sigma[k] x_k,  log Sigma(x) = log Sigma0 + sum_k phi_Sigma[k] x_k
 * (the coordinates as the basis functions; core_var and core_radius of gp_hyper are then unused). This core is
 * nowhere zero, so C_z is zero only outside the support of C_sparse (Eq. C_sparse): pairs with q0 < 1 for the radii
 * r0, or with both points inside the support of one bump family (|x - h_ij| < r_ij for some j). That support depends
 * on r0 and the bumps' centres and radii: the point set is assembled for them (gp_assemble_sparse_support) and
 * serves every setting with the same r0, n1, n2, bump_dims, h and r (amplitudes, shapes, s0, noise and the core's
 * parameters may vary). */
typedef enum { GP_CORE_WENDLAND = 0, GP_CORE_PACIOREK = 1 } gp_core_kind;
typedef struct {
  int32_t kind;               /* gp_core_kind */
  double sigma0, Sigma0;      /* baseline signal standard deviation and squared length scale (> 0) */
  const double* phi_sigma;    /* [d] host */
  const double* phi_Sigma;    /* [d] host */
} gp_core;

/* Steps A1, A2, A5, A6 with the support of C_sparse as the pattern (the non-compact core): pairs with
 * sum_k (u_ik - u_jk)^2 < 1 for u = x / r0 (as gp_assemble computes it with core_radius = r0), or both points inside
 * one bump family (sum over the leading bump_dims coordinates of (x_k - h_k)^2 < r^2 for some bump of the family,
 * each operation rounded separately, in coordinate order). theta: host; its r0, n1, n2, bump_dims, h and r define
 * the support. Synchronous. Errors: as gp_assemble; GP_ERR_ARG also for n1 > 32. */
GP_API gp_status gp_assemble_sparse_support(gp_ctx* ctx, const double* d_X, int64_t n, int d, const gp_hyper* theta,
                                            gp_pointset** ps);

/* Steps A3, A4, A7 for B proposals sharing the point set: bump features, kernel values of the pattern
 * (fused with the scatter into supernodal panels) and the supernodal numeric Cholesky of P C_z P^T.
 * thetas: host array of B settings. Allocates the factor (B copies of the panels plus workspace).
 * A non-positive pivot does not fail the call: it marks that proposal (gp_factor_info, and gp_loglik then
 * returns -inf for it). With TF32 operand pairs (GP_OPT_SPLIT_F16 = 0) GP_MIXED stores only the low half of each
 * pair and lets the MMA read the high half from the FP32 factor, which needs TF32 MMAs that truncate FP32
 * operands: the first such factor on a device checks that with one small MMA (and synchronises the stream once).
 * Errors: GP_ERR_ARG, GP_ERR_NOMEM, GP_ERR_CUDA, GP_ERR_STATE (TF32 pairs on a GPU whose TF32 MMAs round instead
 * of truncating). Asynchronous after allocation. */
GP_API gp_status gp_factor(gp_ctx* ctx, gp_pointset* ps, const gp_hyper* thetas, int B, gp_precision precision,
                    gp_factor_t** f);
/* Re-run A3, A4, A7 on an existing factor with B new settings (same B, precision and point set): the
 * allocation-free inner call of an MCMC loop. Asynchronous. Errors: GP_ERR_ARG, GP_ERR_CUDA. */
GP_API gp_status gp_factor_update(gp_ctx* ctx, gp_factor_t* f, const gp_hyper* thetas);
/* gp_factor / gp_factor_update with a core per setting (cores: host array of B, NULL = the compact Wendland core
 * of gp_hyper for all). The point set's support must fit the core: GP_CORE_WENDLAND on gp_assemble point sets,
 * GP_CORE_PACIOREK on gp_assemble_sparse_support point sets with the settings' r0, h and r equal to the ones it was
 * assembled with (GP_ERR_ARG otherwise). All B settings take the same kind. */
GP_API gp_status gp_factor_core(gp_ctx* ctx, gp_pointset* ps, const gp_hyper* thetas, const gp_core* cores, int B,
                                gp_precision precision, gp_factor_t** f);
GP_API gp_status gp_factor_update_core(gp_ctx* ctx, gp_factor_t* f, const gp_hyper* thetas, const gp_core* cores);
GP_API void gp_factor_free(gp_factor_t* f);
/* Synchronous (reads the per-proposal pivot flags). Returns GP_ERR_TIMEOUT, with info filled in and timed_out set,
 * if a bounded device wait of the factorization ran out (GP_OPT_WAIT_POLLS). */
GP_API gp_status gp_factor_info(const gp_factor_t* f, gp_factor_info_t* info, int32_t* not_pd_column /* [B] or NULL */);

/* Steps A8-A11: forward/backward supernodal solves, quadratic form r^T C_z^{-1} r, log-determinant
 * 2 sum_j log L_jj in a fixed-order tree, and (GP_MIXED) FP64 iterative refinement of alpha = C_z^{-1} r with
 * residuals from the FP64 CSR matrix, until |r - C alpha| / |r| <= 1e-10 (GP_OPT_REFINE_EXP) or 10 sweeps, and the
 * quadratic form r^T C_z^{-1} r as alpha^T (2 r - C_z alpha) in FP64 (exact to second order in the residual).
 *   d_resid: B x n FP64 (r = z - mu per proposal, original point order); d_out: B FP64 log-likelihoods
 *   (-inf for proposals with a non-positive pivot, NaN after a timed-out factorization); d_err_est: B FP64 final
 *   relative residual (nullable).
 * Keeps alpha for gp_predict. Asynchronous on an explicit stream: the refinement's stopping test runs on the
 * device (the whole refinement is one CUDA graph with a conditional loop). On the legacy default stream (NULL at
 * gp_create) GP_MIXED runs the refinement loop from the host and synchronises at each sweep.
 * Errors: GP_ERR_ARG, GP_ERR_CUDA; GP_ERR_TIMEOUT on the legacy default stream when the factorization's bounded
 * waits ran out (on an explicit stream that shows as NaN outputs and in gp_factor_info). */
GP_API gp_status gp_loglik(gp_ctx* ctx, gp_factor_t* f, const double* d_resid, double* d_out, double* d_err_est);

/* Step A12: m*_k = mu*_k + sum_j C_y(x*_k, x_j) alpha_j over the training neighbours of x*_k found in the
 * cell list (no noise term; Sec. 3.2), for proposal b of the factor, after gp_loglik.
 *   d_Xtest: m x d FP64; d_mu_test: m FP64 or NULL (zero mean); d_mean: m FP64 output.
 * GP_MIXED: the first prediction after a gp_loglik refines alpha (all proposals) to a relative residual of 1e-12
 * if gp_loglik stopped above it (the same corrections, on the device).
 * Asynchronous. Errors: GP_ERR_ARG, GP_ERR_STATE (no alpha yet), GP_ERR_CUDA. */
GP_API gp_status gp_predict(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_Xtest, int64_t m,
                     const double* d_mu_test, double* d_mean);

/* Predictive variance (Sec. 3.2): the diagonal of the conditional covariance C_{y|z} = C_y - C_{y,z} C_z^{-1} C_{z,y}
 * at the test inputs, var_k = C_y(x*_k, x*_k) - |w_k|^2 with L w_k = P c_k and c_k = C_y(X, x*_k) (no noise term at
 * test inputs), for proposal b of the factor (gp_loglik is not needed). c_k is nonzero only at the training
 * neighbours of x*_k, so w_k is formed by a forward solve restricted to the supernodes on those neighbours' paths to
 * the root, 32 test points at a time; test points close in space that are passed next to each other share that
 * work. The arithmetic is the factor's: FP64 for GP_FP64; FP32 solves with the FP32 panels for GP_MIXED (relative
 * accuracy of the mixed factor, about 1e-6 of C_y(x*, x*)).
 *   d_Xtest: m x d FP64 (device); d_var: m FP64 (device output).
 * The first call on a factor allocates its workspace (at most 4 GiB or a quarter of the free device memory, within
 * the context budget), held until gp_factor_free; later calls allocate nothing. Asynchronous after that allocation.
 * Errors: GP_ERR_ARG, GP_ERR_NOMEM, GP_ERR_CUDA. */
GP_API gp_status gp_predict_var(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_Xtest, int64_t m, double* d_var);

/* The paper's own approximate computation of the log-likelihood above 100k points (Sec. 3.3), as a comparison for
 * the exact factorization: log det C_z by stochastic Lanczos quadrature (k Lanczos steps from each of P probe
 * vectors, no reorthogonalisation: log det ~ (1/P) sum_p |v_p|^2 sum_i U_1i^2 log theta_i for T_k = U diag(theta)
 * U^T) and r^T C_z^{-1} r by MINRES (Paige and Saunders) from a start vector, stopped when the residual estimate
 * falls to tol |r|; log p ~ -1/2 log det - 1/2 r^T alpha - n/2 log 2 pi. It multiplies by the CSR values of C_z the
 * factor's value step computed for proposal b (the factorization itself is not used).
 *   d_resid: n FP64 (device, r = z - mu); d_probes: P x n FP64 (device; the probe vectors, e.g. +-1 entries as the
 *   paper draws them); d_x0: n FP64 (device; MINRES start, the paper starts at random) or NULL for zero.
 * The first call on a factor allocates its workspace (3 n P + 7 n doubles), held until gp_factor_free.
 * Synchronous (the result is host memory). Errors: GP_ERR_ARG (P outside 1..32, k outside 2..64, tol <= 0,
 * max_iter < 1), GP_ERR_NOMEM, GP_ERR_CUDA. */
typedef struct {
  int32_t probes;          /* P, 1..32 */
  int32_t lanczos_steps;   /* k, 2..64 */
  double tol;              /* MINRES relative residual tolerance (the paper: 1e-8) */
  int32_t max_iter;        /* MINRES iteration cap */
} gp_iterative_opts;
typedef struct {
  double loglik, logdet, quad;   /* estimates */
  int32_t minres_iters;
  int32_t converged;             /* 1 if MINRES reached tol within max_iter */
  double minres_relres;          /* MINRES's own residual estimate / |r| */
  double true_relres;            /* |r - C_z alpha| / |r| recomputed from the result */
} gp_iterative_result;
GP_API gp_status gp_loglik_iterative(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_resid,
                                     const double* d_probes, const double* d_x0, const gp_iterative_opts* opts,
                                     gp_iterative_result* result);

/* Launch profiler. gp_profile(ctx, 1) clears the counters and brackets every later launch of the listed
 * kernel classes with CUDA events on the context stream; gp_profile(ctx, 0) stops. gp_profile_read
 * synchronises the stream and returns, for one class, the summed device time (ms), the launch count and the
 * useful flops those launches performed (0 where no flop count applies). Classes:
 *   0 A4 kernel values, 1 A7 extend-add (GP_MIXED: with the zeroing of the update matrices), 2 A7 small
 *   fronts, 3 A7 diagonal-block POTRF, 4 A7 TRSM, 5 A7 trailing update (SYRK/GEMM; with GP_MIXED the
 *   group-end updates), 6 A8-A10 solve sweep (one span per gp_loglik), 7 A12 prediction, 8 A1-A6 assembly,
 *   9 A7 left-looking block-column updates (GP_MIXED).
 * Errors: GP_ERR_ARG (class out of range), GP_ERR_CUDA. */
GP_API gp_status gp_profile(gp_ctx* ctx, int enable);
GP_API gp_status gp_profile_read(gp_ctx* ctx, int kclass, double* total_ms, int64_t* launches, double* flops);
/* The same, restricted to the launches a factorization issued for elimination-tree level `level` (0 = the
 * leaves' level, as gp_pointset_export's sn_level numbers them; 0 <= level < 64). Classes 1-5 and 9 are issued per
 * level; the others read 0. Errors: GP_ERR_ARG (class or level out of range), GP_ERR_CUDA. */
GP_API gp_status gp_profile_read_level(gp_ctx* ctx, int kclass, int level, double* total_ms, int64_t* launches);

/* Support-pattern row counts without any device allocation (the paper has no counterpart: this serves
 * callers that must not allocate device memory, such as code running under another framework's memory
 * allocator or a memory budget it does not own, that want each point's neighbour count, e.g. to size their
 * own buffers or to pick core radii for a target row count before calling gp_assemble).
 *   d_X: n x d FP64 (device); core_radius: host [d]; d_counts: n int64 (device output), d_counts[i] = number
 *   of points j (i included) with sum_k (u_ik - u_jk)^2 < 1 for u = x / core_radius per coordinate (each division,
 *   difference, product and sum rounded separately, summed in coordinate order), the row lengths of the pattern
 *   gp_assemble builds for the same input.
 * It runs the cell list and count pass of gp_assemble with all scratch in one static device array of 16 MiB
 * that every GPU loading the library keeps until exit: n <= 65536 and at most 2^20 cells of the unit grid in
 * x / core_radius (GP_ERR_ARG beyond). It calls no cudaMalloc/cudaFree. The first call on a device looks up
 * the array's device address; make that first call before any stream capture. Calls share the array, so
 * calls that overlap on the GPU race. Synchronises the context stream once (for the grid extent).
 * Errors: GP_ERR_ARG, GP_ERR_CUDA. */
GP_API gp_status gp_pattern_counts_noalloc(gp_ctx* ctx, const double* d_X, int64_t n, int d, const double* core_radius,
                                           int64_t* d_counts);

/* Number of kernel launches this context has issued (a counter for launch accounting). The passes of the mixed
 * refinement loop, decided on the device, are added when gp_factor_info next reads the factor. */
GP_API int64_t gp_launch_count(const gp_ctx* ctx);

/* Device bytes gp_factor allocates for B settings of `theta`'s shape on point set ps in precision prec (the
 * memory a caller or a server admits against). Host-only. Errors: GP_ERR_ARG. */
GP_API gp_status gp_factor_bytes(const gp_pointset* ps, const gp_hyper* theta, int B, gp_precision prec,
                                 size_t* bytes);

/* Build the per-precision maps of a point set (GP_MIXED: the CSR -> FP32 panel / FP64 tile map) now, on the
 * point set's context, instead of inside the first gp_factor of that precision. A point set may serve
 * factors created on other contexts of the same device (each context its own stream and host thread); prepare
 * it first when such factors can be created concurrently. Synchronous. Errors: GP_ERR_ARG, GP_ERR_NOMEM. */
GP_API gp_status gp_pointset_prepare(gp_ctx* ctx, gp_pointset* ps, gp_precision prec);

/* Autotuner of the mixed path's supernode update tiles (the paper has no counterpart: it is a performance choice
 * of this implementation, not of the method). Large fronts are factored 64 columns at a time; the trailing
 * updates of a group of G such blocks are deferred and applied at the group's end as 128 x TN tensor-core
 * tiles with K = 64 G. For each candidate (G, TN) in {4, 8, 16} x {128, 256} and (32, 256) the point set's update
 * schedule is
 * re-planned, a GP_MIXED factor of B settings is created and gp_factor_update timed `reps` times (CUDA events on
 * the context stream); the fastest candidate stays planned for the point set's later factors (results differ
 * between candidates only by the order of FP32 sums). tried (nullable, room for 7) receives the candidates with
 * their mean time per factorization, *ntried their count. Must run before any factor of the point set exists;
 * on failure the default blocking (G = 8, TN = 256) is planned again.
 * Errors: GP_ERR_ARG, GP_ERR_STATE (factors exist), GP_ERR_NOMEM, GP_ERR_CUDA. */
typedef struct {
  int32_t group_blocks;   /* G */
  int32_t group_tile_n;   /* TN */
  double ms;              /* mean time of one factorization (A3, A4, A7) */
} gp_tune_candidate;
GP_API gp_status gp_autotune(gp_ctx* ctx, gp_pointset* ps, const gp_hyper* thetas, int B, int reps,
                             gp_tune_candidate* tried, int* ntried);
/* Plan a given update blocking (G in 1..64, TN in {128, 256}) for the point set's later GP_MIXED factors
 * (what gp_autotune does with its choice). Errors: GP_ERR_ARG, GP_ERR_STATE (factors exist). */
GP_API gp_status gp_pointset_set_blocking(gp_ctx* ctx, gp_pointset* ps, int group_blocks, int group_tile_n);

/* ----------------------------------------------------------------------------------------- request server
 * A continuous-batching server of log-likelihood (Sec. 3.3) and predictive-mean (Sec. 3.2) requests on one GPU.
 * The paper has no counterpart (it evaluates one likelihood at a time across many GPUs); this is the serving
 * layer over the same hot path. Point sets are added once (A1, A2, A5, A6 cached). Requests of uneven sizes
 * queue in arrival order; `slots` worker threads, each with its own context and CUDA stream, admit the head
 * request when it fits: a slot re-uses an idle factor it holds for the same point set and precision (values
 * and factorization recomputed for the new theta, no allocation), or creates one if its bytes
 * (gp_factor_bytes) fit mem_budget_bytes after evicting idle cached factors, least recently used first.
 * Requests run concurrently on the slots' streams; a result does not depend on what else runs.
 * All device buffers of a request are the caller's and must stay valid until its completion is polled. */
typedef struct gp_server_s gp_server_t;

typedef enum { GP_REQ_LOGLIK = 0, GP_REQ_PREDICT = 1 } gp_request_kind;

typedef struct {
  int kind;                 /* gp_request_kind */
  int32_t pointset;         /* id from gp_server_add_pointset */
  gp_precision precision;
  const gp_hyper* theta;    /* host; copied at submission */
  const double* d_resid;    /* n (device): r = z - mu of the point set's points */
  const double* d_Xtest;    /* m x d (device), GP_REQ_PREDICT */
  int64_t m;                /* test points, GP_REQ_PREDICT */
  const double* d_mu_test;  /* m (device) or NULL, GP_REQ_PREDICT */
  double* d_out;            /* device: 1 log-likelihood (GP_REQ_LOGLIK) or m predictive means (GP_REQ_PREDICT) */
  double* d_err;            /* device or NULL: 1 relative residual |r - C alpha| / |r| */
} gp_request;

typedef struct {
  int64_t id;               /* from gp_server_submit */
  gp_status status;
  int32_t slot;             /* worker that ran it */
  double t_submit, t_start, t_done;   /* seconds on the host's monotonic clock */
} gp_completion;

typedef struct {
  size_t budget, held, peak;          /* factor bytes: budget, reserved or held now, largest held */
  int32_t cached_factors, queued, running, max_running;
  int64_t completed;
} gp_server_stats_t;

/* slots in 1..64; mem_budget_bytes caps the bytes of the factors the server holds (point sets not included).
 * Errors: GP_ERR_ARG, GP_ERR_CUDA. */
GP_API gp_status gp_server_create(int device, int slots, size_t mem_budget_bytes, gp_server_t** out);
/* gp_assemble + gp_pointset_prepare(GP_MIXED) on the server's own context; *id numbers point sets from 0.
 * Synchronous. Errors as gp_assemble. */
GP_API gp_status gp_server_add_pointset(gp_server_t* s, const double* d_X, int64_t n, int d,
                                        const double* core_radius, int32_t* id);
/* Queue a request (non-blocking). Errors: GP_ERR_ARG (bad fields or point set id), GP_ERR_NOMEM (its factor
 * alone exceeds the budget: it could never run). */
GP_API gp_status gp_server_submit(gp_server_t* s, const gp_request* req, int64_t* id);
/* Move up to max completions (in completion order) to out; returns how many (non-blocking). */
GP_API int gp_server_poll(gp_server_t* s, gp_completion* out, int max);
/* Block until the queue is empty and no request runs; timeout_s <= 0 waits without limit.
 * Errors: GP_ERR_TIMEOUT. */
GP_API gp_status gp_server_wait(gp_server_t* s, double timeout_s);
GP_API gp_status gp_server_stats(gp_server_t* s, gp_server_stats_t* stats);
GP_API const char* gp_server_last_error(const gp_server_t* s);
/* Stops the workers after their current requests (queued requests are dropped) and frees everything. */
GP_API void gp_server_destroy(gp_server_t* s);

#ifdef __cplusplus
}
#endif
#endif /* GP_H_ */
