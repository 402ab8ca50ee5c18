// gp_internal.cuh -- shared declarations of the GB300 exact sparse-GP library (libgp.so).
//
// Step map (the hot path, in order):
//   A1 cell list            assemble.cu  (u = x / core_radius, cell keys, radix sort, cell ranges)
//   A2 support pattern      assemble.cu  (neighbour cells, q^2 < 1 without contraction, CSR rows ascending)
//   A5 nested dissection    assemble.cu  (level-synchronous geometric bisection with one-sided separators)
//   A6 symbolic analysis    symbolic.cpp (etree, column counts, relaxed supernodes, frontal plan)
//   A3/A4 kernel values     values.cu    (bump features, C_z entries fused with the scatter into panels)
//   A7 numeric factor       factor.cu    (level-by-level multifrontal supernodal Cholesky)
//   A8-A11 solves           solve.cu     (forward/backward supernodal solves, log-det, refinement)
//   A12 predictive mean     predict.cu
#pragma once
#include <atomic>
#include <mutex>

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gp.h"
#include "tc_gemm.cuh"

#define GP_MAX_D 3
#define GP_MAX_N1 32
#define GP_ND_LEAF 64          // nested-dissection leaves hold at most this many points
#define GP_RELAX_WIDTH 16      // relaxed amalgamation: merge when the merged supernode is this narrow
#define GP_TILE 64             // dense tile edge of the large-front kernels
#define GP_SMALL_M 96          // fronts up to this order are factored by one CTA in shared memory
#define GP_EA_CHUNK 8192       // update-matrix entries per CTA of the mixed path's extend-add and zeroing
#define GP_FLOW_SB_MIN_NB 16   // levels whose largest front has this many 64-column blocks: 2 per solve chain task

// ------------------------------------------------------------------------------------------ errors
struct GpError {
  gp_status st;
  std::string msg;
};

#define GP_CUDA(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      throw GpError{GP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};            \
  } while (0)

#define GP_CHECK_LAUNCH(ctx)                                                                     \
  do {                                                                                           \
    cudaError_t e_ = cudaGetLastError();                                                         \
    if (e_ != cudaSuccess)                                                                       \
      throw GpError{GP_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)};      \
    (ctx)->launches++;                                                                           \
  } while (0)

#define GP_REQUIRE(cond, what)                                                                   \
  do {                                                                                           \
    if (!(cond)) throw GpError{GP_ERR_ARG, what};                                                \
  } while (0)

// ------------------------------------------------------------------------------------------ context
// Kernel classes timed by the optional launch profiler (gp_profile / gp_profile_read).
constexpr int GP_PROF_LEVELS = 64;   // levels the profiler resolves (deeper levels are counted in the totals only)
enum KClass { KC_VALUES = 0, KC_EXTEND_ADD, KC_FRONT_SMALL, KC_POTRF, KC_TRSM, KC_UPDATE, KC_SOLVE, KC_PREDICT,
              KC_ASSEMBLE, KC_UPDATE_LEFT, KC_COUNT };

struct gp_ctx {
  int device = 0;
  int nsm = 1;           // streaming multiprocessors of the device
  cudaStream_t stream = nullptr;
  // a second stream for work the factorization overlaps with its level chain (explicit streams only), and the
  // two events that fork it from and join it back to `stream` (re-recorded at each use)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // a third stream, for the left-looking updates of the rows below a block step's diagonal tiles beside the step's
  // POTRF (GP_MIXED), with its own fork and join events
  cudaStream_t side2 = nullptr;
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  size_t budget = 0;     // 0 = unlimited
  std::atomic<size_t> held{0};   // bytes currently held by this context's handles
  int64_t launches = 0;
  std::string err;
  std::atomic<int64_t> live{0};  // point sets and factors still holding this context
  bool destroyed = false;    // gp_destroy was called; the context goes with its last handle
  // launch profiler: CUDA events around every launch of a class, on the context stream
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[KC_COUNT];
  double prof_ms[KC_COUNT] = {};
  int64_t prof_n[KC_COUNT] = {};
  double prof_flops[KC_COUNT] = {};
  cudaEvent_t prof_open = nullptr;
  // the same by elimination-tree level for the factorization's classes (prof_level: the level whose launches
  // are being issued, -1 outside the level loop)
  int prof_level = -1;
  std::vector<int> prof_lv[KC_COUNT];
  double prof_ms_lv[KC_COUNT][GP_PROF_LEVELS] = {};
  int64_t prof_n_lv[KC_COUNT][GP_PROF_LEVELS] = {};
  // options (gp_set_option); they apply to factors created afterwards
  int opt_diag_fp32 = 0;     // GP_MIXED: diagonal blocks factored in FP32
  int opt_split_f16 = 1;     // GP_MIXED: FP16 operand pairs for the tensor-core updates (0: TF32 pairs)
  tcg::WaitLimit opt_wait = tcg::DEFAULT_WAIT;   // GP_MIXED: limits of the tensor-core kernels' bounded waits
  int opt_refine_exp = 10;   // GP_MIXED: gp_loglik's refinement stops at |r - C alpha| / |r| <= 10^-opt_refine_exp
  ~gp_ctx() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
    if (ev_fork2) cudaEventDestroy(ev_fork2);
    if (ev_join2) cudaEventDestroy(ev_join2);
    if (side2) cudaStreamDestroy(side2);
  }
};

// RAII timer of one launch (no-op unless profiling); `flops` is the useful work the launch performs.
struct ProfScope {
  gp_ctx* c;
  int cls;
  ProfScope(gp_ctx* ctx, int k, double flops = 0.0) : c(ctx), cls(k) {
    if (!c->prof) return;
    cudaEvent_t a;
    cudaEventCreate(&a);
    cudaEventRecord(a, c->stream);
    c->prof_open = a;
    c->prof_flops[k] += flops;
  }
  ~ProfScope() {
    if (!c->prof) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, c->stream);
    c->prof_ev[cls].push_back({c->prof_open, b});
    c->prof_lv[cls].push_back(c->prof_level);
    c->prof_n[cls]++;
  }
};

// Clears the profiler's current level when a factorization's level loop ends (normally or by an exception).
struct ProfLevelScope {
  gp_ctx* c;
  explicit ProfLevelScope(gp_ctx* ctx) : c(ctx) {}
  ~ProfLevelScope() { c->prof_level = -1; }
};

// Device buffer owned by a handle; charged against the context budget.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};
void* dev_alloc(gp_ctx* ctx, std::vector<DevBuf>& owner, size_t bytes);
void dev_free_all(gp_ctx* ctx, std::vector<DevBuf>& owner);
template <class T>
T* dalloc(gp_ctx* ctx, std::vector<DevBuf>& owner, size_t count) {
  return static_cast<T*>(dev_alloc(ctx, owner, count * sizeof(T)));
}
template <class T>
void h2d(gp_ctx* ctx, T* dst, const T* src, size_t count) {
  GP_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
}
template <class T>
void d2h(gp_ctx* ctx, T* dst, const T* src, size_t count) {
  GP_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
}

// ------------------------------------------------------------------------------------------ symbolic plan
// Host-side result of A6, plus the device copies the numeric kernels read.
#define GP_GROUP 8   // default 64-column blocks per deferred-update group of the mixed path
#define GP_TN_LEFT 64     // tensor-core tile width (columns) of the mixed path's left-looking block updates
#define GP_TN_GROUP 256   // default tile width of its group-end updates (rows stay 128 per tile)

struct SymPlan {
  int64_t n = 0;
  int64_t ns = 0;                    // supernodes
  int32_t nlevels = 0;
  std::vector<int32_t> perm;         // final order: nested dissection relabelled by its etree postorder
  std::vector<int32_t> parent, eta;  // etree and exact column counts (permuted columns)
  std::vector<int32_t> sn_first;     // ns+1
  std::vector<int64_t> sn_rowptr;    // ns+1 into sn_rows
  std::vector<int32_t> sn_rows;      // rows strictly below each supernode (ascending)
  std::vector<int32_t> sn_parent, sn_level;
  std::vector<int32_t> sn_w, sn_r;   // width, rows below
  std::vector<int64_t> sn_loff;      // panel offset (column-major m x w, ld m)
  std::vector<int64_t> sn_uoff;      // update-matrix offset (r x r column-major)
  std::vector<int64_t> sn_frow;      // offset of the front row list (m entries: own columns then sn_rows)
  std::vector<int32_t> frows;        // concatenated front rows
  std::vector<int32_t> ch_ptr, ch_idx;        // children (ascending) of each supernode
  std::vector<int64_t> relidx_off;   // per supernode: offset of its r relative indices into the parent front
  std::vector<int32_t> relidx;
  std::vector<int32_t> lev_ptr, lev_sn;       // supernodes grouped by level (ascending index within)
  std::vector<int32_t> sn_of_col;    // supernode of each permuted column
  int64_t nnzL = 0;
  int64_t panel_entries = 0;
  int64_t update_entries = 0;        // peak of the update-matrix memory plan
  int64_t vec_update_entries = 0;    // sum of r over supernodes (solve update vectors)
  double flops = 0.0;
  int32_t max_front = 0;
  // mixed-precision layout: FP32 panels row-major (m x ldw, ldw = w rounded up to 4, 16-byte aligned rows),
  // FP64 64 x 64 diagonal tiles (row-major), FP32 update matrices (row-major r x r)
  std::vector<int32_t> sn_ldw;
  std::vector<int64_t> sn_loff32, sn_doff;
  int64_t panel32_entries = 0, diag_entries = 0;
  // the tensor-core operands of the large fronts' factored panel entries, at sn_lo_off in a per-level workspace
  // of lo_entries 4-byte entries (the largest level's total; a multiple of 8), m x ldh per front (ldh = ldw
  // rounded up to 8). TF32 split: the low parts (lo = x - the TF32 truncation of x, row stride ldw; the high part
  // is the FP32 panel itself, whose low 13 mantissa bits the TF32 MMAs ignore). FP16 split: the scaled FP16
  // high parts (m x ldh halves) followed by the FP16 low parts (m x ldh halves).
  std::vector<int64_t> sn_lo_off;
  int64_t lo_entries = 8;
  int group = GP_GROUP, tn_group = GP_TN_GROUP;   // mixed-path update blocking (plan_mixed_updates)
  std::vector<int32_t> upd_fronts;   // per step: fronts of the left-looking and of the group update
  std::vector<int64_t> upd_pre;      // their tile prefixes

  // schedule for the numeric factorization, per level
  struct EaLaunch { int64_t tab_off; int64_t ncta; };            // extend-add: CTAs of one child slot
  struct StepLaunch { int64_t fr_off; int32_t nfront; int32_t kb; int64_t trsm_total; int64_t upd_total; int64_t pre_off;
                      // forward solve, steps taken in pairs (set on the first step of a pair): the tile prefix
                      // over this step's fronts, its total, and how many of them also have block kb + 1
                      int64_t pair_pre_off, pair_total; int32_t pair_n2;
                      // mixed path, (64 GP_GROUP)-column groups: left-looking update of this block column
                      // (rows >= c0 x its 64 columns, K = the group's earlier blocks) and, at a group's last block,
                      // the deferred group update (rows/columns after the group, K = the group's width); fronts
                      // and tile prefixes of each
                      int64_t left_off, left_pre_off, left_total; int32_t n_left;
                      // the same left update without the strip's first 128-row tile of each front (the rows of
                      // the step's diagonal tiles): prefix of the other tiles, and their total
                      int64_t lrest_pre_off, lrest_total;
                      int64_t group_off, group_pre_off, group_total; int32_t n_group;
                      double left_flops, group_flops;
                      double left2_flops;   // the left update of block columns kb and kb + 1 together
                      double potrf_flops, trsm_flops, upd_flops; };   // useful flops of the step's launches
  struct Level {
    std::vector<EaLaunch> ea;        // one per child slot
    std::vector<EaLaunch> ea32;      // the same in chunks of GP_EA_CHUNK update-matrix entries (mixed path)
    int64_t zero_off = 0, zero_n = 0; // into zero_tab: this level's update matrices in chunks (mixed path)
    int64_t small_off = 0; int32_t nsmall = 0;   // into small_list
    std::vector<StepLaunch> steps;   // large fronts, one per block column
    int32_t flow_sb = 1;             // 64-column blocks per chain task of this level's solve tasks (1 or 2)
  };
  std::vector<Level> levels;
  std::vector<int2> ea_tab;          // (child supernode, first column) per extend-add CTA (8 columns each)
  // mixed path: (child supernode, chunk) per extend-add CTA and (supernode, chunk) per zeroing CTA, a chunk being
  // GP_EA_CHUNK consecutive entries of the lower triangle of the update matrix in row order
  std::vector<int2> ea32_tab, zero_tab;
  std::vector<int32_t> small_list;   // supernodes factored in shared memory
  std::vector<int32_t> large_fronts; // per step: fronts (sorted by width descending within a level)
  std::vector<int32_t> large_kb;     // block-column index of each large_fronts entry (its step)
  struct LevelLarge { int64_t off = 0; int64_t count = 0; };    // all steps' entries of a level, contiguous
  std::vector<LevelLarge> level_large;
  std::vector<int64_t> step_pre;     // per step: prefix of TRSM tasks then of UPDATE tasks (2*(nfront+1))
  std::vector<int64_t> pair_pre;     // per step pair: prefix of the paired forward-solve row tiles
  // Solves of the large fronts as one launch per level (tasks that wait for the blocks they need), with SB =
  // the level's flow_sb blocks per chain task and nbs = ceil(nb / SB) chain tasks per front:
  //   flow_fwd: per level, the forward tasks (front, k): k < nbs the block rows SB k + [0, SB), k >= nbs the
  //     (64 SB)-row tile k - nbs of the rows below the front's columns;
  //   flow_bwd: per level, the backward tasks (front, k): the block columns SB k + [0, SB);
  //   sn_fl: first readiness flag of each large front (one per 64-column block; -1 for small fronts).
  // Every task waits only for tasks earlier in its list.
  std::vector<int2> flow_fwd, flow_bwd;
  std::vector<int32_t> sn_fl;
  int64_t n_fl = 0;
  std::vector<int64_t> flow_fwd_ptr, flow_bwd_ptr;   // nlevels + 1
};

// Device mirror of the plan (pointers into one allocation set owned by the point set).
struct DevPlan {
  int32_t *w, *r;
  int64_t *loff, *uoff, *frow_off;
  int32_t* frows;
  int32_t *ch_ptr, *ch_idx;
  int64_t* relidx_off;
  int32_t* relidx;
  int32_t* sn_first;
  int32_t* sn_of_col;
  int2* ea_tab;
  int2 *ea32_tab, *zero_tab;
  int32_t* small_list;
  int32_t* large_fronts;
  int64_t* step_pre;
  int32_t* lev_sn;
  int32_t* sn_parent;
  int32_t* ldw;
  int64_t *loff32, *doff;
  int64_t* lo_off;
  int32_t* large_kb;
  int32_t* upd_fronts;
  int64_t* upd_pre;
  int64_t* pair_pre;
  int32_t* sn_fl;
  int2 *flow_fwd, *flow_bwd;
};

void build_symbolic(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* perm, SymPlan& sp);

// ------------------------------------------------------------------------------------------ handles
struct gp_pointset {
  gp_ctx* ctx = nullptr;
  std::vector<DevBuf> bufs;
  std::vector<DevBuf> sched_bufs;     // the mixed-path update schedule (re-planned by gp_autotune)
  std::atomic<int64_t> nfactors{0};   // live factors on this point set
  int64_t n = 0;
  int d = 0;
  double rho[GP_MAX_D] = {1, 1, 1};
  double* X = nullptr;          // n x d copy of the points
  double* U = nullptr;          // n x d scaled coordinates, index order
  double* Us = nullptr;         // n x d scaled coordinates, cell order
  int32_t* cell_perm = nullptr; // cell order -> point
  int64_t* cell_start = nullptr;// ncells + 1
  int64_t ncells = 0;
  int64_t c0[GP_MAX_D] = {0, 0, 0};
  int64_t nc[GP_MAX_D] = {1, 1, 1};
  int64_t* rowptr = nullptr;    // n+1
  int32_t* col = nullptr;       // nnz
  int64_t nnz = 0;
  int32_t* perm = nullptr;      // new -> old
  int32_t* pinv = nullptr;      // old -> new
  int64_t* dest = nullptr;      // per CSR entry: panel offset of its lower-triangle copy, or -1
  int64_t* dest32 = nullptr;    // mixed layout: FP32 panel offset, or DIAG_FLAG | diagonal-tile offset, or -1
  SymPlan sp;
  DevPlan dp{};
  // support of the pattern: 0 the compact core's (core radii); 1 that of C_sparse (gp_assemble_sparse_support:
  // q0 < 1 for the radii r0, or both points in one bump family), recorded to check the settings factored on it
  int support = 0;
  int sup_n1 = 0, sup_n2 = 0, sup_bd = 0;
  std::vector<double> sup_h, sup_r;
  uint32_t* fam = nullptr;      // support 1: per point, bit i set when it lies in bump family i's support
};

struct gp_factor_s {
  gp_ctx* ctx = nullptr;
  gp_pointset* ps = nullptr;
  std::vector<DevBuf> bufs;
  int B = 0;
  gp_precision prec = GP_FP64;
  bool diag_fp32 = false;       // GP_MIXED: diagonal blocks factored in FP32 (default FP64)
  tcg::WaitLimit wait_lim = tcg::DEFAULT_WAIT;   // bounded-wait limits (tensor-core kernels, solve tasks)
  double refine_tol = 1e-10;    // GP_MIXED: relative residual at which gp_loglik's refinement stops
  double* theta_dev = nullptr;  // B packed settings
  int64_t theta_stride = 0;
  double* F = nullptr;          // B x n x n1 bump features
  double* Cpt = nullptr;        // non-compact core: B x n x 2 (sigma(x), Sigma(x)) per point
  int core_kind = 0;
  int n1max = 0;
  double* panels = nullptr;     // FP64 panels, B x panel_entries
  float* panels32 = nullptr;    // GP_MIXED: FP32 panels, row-major, B x panel32_entries
  float* op_lo = nullptr;       // GP_MIXED: tensor-core operands of the factored panel entries of one level's
                                //   large fronts, B x lo_entries: the low TF32 parts (the high parts are
                                //   panels32 itself) or, with op_f16, the FP16 pairs
  uint8_t* op_maps = nullptr;   // GP_MIXED: TMA maps of the high and low operands, 2 x 128 bytes per updated front
  bool op_f16 = false;          // GP_MIXED: FP16 operand pairs (GP_OPT_SPLIT_F16) instead of TF32 pairs
  unsigned long long* op_dmax = nullptr;   // GP_MIXED: per proposal, the bits of max_i C_ii (FP64, >= 0): the
                                //   FP16 pairs' power-of-two scale
  int32_t* op_slot = nullptr;   // GP_MIXED: per supernode, its map pair (-1 = none)
  double* diag = nullptr;       // GP_MIXED: FP64 64 x 64 diagonal tiles, B x diag_entries
  double* delta = nullptr;      // GP_MIXED: refinement vectors (residual and correction), B x 2n
  double* dinv = nullptr;       // FP64 inverses of the 64 x 64 diagonal blocks (row-major), B x diag_entries
  float* dinv32 = nullptr;      // GP_MIXED: the same inverses in FP32 (the TRSM's operand)
  double* rhs = nullptr;        // B x n copy of the caller's residual (the solve graph reads it from here)
  // CUDA graphs of the fixed launch sequences, captured on first use and replayed (launch counts per replay)
  cudaGraphExec_t gx_factor = nullptr, gx_solve = nullptr, gx_cor = nullptr;
  int64_t n_factor = 0, n_solve = 0, n_cor = 0;
  cudaGraphExec_t gx_refine = nullptr;   // GP_MIXED: the refinement loop with its test on the device
  cudaGraphExec_t gx_tail = nullptr;     // GP_MIXED: the loop alone, to the residual prediction needs
  int64_t n_tail = 0;
  double alpha_tol = 1.0;                // GP_MIXED: the residual tolerance alpha was last refined to
  int64_t n_refine = 0;
  const double* refine_out = nullptr;    // the output pointers gx_refine writes (ll_buf)
  const double* refine_err = nullptr;
  double* ll_buf = nullptr;              // GP_MIXED: 2B, the refinement graph's log-likelihoods and residuals
  int32_t* refine_it = nullptr;          // GP_MIXED: its correction counter
  unsigned long long* refine_runs = nullptr;   // corrections the loop has run (device, for launch accounting)
  int64_t n_refine_body = 0;             // launches of one pass of the loop body
  unsigned long long refine_runs_seen = 0;     // corrections already added to the context's launch count
  int32_t* tiles_err = nullptr; // set when a bounded wait (tensor-core updates, solve tasks) ran out
  int32_t* flow_sync = nullptr; // the solve tasks' tickets and readiness flags (flow_sync_entries)
  double* upd = nullptr;        // B x update_entries
  float* upd32 = nullptr;
  double* val = nullptr;        // B x nnz CSR values of C_z (refinement SpMV)
  int32_t* notpd = nullptr;     // B: smallest failing permuted column (INT_MAX = none)
  double* alpha = nullptr;      // B x n
  double* work = nullptr;       // solve workspace
  double* bwd_part = nullptr;   // backward partial sums over row chunks (B x bwd_part_entries)
  double* red = nullptr;        // reduction partials, B x red_stride
  int64_t red_stride = 0;
  int64_t work_stride = 0;
  bool have_alpha = false;
  std::vector<gp_hyper> thetas_host;
  uint8_t* var_work = nullptr;  // gp_predict_var workspace (allocated on its first call), var_nc chunks
  int var_nc = 0;
  uint8_t* it_work = nullptr;   // gp_loglik_iterative workspace (allocated on demand)
  size_t it_bytes = 0;
};

// ------------------------------------------------------------------------------------------ packed theta
// Layout on the device per proposal: [core_var, s0, noise_var, core_radius[3], r0[3], core kind, sigma0, Sigma0,
// phi_sigma[3], phi_Sigma[3], then per bump (h[bump_dims], a, b, r)]. n1/n2/bump_dims are shared by the batch.
// Core kind 0: the compact Wendland-type core core_var f0(q; core_radius); kind 1: the parametric nonstationary
// Matern core of App. B (Eq. PScov) with log-linear sigma(x), Sigma(x) (core_radius is then stored as r0, the
// unit of the point set's grid).
struct ThetaDims {
  int d, n1, n2, bd;
};
#define TH_CORE_VAR 0
#define TH_S0 1
#define TH_NOISE 2
#define TH_CRAD 3
#define TH_R0 6
#define TH_KIND 9
#define TH_SIG0 10
#define TH_SIGMA0 11
#define TH_PHIS 12
#define TH_PHIS2 15
#define TH_BUMPS 18
inline int64_t theta_stride_of(const ThetaDims& t) { return TH_BUMPS + (int64_t)t.n1 * t.n2 * (t.bd + 3); }

// ------------------------------------------------------------------------------------------ launchers
// sort.cu
size_t radix_sort_temp_bytes(int64_t n);
void radix_sort_pairs(gp_ctx* ctx, uint64_t* keys, uint32_t* vals, int64_t n, int begin_bit, int end_bit,
                      void* temp);
void exclusive_scan_i64(gp_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, void* temp);
size_t scan_temp_bytes(int64_t n);

// assemble.cu
void assemble_pointset(gp_ctx* ctx, gp_pointset* ps, const double* d_X);

// values.cu / factor.cu / solve.cu / predict.cu
void factor_run(gp_ctx* ctx, gp_factor_t* f);
void loglik_run(gp_ctx* ctx, gp_factor_t* f, const double* d_resid, double* d_out, double* d_err);
void refine_alpha_for_predict(gp_ctx* ctx, gp_factor_t* f);
void predict_run(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_Xt, int64_t m, const double* d_mu, double* d_mean);
void variance_run(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_Xt, int64_t m, double* d_var);
void iterative_run(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_resid, const double* d_probes,
                   const double* d_x0, const gp_iterative_opts& o, gp_iterative_result* res);
void compute_dest_map(gp_ctx* ctx, gp_pointset* ps);
void compute_dest_map_mixed(gp_ctx* ctx, gp_pointset* ps);
void build_update_maps(gp_ctx* ctx, gp_factor_t* f);
int64_t bwd_part_entries(const SymPlan& sp);
// The solve tasks' tickets (forward and backward, one each per level) and readiness flags (forward and
// backward, B x n_fl each).
inline int64_t flow_sync_entries(const SymPlan& sp, int B) {
  return 2 * (int64_t)sp.nlevels + 2 * (int64_t)B * sp.n_fl;
}
void plan_mixed_updates(SymPlan& sp, int group, int tn);
void upload_schedule(gp_ctx* ctx, gp_pointset* ps);
size_t factor_bytes(const gp_pointset* ps, gp_precision prec, int B, const ThetaDims& td);
#define DIAG_FLAG ((int64_t)1 << 62)

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

// Graph replay is used on an explicit (non-legacy) stream when the launch profiler is off.
inline bool use_graphs(const gp_ctx* ctx) { return ctx->stream != nullptr && !ctx->prof; }

// Capture the launches `body` issues on the context stream into an executable graph; *nlaunch receives the
// number of kernels captured (the context's counter is restored: replays add it per launch).
template <class F>
cudaGraphExec_t capture_graph(gp_ctx* ctx, F&& body, int64_t* nlaunch) {
  const int64_t l0 = ctx->launches;
  GP_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  try {
    body();
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(ctx->stream, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    ctx->launches = l0;
    throw;
  }
  cudaGraph_t g = nullptr;
  GP_CUDA(cudaStreamEndCapture(ctx->stream, &g));
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) throw GpError{GP_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)};
  *nlaunch = ctx->launches - l0;
  ctx->launches = l0;
  return ex;
}

inline void replay_graph(gp_ctx* ctx, cudaGraphExec_t ex, int64_t nlaunch) {
  GP_CUDA(cudaGraphLaunch(ex, ctx->stream));
  ctx->launches += nlaunch;
}

// Inverse of a bw x bw lower-triangular block (row-major, leading dimension GP_TILE, shared memory) into Inv
// (same layout), one column per thread: Inv[j][j] = 1/A[j][j], Inv[i][j] = -(sum_{j<=k<i} A[i][k] Inv[k][j]) / A[i][i].
// Entries outside the lower bw x bw triangle are set to zero. Ends with a barrier.
// R is the arithmetic type: double for the FP64 path; float where the result only preconditions an FP64
// refinement (the mixed path), since FP64 instructions issue at a small fraction of the FP32 rate on GB300.
template <class R>
__device__ __forceinline__ void tri_inverse_lower(const double* A, R* Inv, int bw) {
  constexpr int T = GP_TILE;
  for (int q = threadIdx.x; q < T * T; q += blockDim.x) Inv[q] = R(0);
  __syncthreads();
  for (int j = threadIdx.x; j < bw; j += blockDim.x) {
    Inv[j * T + j] = R(1) / R(A[j * T + j]);
    for (int i = j + 1; i < bw; i++) {
      R s0 = R(0), s1 = R(0);
      int k = j;
      for (; k + 1 < i; k += 2) {
        s0 += R(A[i * T + k]) * Inv[k * T + j];
        s1 += R(A[i * T + k + 1]) * Inv[(k + 1) * T + j];
      }
      if (k < i) s0 += R(A[i * T + k]) * Inv[k * T + j];
      Inv[i * T + j] = -(s0 + s1) / R(A[i * T + i]);
    }
  }
  __syncthreads();
}

inline unsigned grid_for(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 2147483647LL) g = 2147483647LL;
  return (unsigned)g;
}
