// solve.cu -- steps A8-A10 (and the FP64 residual of A11): supernodal forward and backward solves with the
// multifrontal factor, the quadratic form, the log-determinant and the log-likelihood
//   log p(z | beta, theta) = -1/2 log det C_z - 1/2 r^T C_z^{-1} r - n/2 log(2 pi)      (Sec. 3.3)
// with log det C_z = 2 sum_j log L_jj and r^T C_z^{-1} r = |L^{-1} P r|^2.
//
// Forward (levels ascending): the front vector of supernode s (m entries, own columns then the rows below)
// starts as the permuted right-hand side on its columns, receives every child's update vector through the
// child's relative indices (children in order), then x = L11^{-1} f_1 and f_2 -= L21 x; f_2 is the update
// vector handed to the parent. Backward (levels descending): t = x - L21^T alpha'(rows below), then
// L11^T z = t. Fronts of order <= 96 use one CTA; larger ones advance 64 columns per launch, every CTA
// re-solving the 64 x 64 diagonal block from L2 and applying it to its own 64-row (or 64-column) tile.
// Sums (log-det, quadratic form, residual norms) use fixed-shape trees, so results are bitwise reproducible.
#include <cmath>

#include "gp_internal.cuh"

namespace {

constexpr int T = GP_TILE;

__global__ void k_rhs(const double* __restrict__ resid, const int32_t* __restrict__ perm, int64_t n,
                      DevPlan dp, double* __restrict__ work, int64_t ws) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (j >= n) return;
  int32_t s = dp.sn_of_col[j];
  work[(int64_t)b * ws + dp.frow_off[s] + (j - dp.sn_first[s])] = resid[(int64_t)b * n + perm[j]];
}

// Children's update vectors into the front vector of each supernode of the list.
__global__ void k_fwd_gather(const int32_t* __restrict__ list, DevPlan dp, double* __restrict__ work, int64_t ws) {
  int32_t s = list[blockIdx.x];
  double* W = work + (int64_t)blockIdx.y * ws;
  double* fv = W + dp.frow_off[s];
  for (int32_t q = dp.ch_ptr[s]; q < dp.ch_ptr[s + 1]; q++) {
    int32_t c = dp.ch_idx[q];
    const double* uc = W + dp.frow_off[c] + dp.w[c];
    const int32_t* rel = dp.relidx + dp.relidx_off[c];
    for (int32_t a = threadIdx.x; a < dp.r[c]; a += blockDim.x) fv[rel[a]] += uc[a];
    __syncthreads();
  }
}

// Forward elimination of a whole (small) front by one CTA.
__global__ void k_fwd_small(const int32_t* __restrict__ list, DevPlan dp, const double* __restrict__ panels,
                            int64_t PE, double* __restrict__ work, int64_t ws, int64_t xv_off) {
  __shared__ double xs;
  int32_t s = list[blockIdx.x];
  int b = blockIdx.y;
  const double* P = panels + (int64_t)b * PE + dp.loff[s];
  double* fv = work + (int64_t)b * ws + dp.frow_off[s];
  double* xv = work + (int64_t)b * ws + xv_off + dp.sn_first[s];
  const int w = dp.w[s];
  const int64_t m = (int64_t)w + dp.r[s];
  for (int j = 0; j < w; j++) {
    if (threadIdx.x == 0) {
      xs = fv[j] / P[(int64_t)j * m + j];
      fv[j] = xs;
      xv[j] = xs;
    }
    __syncthreads();
    double x = xs;
    for (int64_t i = j + 1 + threadIdx.x; i < m; i += blockDim.x) fv[i] -= P[(int64_t)j * m + i] * x;
    __syncthreads();
  }
}

__device__ __forceinline__ int find_front(const int64_t* pre, int nfront, int64_t t) {
  int lo = 0, hi = nfront - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Solve the bw x bw lower block L_JJ x = t in shared memory (warp 0); x overwrites t.
__device__ __forceinline__ void block_lower_solve(const double* L, double* t, int bw) {
  if (threadIdx.x < 32) {
    for (int j = 0; j < bw; j++) {
      double x = t[j] / L[j * T + j];
      __syncwarp();
      for (int i = j + 1 + threadIdx.x; i < bw; i += 32) t[i] -= L[j * T + i] * x;
      if (threadIdx.x == 0) t[j] = x;
      __syncwarp();
    }
  }
  __syncthreads();
}
// Solve L_JJ^T z = t (upper triangular) in shared memory (warp 0); z overwrites t.
__device__ __forceinline__ void block_upper_solve(const double* L, double* t, int bw) {
  if (threadIdx.x < 32) {
    for (int j = bw - 1; j >= 0; j--) {
      double z = t[j] / L[j * T + j];
      __syncwarp();
      for (int k = threadIdx.x; k < j; k += 32) t[k] -= L[k * T + j] * z;
      if (threadIdx.x == 0) t[j] = z;
      __syncwarp();
    }
  }
  __syncthreads();
}

// One block column kb of the forward solve for every large front of a step. Tasks: [0, nfront) write the
// block's solution to x (a separate vector, since the other tasks still read the block's right-hand side);
// the rest (from the tile prefix) update one 64-row tile below the block.
__global__ void k_fwd_step(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre, int nfront, int kb,
                           DevPlan dp, const double* __restrict__ panels, int64_t PE, double* __restrict__ work,
                           int64_t ws, int64_t xv_off) {
  __shared__ double L[T * T];
  __shared__ double x[T];
  int64_t t = blockIdx.x;
  bool writer = t < nfront;
  int fi = writer ? (int)t : find_front(pre, nfront, t - nfront);
  int32_t s = fronts[fi];
  int b = blockIdx.y;
  const double* P = panels + (int64_t)b * PE + dp.loff[s];
  double* fv = work + (int64_t)b * ws + dp.frow_off[s];
  const int w = dp.w[s];
  const int64_t m = (int64_t)w + dp.r[s];
  const int c0 = kb * T, bw = min(T, w - c0), c1 = c0 + bw;
  for (int q = threadIdx.x; q < bw * bw; q += blockDim.x) {
    int i = q % bw, j = q / bw;
    L[j * T + i] = i >= j ? P[(int64_t)(c0 + j) * m + c0 + i] : 0.0;
  }
  for (int q = threadIdx.x; q < bw; q += blockDim.x) x[q] = fv[c0 + q];
  __syncthreads();
  block_lower_solve(L, x, bw);
  if (writer) {
    double* xv = work + (int64_t)b * ws + xv_off + dp.sn_first[s];
    for (int q = threadIdx.x; q < bw; q += blockDim.x) xv[c0 + q] = x[q];
    return;
  }
  int64_t r0 = c1 + (t - nfront - pre[fi]) * T;
  for (int64_t i = r0 + threadIdx.x; i < imin64(r0 + T, m); i += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < bw; l++) acc += P[(int64_t)(c0 + l) * m + i] * x[l];
    fv[i] -= acc;
  }
}

// t_j = x_j - sum_{a < r} L[w + a, j] alpha'(R_s[a]) for every column j of the front (warp per column);
// small fronts then finish L11^T z = t in the same CTA and write alpha'.
__global__ void k_bwd_prep(const int32_t* __restrict__ list, int solve_small, DevPlan dp,
                           const double* __restrict__ panels, int64_t PE, double* __restrict__ work, int64_t ws,
                           int64_t apv_off, int64_t xv_off) {
  __shared__ double zs;
  int32_t s = list[blockIdx.x];
  int b = blockIdx.y;
  const double* P = panels + (int64_t)b * PE + dp.loff[s];
  double* W = work + (int64_t)b * ws;
  double* fv = W + dp.frow_off[s];
  double* apv = W + apv_off;
  const int w = dp.w[s], r = dp.r[s];
  const int64_t m = (int64_t)w + r;
  const int32_t* R = dp.frows + dp.frow_off[s] + w;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < w; j += nw) {
    double acc = 0.0;
    for (int a = lane; a < r; a += 32) acc += P[(int64_t)j * m + w + a] * apv[R[a]];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) fv[j] = W[xv_off + dp.sn_first[s] + j] - acc;
  }
  __syncthreads();
  if (!solve_small) return;
  const int32_t first = dp.sn_first[s];
  for (int j = w - 1; j >= 0; j--) {
    if (threadIdx.x == 0) {
      zs = fv[j] / P[(int64_t)j * m + j];
      fv[j] = zs;
      apv[first + j] = zs;
    }
    __syncthreads();
    double z = zs;
    for (int k = threadIdx.x; k < j; k += blockDim.x) fv[k] -= P[(int64_t)k * m + j] * z;
    __syncthreads();
  }
}

// One block column kb of the backward solve for every large front of a step. Tasks per front: one writer
// (z of the block into alpha') and kb column tiles of the earlier columns (t_k -= L[J, k]^T z_J).
__global__ void k_bwd_step(const int32_t* __restrict__ fronts, int nfront, int kb, DevPlan dp,
                           const double* __restrict__ panels, int64_t PE, double* __restrict__ work, int64_t ws,
                           int64_t apv_off) {
  __shared__ double L[T * (T + 1)];   // the diagonal block, then (reused) the tile's rows of the block
  __shared__ double z[T];
  double* Lt = L;
  int64_t t = blockIdx.x;
  int fi = (int)(t / (kb + 1));
  int task = (int)(t % (kb + 1));   // 0 = writer, 1..kb = column tile task-1
  int32_t s = fronts[fi];
  int b = blockIdx.y;
  const double* P = panels + (int64_t)b * PE + dp.loff[s];
  double* W = work + (int64_t)b * ws;
  double* fv = W + dp.frow_off[s];
  const int w = dp.w[s];
  const int64_t m = (int64_t)w + dp.r[s];
  const int c0 = kb * T, bw = min(T, w - c0);
  for (int q = threadIdx.x; q < bw * bw; q += blockDim.x) {
    int i = q % bw, j = q / bw;
    L[j * T + i] = i >= j ? P[(int64_t)(c0 + j) * m + c0 + i] : 0.0;
  }
  for (int q = threadIdx.x; q < bw; q += blockDim.x) z[q] = fv[c0 + q];
  __syncthreads();
  block_upper_solve(L, z, bw);
  if (task == 0) {   // the block's right-hand side stays in place: the other tasks are still reading it
    double* apv = W + apv_off;
    const int32_t first = dp.sn_first[s];
    for (int q = threadIdx.x; q < bw; q += blockDim.x) apv[first + c0 + q] = z[q];
    return;
  }
  const int k0 = (task - 1) * T;   // columns [k0, k0 + 64) < c0
  // Lt[l][k] = L[c0 + l, k0 + k]: the block's rows for the tile's columns (global reads coalesced by rows)
  for (int q = threadIdx.x; q < T * bw; q += blockDim.x) {
    int l = q % bw, k = q / bw;
    Lt[l * (T + 1) + k] = P[(int64_t)(k0 + k) * m + c0 + l];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < T; k += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < bw; l++) acc += Lt[l * (T + 1) + k] * z[l];
    fv[k0 + k] -= acc;
  }
}

// Per-block partial sums: log L_jj and x_j^2 (x = forward solution on own columns).
__global__ void k_partials(int64_t n, DevPlan dp, const double* __restrict__ panels, int64_t PE,
                           const double* __restrict__ work, int64_t ws, int64_t xv_off, double* __restrict__ red,
                           int64_t rs, int nblk) {
  __shared__ double sa[1024], sb[1024];
  int b = blockIdx.y;
  int64_t j = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  double la = 0.0, lb = 0.0;
  if (j < n) {
    int32_t s = dp.sn_of_col[j];
    int64_t jl = j - dp.sn_first[s];
    int64_t m = (int64_t)dp.w[s] + dp.r[s];
    la = log(panels[(int64_t)b * PE + dp.loff[s] + jl * m + jl]);
    double x = work[(int64_t)b * ws + xv_off + j];
    lb = x * x;
  }
  sa[threadIdx.x] = la;
  sb[threadIdx.x] = lb;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    red[(int64_t)b * rs + blockIdx.x] = sa[0];
    red[(int64_t)b * rs + nblk + blockIdx.x] = sb[0];
  }
}

// Fixed-order reduction of the partials and the log-likelihood of each proposal.
__global__ void k_loglik(int64_t n, const double* __restrict__ red, int64_t rs, int nblk,
                         const int32_t* __restrict__ notpd, double* __restrict__ out, double* __restrict__ stats) {
  __shared__ double sa[256], sb[256];
  int b = blockIdx.x;
  double ta = 0.0, tb = 0.0;
  for (int base = 0; base < nblk; base += 256) {
    int i = base + threadIdx.x;
    sa[threadIdx.x] = i < nblk ? red[(int64_t)b * rs + i] : 0.0;
    sb[threadIdx.x] = i < nblk ? red[(int64_t)b * rs + nblk + i] : 0.0;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        sa[threadIdx.x] += sa[threadIdx.x + o];
        sb[threadIdx.x] += sb[threadIdx.x + o];
      }
      __syncthreads();
    }
    ta += sa[0];
    tb += sb[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double logdet = 2.0 * ta;
    double ll = -0.5 * logdet - 0.5 * tb - 0.5 * (double)n * log(2.0 * 3.14159265358979323846);
    if (notpd[b] != 0x7fffffff) ll = -INFINITY;
    out[b] = ll;
    if (stats) {
      stats[2 * b] = logdet;
      stats[2 * b + 1] = tb;
    }
  }
}

__global__ void k_alpha(const double* __restrict__ work, int64_t ws, int64_t apv_off, const int32_t* __restrict__ perm,
                        int64_t n, double* __restrict__ alpha) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (j < n) alpha[(int64_t)b * n + perm[j]] = work[(int64_t)b * ws + apv_off + j];
}

// res = r - C alpha (warp per CSR row, fixed lane order) and per-block sums of res^2 and r^2.
__global__ void k_residual(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n,
                           int64_t nnz, const double* __restrict__ val, const double* __restrict__ alpha,
                           const double* __restrict__ resid, double* __restrict__ res, double* __restrict__ red,
                           int64_t rs, int nblk) {
  __shared__ double s1[8], s2[8];
  int b = blockIdx.y;
  int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  if (i < n) {
    const double* v = val + (int64_t)b * nnz;
    const double* a = alpha + (int64_t)b * n;
    for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) acc += v[e] * a[col[e]];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  double rr = 0.0, ri = 0.0;
  if (i < n && lane == 0) {
    ri = resid[(int64_t)b * n + i];
    rr = ri - acc;
    if (res) res[(int64_t)b * n + i] = rr;
  }
  if (lane == 0) {
    s1[warp] = rr * rr;
    s2[warp] = ri * ri;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a1 = 0.0, a2 = 0.0;
    for (int q = 0; q < 8; q++) {
      a1 += s1[q];
      a2 += s2[q];
    }
    red[(int64_t)b * rs + blockIdx.x] = a1;
    red[(int64_t)b * rs + nblk + blockIdx.x] = a2;
  }
}

__global__ void k_relres(const double* __restrict__ red, int64_t rs, int nblk, double* __restrict__ err) {
  __shared__ double sa[256], sb[256];
  int b = blockIdx.x;
  double ta = 0.0, tb = 0.0;
  for (int base = 0; base < nblk; base += 256) {
    int i = base + threadIdx.x;
    sa[threadIdx.x] = i < nblk ? red[(int64_t)b * rs + i] : 0.0;
    sb[threadIdx.x] = i < nblk ? red[(int64_t)b * rs + nblk + i] : 0.0;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        sa[threadIdx.x] += sa[threadIdx.x + o];
        sb[threadIdx.x] += sb[threadIdx.x + o];
      }
      __syncthreads();
    }
    ta += sa[0];
    tb += sb[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) err[b] = tb > 0.0 ? sqrt(ta / tb) : sqrt(ta);
}

}  // namespace

// Forward and backward solves for all B right-hand sides; alpha (original order) into f->alpha.
// Returns nothing; the front vectors keep x for the quadratic form until the backward pass overwrites them,
// so the partial sums are taken in between.
void solve_run(gp_ctx* ctx, gp_factor_t* f, const double* d_resid, bool partials) {
  gp_pointset* ps = f->ps;
  const SymPlan& sp = ps->sp;
  const DevPlan& dp = ps->dp;
  cudaStream_t st = ctx->stream;
  const int B = f->B;
  const int64_t n = ps->n, PE = sp.panel_entries, ws = f->work_stride;
  const int64_t apv_off = sp.sn_frow[sp.ns];   // work layout: front vectors, alpha' (n), x (n)
  const int64_t xv_off = apv_off + n;
  GP_CUDA(cudaMemsetAsync(f->work, 0, sizeof(double) * (size_t)B * ws, st));
  k_rhs<<<dim3(grid_for(n, 256), B), 256, 0, st>>>(d_resid, ps->perm, n, dp, f->work, ws);
  GP_CHECK_LAUNCH(ctx);
  for (int32_t L = 0; L < sp.nlevels; L++) {
    const SymPlan::Level& lv = sp.levels[L];
    int32_t nl = sp.lev_ptr[L + 1] - sp.lev_ptr[L];
    if (L > 0) {
      k_fwd_gather<<<dim3(nl, B), 256, 0, st>>>(dp.lev_sn + sp.lev_ptr[L], dp, f->work, ws);
      GP_CHECK_LAUNCH(ctx);
    }
    if (lv.nsmall > 0) {
      k_fwd_small<<<dim3(lv.nsmall, B), 128, 0, st>>>(dp.small_list + lv.small_off, dp, f->panels, PE, f->work, ws,
                                                       xv_off);
      GP_CHECK_LAUNCH(ctx);
    }
    for (const auto& stp : lv.steps) {
      int64_t tasks = stp.nfront + stp.trsm_total;
      k_fwd_step<<<dim3((unsigned)tasks, B), 64, 0, st>>>(dp.large_fronts + stp.fr_off, dp.step_pre + stp.pre_off,
                                                          stp.nfront, stp.kb, dp, f->panels, PE, f->work, ws, xv_off);
      GP_CHECK_LAUNCH(ctx);
    }
  }
  if (partials) {
    int nblk = (int)((n + 1023) / 1024);
    k_partials<<<dim3(nblk, B), 1024, 0, st>>>(n, dp, f->panels, PE, f->work, ws, xv_off, f->red, f->red_stride,
                                                nblk);
    GP_CHECK_LAUNCH(ctx);
  }
  for (int32_t L = sp.nlevels - 1; L >= 0; L--) {
    const SymPlan::Level& lv = sp.levels[L];
    if (lv.nsmall > 0) {
      k_bwd_prep<<<dim3(lv.nsmall, B), 256, 0, st>>>(dp.small_list + lv.small_off, 1, dp, f->panels, PE, f->work, ws,
                                                      apv_off, xv_off);
      GP_CHECK_LAUNCH(ctx);
    }
    if (!lv.steps.empty()) {
      const auto& s0 = lv.steps[0];
      k_bwd_prep<<<dim3(s0.nfront, B), 256, 0, st>>>(dp.large_fronts + s0.fr_off, 0, dp, f->panels, PE, f->work, ws,
                                                      apv_off, xv_off);
      GP_CHECK_LAUNCH(ctx);
      for (int q = (int)lv.steps.size() - 1; q >= 0; q--) {
        const auto& stp = lv.steps[q];
        int64_t tasks = (int64_t)stp.nfront * (stp.kb + 1);
        k_bwd_step<<<dim3((unsigned)tasks, B), 64, 0, st>>>(dp.large_fronts + stp.fr_off, stp.nfront, stp.kb, dp,
                                                            f->panels, PE, f->work, ws, apv_off);
        GP_CHECK_LAUNCH(ctx);
      }
    }
  }
  k_alpha<<<dim3(grid_for(n, 256), B), 256, 0, st>>>(f->work, ws, apv_off, ps->perm, n, f->alpha);
  GP_CHECK_LAUNCH(ctx);
}

void residual_run(gp_ctx* ctx, gp_factor_t* f, const double* d_resid, double* d_res, double* d_err) {
  gp_pointset* ps = f->ps;
  const int64_t n = ps->n;
  int nblk = (int)((n + 7) / 8);
  // the partial buffer of the log-likelihood is sized for n/1024 blocks; residual partials use work space
  double* red = f->work;   // work is free after alpha has been extracted
  int64_t rs = 2 * (int64_t)nblk + 2;
  GP_REQUIRE(rs <= f->work_stride, "residual partials exceed the workspace");
  k_residual<<<dim3(nblk, f->B), 256, 0, ctx->stream>>>(ps->rowptr, ps->col, n, ps->nnz, f->val, f->alpha, d_resid,
                                                        d_res, red, f->work_stride, nblk);
  GP_CHECK_LAUNCH(ctx);
  k_relres<<<f->B, 256, 0, ctx->stream>>>(red, f->work_stride, nblk, d_err);
  GP_CHECK_LAUNCH(ctx);
  (void)rs;
}

void loglik_run(gp_ctx* ctx, gp_factor_t* f, const double* d_resid, double* d_out, double* d_err) {
  {
    ProfScope ps_(ctx, KC_SOLVE);   // the whole forward/backward sweep as one timed span
    solve_run(ctx, f, d_resid, true);
  }
  int nblk = (int)((f->ps->n + 1023) / 1024);
  k_loglik<<<f->B, 256, 0, ctx->stream>>>(f->ps->n, f->red, f->red_stride, nblk, f->notpd, d_out, nullptr);
  GP_CHECK_LAUNCH(ctx);
  if (d_err) residual_run(ctx, f, d_resid, nullptr, d_err);
}
