// factor.cu -- step A7: multifrontal supernodal Cholesky of P C_z P^T, level by level over the supernodal
// elimination tree, every launch batched over the B proposals (grid y).
//
// Front of supernode s: order m = w + r, rows = its w columns then the r rows below it. Its first w columns
// are the panel (stored column-major, ld m, in the factor); the trailing r x r block is the update matrix U_s
// (column-major, ld r, in the update workspace). Per level:
//   1. zero the update matrices of the level's supernodes;
//   2. extend-add: every child's update matrix is added into its parent's front through the child's
//      relative indices, one launch per child slot so that contributions arrive in a fixed order;
//   3. partial factorization of each front: POTRF of the w x w diagonal block, TRSM of the r rows below,
//      SYRK of U_s -= L21 L21^T. Fronts of order <= 96 are factored by one CTA in shared memory; larger
//      ones by 64-wide block columns (POTRF, TRSM tiles, lower-triangular update tiles), all large fronts of a
//      level advancing together one block column per launch triple.
// A non-positive pivot records the smallest failing permuted column of that proposal and continues with a
// unit pivot, so the launch sequence is fixed and no kernel traps.
#include <climits>

#include "gp_internal.cuh"

void values_run(gp_ctx* ctx, gp_factor_t* f);

namespace {

constexpr int T = GP_TILE;

struct FrontRef {
  int32_t w, r;
  int64_t m;
  double* P;   // panel
  double* Uu;  // update matrix
};

__device__ __forceinline__ FrontRef front_of(const DevPlan& dp, int32_t s, double* panels, double* upd) {
  FrontRef fr;
  fr.w = dp.w[s];
  fr.r = dp.r[s];
  fr.m = (int64_t)fr.w + fr.r;
  fr.P = panels + dp.loff[s];
  fr.Uu = upd + dp.uoff[s];
  return fr;
}

// Address of front entry (i, j), i >= j, in panel or update storage.
__device__ __forceinline__ double* front_at(const FrontRef& fr, int64_t i, int64_t j) {
  return j < fr.w ? fr.P + j * fr.m + i : fr.Uu + (j - fr.w) * fr.r + (i - fr.w);
}

__device__ __forceinline__ double checked_sqrt(double d, int32_t* notpd, int32_t col) {
  if (!(d > 0.0)) {
    atomicMin(notpd, col);
    return 1.0;
  }
  return sqrt(d);
}

__global__ void k_zero_updates(const int32_t* __restrict__ list, DevPlan dp, double* __restrict__ upd, int64_t UE) {
  int32_t s = list[blockIdx.x];
  double* U = upd + (int64_t)blockIdx.y * UE + dp.uoff[s];
  int64_t cnt = (int64_t)dp.r[s] * dp.r[s];
  for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) U[t] = 0.0;
}

// One CTA per (child, 8 update columns); adds U_child into the parent's front.
__global__ void k_extend_add(const int2* __restrict__ tab, DevPlan dp, const int32_t* __restrict__ sn_parent,
                             double* __restrict__ panels, double* __restrict__ upd, int64_t PE, int64_t UE) {
  int2 task = tab[blockIdx.x];
  int32_t c = task.x, c0 = task.y;
  int b = blockIdx.y;
  double* pan = panels + (int64_t)b * PE;
  double* up = upd + (int64_t)b * UE;
  int32_t p = sn_parent[c];
  int32_t rc = dp.r[c];
  const double* Uc = up + dp.uoff[c];
  const int32_t* rel = dp.relidx + dp.relidx_off[c];
  FrontRef fp = front_of(dp, p, pan, up);
  int32_t c1 = min(c0 + 8, rc);
  for (int32_t bc = c0; bc < c1; bc++) {
    int32_t tc = rel[bc];
    for (int32_t a = bc + threadIdx.x; a < rc; a += blockDim.x) {
      int32_t tr = rel[a];
      *front_at(fp, tr, tc) += Uc[(int64_t)bc * rc + a];
    }
  }
}

// Whole partial factorization of a front of order <= GP_SMALL_M in shared memory.
__global__ void k_small_front(const int32_t* __restrict__ list, DevPlan dp, double* __restrict__ panels,
                              double* __restrict__ upd, int64_t PE, int64_t UE, int32_t* __restrict__ notpd) {
  extern __shared__ double A[];   // m x m, column-major, lower part used
  int32_t s = list[blockIdx.x];
  int b = blockIdx.y;
  FrontRef fr = front_of(dp, s, panels + (int64_t)b * PE, upd + (int64_t)b * UE);
  const int m = (int)fr.m, w = fr.w;
  const int32_t first = dp.sn_first[s];
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t % m, j = t / m;
    if (i >= j) A[t] = *front_at(fr, i, j);
  }
  __syncthreads();
  __shared__ double piv;
  for (int k = 0; k < w; k++) {
    if (threadIdx.x == 0) {
      piv = checked_sqrt(A[k * m + k], notpd + b, first + k);
      A[k * m + k] = piv;
    }
    __syncthreads();
    double inv = 1.0 / piv;
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) A[k * m + i] *= inv;
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 columns x 32 rows (blockDim = 256)
    for (int j = k + 1 + ty; j < m; j += 8) {
      const double ajk = A[k * m + j];
      for (int i = j + tx; i < m; i += 32) A[j * m + i] -= A[k * m + i] * ajk;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t % m, j = t / m;
    if (i >= j) *front_at(fr, i, j) = A[t];
  }
}

__device__ __forceinline__ int find_front(const int64_t* pre, int nfront, int64_t t) {
  int lo = 0, hi = nfront - 1;   // largest f with pre[f] <= t
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// POTRF of the diagonal block of block column kb, one CTA per large front.
__global__ void k_potrf(const int32_t* __restrict__ fronts, int kb, DevPlan dp, double* __restrict__ panels,
                        double* __restrict__ upd, int64_t PE, int64_t UE, int32_t* __restrict__ notpd,
                        double* __restrict__ dinv, int64_t DE) {
  extern __shared__ double sm64[];
  double* A = sm64;           // factor, column-major
  double* R = sm64 + T * T;   // factor, row-major (input of the inverse)
  __shared__ double piv;
  int32_t s = fronts[blockIdx.x];
  int b = blockIdx.y;
  FrontRef fr = front_of(dp, s, panels + (int64_t)b * PE, upd + (int64_t)b * UE);
  const int c0 = kb * T, bw = min(T, fr.w - c0);
  const int32_t first = dp.sn_first[s];
  for (int t = threadIdx.x; t < bw * bw; t += blockDim.x) {
    int i = t % bw, j = t / bw;
    if (i >= j) A[j * T + i] = fr.P[(int64_t)(c0 + j) * fr.m + c0 + i];
  }
  __syncthreads();
  for (int k = 0; k < bw; k++) {
    if (threadIdx.x == 0) {
      piv = checked_sqrt(A[k * T + k], notpd + b, first + c0 + k);
      A[k * T + k] = piv;
    }
    __syncthreads();
    double inv = 1.0 / piv;
    for (int i = k + 1 + threadIdx.x; i < bw; i += blockDim.x) A[k * T + i] *= inv;
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 4 columns x 32 rows (blockDim = 128)
    for (int j = k + 1 + ty; j < bw; j += 4) {
      const double ajk = A[k * T + j];
      for (int i = j + tx; i < bw; i += 32) A[j * T + i] -= A[k * T + i] * ajk;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < T * T; t += blockDim.x) {
    int i = t % T, j = t / T;
    bool lower = i >= j && i < bw;
    if (lower) fr.P[(int64_t)(c0 + j) * fr.m + c0 + i] = A[j * T + i];
    R[i * T + j] = lower ? A[j * T + i] : 0.0;
  }
  __syncthreads();
  tri_inverse_lower<double>(R, A, bw);   // inverse of the diagonal block (row-major) for the solves
  double* DI = dinv + (int64_t)b * DE + dp.doff[s] + (int64_t)kb * T * T;
  for (int t = threadIdx.x; t < T * T; t += blockDim.x) DI[t] = A[t];
}

// TRSM: rows below the diagonal block (within the panel) times L11^{-T}; one CTA per 64-row tile.
__global__ void k_trsm(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre, int nfront, int kb,
                       DevPlan dp, double* __restrict__ panels, int64_t PE) {
  extern __shared__ double sm[];
  double* L = sm;            // T x T, column-major
  double* X = sm + T * T;    // T rows x T cols, column-major (ld T)
  int64_t t = blockIdx.x;
  int fi = find_front(pre, nfront, t);
  int32_t s = fronts[fi];
  int b = blockIdx.y;
  double* P = panels + (int64_t)b * PE + dp.loff[s];
  const int w = dp.w[s];
  const int64_t m = (int64_t)w + dp.r[s];
  const int c0 = kb * T, bw = min(T, w - c0), c1 = c0 + bw;
  const int64_t r0 = c1 + (t - pre[fi]) * T;
  const int nr = (int)imin64(T, m - r0);
  for (int q = threadIdx.x; q < bw * bw; q += blockDim.x) {
    int i = q % bw, j = q / bw;
    L[j * T + i] = (i >= j) ? P[(int64_t)(c0 + j) * m + c0 + i] : 0.0;
  }
  for (int q = threadIdx.x; q < T * bw; q += blockDim.x) {
    int i = q % T, j = q / T;
    X[j * T + i] = i < nr ? P[(int64_t)(c0 + j) * m + r0 + i] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < bw; j++) {
    double inv = 1.0 / L[j * T + j];
    for (int i = threadIdx.x; i < T; i += blockDim.x) X[j * T + i] *= inv;
    __syncthreads();
    int rem = bw - j - 1;
    for (int q = threadIdx.x; q < T * rem; q += blockDim.x) {
      int i = q % T, jj = j + 1 + q / T;
      X[jj * T + i] -= X[j * T + i] * L[j * T + jj];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < T * bw; q += blockDim.x) {
    int i = q % T, j = q / T;
    if (i < nr) P[(int64_t)(c0 + j) * m + r0 + i] = X[j * T + i];
  }
}

// Trailing update of block column kb: F[I, J] -= L[I, kb] L[J, kb]^T over lower-triangular 64x64 tiles of
// the rows/columns after the block column (panel columns and update matrix alike). 256 threads, 4x4 each.
__global__ void __launch_bounds__(256) k_update(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre,
                                                int nfront, int kb, DevPlan dp, double* __restrict__ panels,
                                                double* __restrict__ upd, int64_t PE, int64_t UE) {
  extern __shared__ double sm[];
  double* AI = sm;           // [l][i]  T x T
  double* AJ = sm + T * T;   // [l][j]
  int64_t t = blockIdx.x;
  int fi = find_front(pre, nfront, t);
  int32_t s = fronts[fi];
  int b = blockIdx.y;
  FrontRef fr = front_of(dp, s, panels + (int64_t)b * PE, upd + (int64_t)b * UE);
  const int c0 = kb * T, bw = min(T, fr.w - c0), c1 = c0 + bw;
  int64_t loc = t - pre[fi];
  int64_t I = (int64_t)((sqrt(8.0 * (double)loc + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= loc) I++;
  while (I * (I + 1) / 2 > loc) I--;
  int64_t J = loc - I * (I + 1) / 2;
  const int64_t i0 = c1 + I * T, j0 = c1 + J * T;
  const int ni = (int)imin64(T, fr.m - i0), nj = (int)imin64(T, fr.m - j0);
  for (int q = threadIdx.x; q < T * T; q += blockDim.x) {
    int i = q % T, l = q / T;
    bool okl = l < bw;
    AI[l * T + i] = (okl && i < ni) ? fr.P[(int64_t)(c0 + l) * fr.m + i0 + i] : 0.0;
    AJ[l * T + i] = (okl && i < nj) ? fr.P[(int64_t)(c0 + l) * fr.m + j0 + i] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int c = 0; c < 4; c++) acc[a][c] = 0.0;
  for (int l = 0; l < bw; l++) {
    double ai[4], aj[4];
#pragma unroll
    for (int a = 0; a < 4; a++) ai[a] = AI[l * T + tx + 16 * a];
#pragma unroll
    for (int c = 0; c < 4; c++) aj[c] = AJ[l * T + ty + 16 * c];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 4; c++) acc[a][c] = fma(ai[a], aj[c], acc[a][c]);
  }
#pragma unroll
  for (int c = 0; c < 4; c++) {
    int jl = ty + 16 * c;
    if (jl >= nj) continue;
    int64_t j = j0 + jl;
#pragma unroll
    for (int a = 0; a < 4; a++) {
      int il = tx + 16 * a;
      int64_t i = i0 + il;
      if (il < ni && i >= j) *front_at(fr, i, j) -= acc[a][c];
    }
  }
}

std::once_flag g_attrs_once;
void set_attrs() {   // once per process (contexts may run on several host threads)
  std::call_once(g_attrs_once, [] {
    GP_CUDA(cudaFuncSetAttribute(k_small_front, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 GP_SMALL_M * GP_SMALL_M * (int)sizeof(double)));
    GP_CUDA(cudaFuncSetAttribute(k_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * T * T * (int)sizeof(double)));
    GP_CUDA(cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * T * T * (int)sizeof(double)));
    GP_CUDA(cudaFuncSetAttribute(k_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * T * T * (int)sizeof(double)));
  });
}

__global__ void k_fill_i32(int32_t* p, int n, int32_t v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace

void factor_run_mixed(gp_ctx* ctx, gp_factor_t* f);
void set_attrs_mixed();
static void factor_body(gp_ctx* ctx, gp_factor_t* f);

// A3, A4, A7: the launch sequence is fixed by the plan, so it is captured once per factor as a CUDA graph
// and replayed (theta only changes the device-side parameter block).
void factor_run(gp_ctx* ctx, gp_factor_t* f) {
  set_attrs();
  set_attrs_mixed();
  if (!use_graphs(ctx)) {
    factor_body(ctx, f);
    return;
  }
  if (!f->gx_factor) f->gx_factor = capture_graph(ctx, [&] { factor_body(ctx, f); }, &f->n_factor);
  replay_graph(ctx, f->gx_factor, f->n_factor);
}

static void factor_body(gp_ctx* ctx, gp_factor_t* f) {
  if (f->prec == GP_MIXED) {
    factor_run_mixed(ctx, f);
    return;
  }
  gp_pointset* ps = f->ps;
  const SymPlan& sp = ps->sp;
  const DevPlan& dp = ps->dp;
  cudaStream_t st = ctx->stream;
  set_attrs();
  const int B = f->B;
  const int64_t PE = sp.panel_entries, UE = sp.update_entries;
  values_run(ctx, f);   // A3, A4 (zeroes and fills the panels)
  k_fill_i32<<<grid_for(B, 128), 128, 0, st>>>(f->notpd, B, INT_MAX);
  GP_CHECK_LAUNCH(ctx);
  GP_CUDA(cudaMemsetAsync(f->tiles_err, 0, sizeof(int32_t), st));
  const int32_t* d_sn_parent = dp.sn_parent;
  ProfLevelScope pls_(ctx);
  for (int32_t L = 0; L < sp.nlevels; L++) {
    const SymPlan::Level& lv = sp.levels[L];
    ctx->prof_level = L;
    int32_t nl = sp.lev_ptr[L + 1] - sp.lev_ptr[L];
    k_zero_updates<<<dim3(nl, B), 256, 0, st>>>(dp.lev_sn + sp.lev_ptr[L], dp, f->upd, UE);
    GP_CHECK_LAUNCH(ctx);
    for (const auto& ea : lv.ea) {
      ProfScope ps_(ctx, KC_EXTEND_ADD);
      k_extend_add<<<dim3((unsigned)ea.ncta, B), 128, 0, st>>>(dp.ea_tab + ea.tab_off, dp, d_sn_parent, f->panels,
                                                               f->upd, PE, UE);
      GP_CHECK_LAUNCH(ctx);
    }
    if (lv.nsmall > 0) {
      // the largest small front of this level sets the shared memory size
      int32_t mmax = 1;
      for (int32_t q = 0; q < lv.nsmall; q++) {
        int32_t s = sp.small_list[lv.small_off + q];
        mmax = std::max(mmax, sp.sn_w[s] + sp.sn_r[s]);
      }
      ProfScope ps_(ctx, KC_FRONT_SMALL);
      k_small_front<<<dim3(lv.nsmall, B), 256, (size_t)mmax * mmax * sizeof(double), st>>>(
          dp.small_list + lv.small_off, dp, f->panels, f->upd, PE, UE, f->notpd);
      GP_CHECK_LAUNCH(ctx);
    }
    for (const auto& stp : lv.steps) {
      const int32_t* fronts = dp.large_fronts + stp.fr_off;
      const int64_t* pre_tr = dp.step_pre + stp.pre_off;
      const int64_t* pre_up = pre_tr + stp.nfront + 1;
      {
        ProfScope ps_(ctx, KC_POTRF, B * stp.potrf_flops);
        k_potrf<<<dim3(stp.nfront, B), 128, 2 * T * T * sizeof(double), st>>>(
            fronts, stp.kb, dp, f->panels, f->upd, PE, UE, f->notpd, f->dinv, sp.diag_entries);
        GP_CHECK_LAUNCH(ctx);
      }
      if (stp.trsm_total > 0) {
        ProfScope ps_(ctx, KC_TRSM, B * stp.trsm_flops);
        k_trsm<<<dim3((unsigned)stp.trsm_total, B), 256, 2 * T * T * sizeof(double), st>>>(
            fronts, pre_tr, stp.nfront, stp.kb, dp, f->panels, PE);
        GP_CHECK_LAUNCH(ctx);
      }
      if (stp.upd_total > 0) {
        ProfScope ps_(ctx, KC_UPDATE, B * stp.upd_flops);
        k_update<<<dim3((unsigned)stp.upd_total, B), 256, 2 * T * T * sizeof(double), st>>>(
            fronts, pre_up, stp.nfront, stp.kb, dp, f->panels, f->upd, PE, UE);
        GP_CHECK_LAUNCH(ctx);
      }
    }
  }
}
