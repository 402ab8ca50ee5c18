// variance.cu -- the predictive variance (Sec. 3.2): the diagonal of the conditional covariance
//   C_{y|z} = C_y - C_{y,z} C_z^{-1} C_{z,y},   var_k = C_y(x*_k, x*_k) - |w_k|^2,   L w_k = P c_k,
// c_k = C_y(X, x*_k) the cross-covariance column of test point k (no noise term at test inputs, Sec. 3.2) and
// C_y(x*, x*) = core_var (s0 + sum_i f_i(x*)^2) (f0(0) = 1 for the core and for C_sparse).
//
// c_k is nonzero only at the training neighbours of x*_k (the core support), so w_k is nonzero only on the
// supernodes on the paths from those neighbours' supernodes to the root of the supernodal elimination tree. Test
// points go through the factor's forward sweep R = 32 at a time (a chunk; NC chunks side by side in the grid):
//   mark  (warp per test point): the prior C_y(x*, x*) into the output, and every supernode on a neighbour's path
//         marked active for the chunk;
//   zero / scatter: the active supernodes' front vectors (m_s x R) cleared, then c_k written at its neighbours'
//         rows;
//   levels ascending: children's update vectors added into the parents (in child order), fronts of order <= 96
//         eliminated by one CTA, larger fronts 64 columns per launch: every CTA forms X_J = inv(L_JJ) F_J for
//         its front (a 64 x 64 by 64 x R product) and either stores X_J (the entries of w) or applies
//         F_I -= L_IJ X_J to one 64-row tile below; inactive (front, chunk) pairs return at once;
//   sum: |w_k|^2 over all entries in a fixed order, var_k = prior_k - |w_k|^2.
// The arithmetic is the factor's working precision: FP64 with the FP64 factor; FP32 vectors with the mixed
// factor's FP32 panels and inverses (the variance then carries the mixed factor's ~1e-6 relative accuracy).
#include <algorithm>

#include "factor_access.cuh"
#include "gp_internal.cuh"
#include "testpoint.cuh"

namespace {

constexpr int T = GP_TILE;
constexpr int R = 32;   // test points per chunk
using fa::find_front;

// Per chunk c: front vectors at F + c * cs (row i of front s at (frow_off[s] + i) * R), then the w entries of the
// n permuted columns at X + c * cs (column j at j * R).
template <class V>
struct VarWork {
  V* F;
  V* X;
  int64_t cs;             // entries per chunk (front rows x R + n x R)
  uint8_t* active;        // NC x ns
  int64_t ns;
};

__global__ void k_var_mark(const double* __restrict__ Xt, int64_t m, int64_t k0, tp::GridInfo g,
                           const double* __restrict__ X, const double* __restrict__ Us,
                           const int32_t* __restrict__ cell_perm, const int64_t* __restrict__ cell_start,
                           const double* __restrict__ theta, int n1, int n2, int bd, const double* __restrict__ F,
                           const double* __restrict__ Cpt, const int32_t* __restrict__ pinv, DevPlan dp,
                           uint8_t* __restrict__ active, int64_t ns, double* __restrict__ var) {
  __shared__ double fs[8][GP_MAX_N1];
  __shared__ double gs[8][64];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 8 + wi;   // index in the batch
  const int64_t k = k0 + q;
  if (k >= m) return;
  const tp::TestPoint p = tp::load_features(Xt, k, g, theta, n1, n2, bd, fs[wi], gs[wi]);
  uint8_t* act = active + (q / R) * ns;
  tp::for_each_neighbour(p, g, X, Us, cell_perm, cell_start, theta, n1, fs[wi], F, Cpt, [&](int32_t j, double) {
    for (int32_t s = dp.sn_of_col[pinv[j]]; s >= 0 && !act[s]; s = dp.sn_parent[s]) act[s] = 1;
  });
  if (lane == 0) {   // C_y(x*, x*) = C_core(x*, x*) (s0 + sum_i f_i(x*)^2)
    double ss = theta[TH_S0];
    for (int i = 0; i < n1; i++) ss += fs[wi][i] * fs[wi][i];
    double core = theta[TH_CORE_VAR];
    if (theta[TH_KIND] != 0.0) {
      double cs[2];
      tp::core_point(theta, p.xs, g.d, cs);
      core = tp::core_paciorek(cs, cs, p.xs, p.xs, g.d);
    }
    var[k] = core * ss;
  }
}

// A warp per (supernode, chunk): clears the active supernodes' front vectors.
template <class V>
__global__ void k_var_zero(DevPlan dp, int64_t ns, VarWork<V> vw) {
  const int64_t s = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int c = blockIdx.y, lane = threadIdx.x & 31;
  if (s >= ns || !vw.active[c * ns + s]) return;
  V* f = vw.F + c * vw.cs + dp.frow_off[s] * R;
  const int64_t cnt = ((int64_t)dp.w[s] + dp.r[s]) * R;
  for (int64_t e = lane; e < cnt; e += 32) f[e] = V(0);
}

template <class V>
__global__ void k_var_scatter(const double* __restrict__ Xt, int64_t m, int64_t k0, tp::GridInfo g,
                              const double* __restrict__ X, const double* __restrict__ Us,
                              const int32_t* __restrict__ cell_perm, const int64_t* __restrict__ cell_start,
                              const double* __restrict__ theta, int n1, int n2, int bd, const double* __restrict__ F,
                              const double* __restrict__ Cpt, const int32_t* __restrict__ pinv, DevPlan dp,
                              VarWork<V> vw) {
  __shared__ double fs[8][GP_MAX_N1];
  __shared__ double gs[8][64];
  const int wi = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 8 + wi;
  const int64_t k = k0 + q;
  if (k >= m) return;
  const tp::TestPoint p = tp::load_features(Xt, k, g, theta, n1, n2, bd, fs[wi], gs[wi]);
  V* base = vw.F + (q / R) * vw.cs;
  const int r = (int)(q % R);
  tp::for_each_neighbour(p, g, X, Us, cell_perm, cell_start, theta, n1, fs[wi], F, Cpt, [&](int32_t j, double cy) {
    const int32_t pj = pinv[j];
    const int32_t s = dp.sn_of_col[pj];
    base[(dp.frow_off[s] + (pj - dp.sn_first[s])) * R + r] = (V)cy;
  });
}

// Children's update vectors into the front vectors of the level's supernodes (children in order).
template <class V>
__global__ void k_var_gather(const int32_t* __restrict__ list, DevPlan dp, VarWork<V> vw) {
  const int32_t s = list[blockIdx.x];
  const int c = blockIdx.y;
  const uint8_t* act = vw.active + c * vw.ns;
  if (!act[s]) return;
  V* W = vw.F + c * vw.cs;
  V* fv = W + dp.frow_off[s] * R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int32_t qc = dp.ch_ptr[s]; qc < dp.ch_ptr[s + 1]; qc++) {
    const int32_t ch = dp.ch_idx[qc];
    if (!act[ch]) continue;
    const V* uc = W + ((int64_t)dp.frow_off[ch] + dp.w[ch]) * R;
    const int32_t* rel = dp.relidx + dp.relidx_off[ch];
    for (int32_t a = warp; a < dp.r[ch]; a += nw) fv[(int64_t)rel[a] * R + lane] += uc[(int64_t)a * R + lane];
    __syncthreads();
  }
}

// Fronts of order <= GP_SMALL_M: forward elimination of the whole front, R right-hand sides, one CTA.
template <class St>
__global__ void k_var_small(const int32_t* __restrict__ list, DevPlan dp, St store, int b,
                            VarWork<typename St::V> vw) {
  using V = typename St::V;
  __shared__ V Fs[GP_SMALL_M][R];
  __shared__ V xr[R];
  const int32_t s = list[blockIdx.x];
  const int c = blockIdx.y;
  if (!vw.active[c * vw.ns + s]) return;
  auto A = store.acc(dp, s, b);
  V* fv = vw.F + c * vw.cs + dp.frow_off[s] * R;
  V* xv = vw.X + c * vw.cs + (int64_t)dp.sn_first[s] * R;
  const int w = dp.w[s], m = w + dp.r[s];
  for (int e = threadIdx.x; e < m * R; e += blockDim.x) Fs[e / R][e % R] = fv[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < w; j++) {
    if (warp == 0) {
      const V x = Fs[j][lane] / A.L(j, j);
      xr[lane] = x;
      xv[(int64_t)j * R + lane] = x;
    }
    __syncthreads();
    for (int i = j + 1 + warp; i < m; i += nw) Fs[i][lane] -= A.L(i, j) * xr[lane];
    __syncthreads();
  }
  for (int e = threadIdx.x; e < (m - w) * R; e += blockDim.x) fv[(int64_t)w * R + e] = Fs[w + e / R][e % R];
}

// Block column kb of the large fronts of a step: tasks [0, nfront) store X_J = inv(L_JJ) F_J (the w entries of
// the block's columns), the rest (the tile prefix of the rows below) apply F_I -= L_IJ X_J to one 64-row tile.
// 256 threads; thread t forms 8 entries of its row (t >> 2) and right-hand sides 8 (t & 3) .. + 7.
template <class St>
__global__ void __launch_bounds__(256) k_var_step(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre,
                                                  int nfront, int kb, DevPlan dp, St store, int b,
                                                  VarWork<typename St::V> vw) {
  using V = typename St::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Mt = reinterpret_cast<V*>(smem_raw);   // Mt[l][i]: inv[i][l], then L[r0 + i][c0 + l]   (64 x 65)
  V* Fb = Mt + T * (T + 1);                 // Fb[l][r]: F_J, then X_J                            (64 x R)
  const int64_t t = blockIdx.x;
  const bool writer = t < nfront;
  const int fi = writer ? (int)t : find_front(pre, nfront, t - nfront);
  const int32_t s = fronts[fi];
  const int c = blockIdx.y;
  if (!vw.active[c * vw.ns + s]) return;
  auto A = store.acc(dp, s, b);
  V* fv = vw.F + c * vw.cs + dp.frow_off[s] * R;
  const int w = dp.w[s];
  const int64_t m = (int64_t)w + dp.r[s];
  const int c0 = kb * T, bw = min(T, w - c0), c1 = c0 + bw;
  const V* inv = store.inv(dp, s, b) + (int64_t)kb * T * T;
  for (int e = threadIdx.x; e < T * T; e += 256) Mt[(e & 63) * (T + 1) + (e >> 6)] = inv[e];   // zero past bw
  for (int e = threadIdx.x; e < T * R; e += 256) {
    const int l = e / R;
    Fb[e] = l < bw ? fv[(int64_t)(c0 + l) * R + (e % R)] : V(0);
  }
  __syncthreads();
  const int ti = threadIdx.x >> 2, tr = (threadIdx.x & 3) * 8;
  V acc[8];
#pragma unroll
  for (int e = 0; e < 8; e++) acc[e] = V(0);
  for (int l = 0; l < T; l++) {
    const V a = Mt[l * (T + 1) + ti];
#pragma unroll
    for (int e = 0; e < 8; e++) acc[e] += a * Fb[l * R + tr + e];
  }
  __syncthreads();   // every thread has read F_J and the inverse
#pragma unroll
  for (int e = 0; e < 8; e++) Fb[ti * R + tr + e] = ti < bw ? acc[e] : V(0);   // X_J
  if (writer) {
    if (ti < bw) {
      V* xv = vw.X + c * vw.cs + ((int64_t)dp.sn_first[s] + c0 + ti) * R;
#pragma unroll
      for (int e = 0; e < 8; e++) xv[tr + e] = acc[e];
    }
    return;
  }
  const int64_t r0 = c1 + (t - nfront - pre[fi]) * T;
  const int nr = (int)imin64(T, m - r0);
  for (int e = threadIdx.x; e < T * T; e += 256) {   // L[r0 + i][c0 + l] -> Mt[l][i], reads along the storage
    const int i = St::kRowMajor ? e >> 6 : e & 63, l = St::kRowMajor ? e & 63 : e >> 6;
    Mt[l * (T + 1) + i] = (i < nr && l < bw) ? (V)A.L(r0 + i, c0 + l) : V(0);
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < 8; e++) acc[e] = V(0);
  for (int l = 0; l < bw; l++) {
    const V a = Mt[l * (T + 1) + ti];
#pragma unroll
    for (int e = 0; e < 8; e++) acc[e] += a * Fb[l * R + tr + e];
  }
  if (ti < nr) {
    V* row = fv + (r0 + ti) * R + tr;
#pragma unroll
    for (int e = 0; e < 8; e++) row[e] -= acc[e];
  }
}

// Partial sums of w^2 per (chunk, right-hand side) over column slices, in a fixed order: CTA g of chunk c sums
// columns j = 8 g' + (t >> 5) for its slice, lanes = right-hand sides.
constexpr int SUM_CTAS = 64;
template <class V>
__global__ void k_var_sumsq(int64_t n, VarWork<V> vw, double* __restrict__ part) {
  __shared__ double sp[8][R];
  const int c = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const V* x = vw.X + c * vw.cs;
  double acc = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * 8 + warp; j < n; j += (int64_t)gridDim.x * 8) {
    const double v = (double)x[j * R + lane];
    acc += v * v;
  }
  sp[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    double a = 0.0;
    for (int q = 0; q < 8; q++) a += sp[q][lane];
    part[((int64_t)c * gridDim.x + blockIdx.x) * R + lane] = a;
  }
}

__global__ void k_var_final(const double* __restrict__ part, int nparts, int64_t m, int64_t k0,
                            double* __restrict__ var) {
  const int c = blockIdx.x, r = threadIdx.x;
  const int64_t k = k0 + (int64_t)c * R + r;
  if (k >= m) return;
  double a = 0.0;
  for (int q = 0; q < nparts; q++) a += part[((int64_t)c * nparts + q) * R + r];
  var[k] -= a;
}

template <class St>
void variance_impl(gp_ctx* ctx, gp_factor_t* f, const St& store, int b, const double* d_Xt, int64_t m,
                   double* d_var) {
  using V = typename St::V;
  gp_pointset* ps = f->ps;
  const SymPlan& sp = ps->sp;
  const DevPlan& dp = ps->dp;
  cudaStream_t st = ctx->stream;
  const int64_t n = ps->n, ns = sp.ns, FR = sp.sn_frow[ns];
  const int64_t cs = (FR + n) * R;
  const int64_t per_chunk = cs * (int64_t)sizeof(V) + ns + SUM_CTAS * R * 8;
  const int64_t want = (m + R - 1) / R;
  if (!f->var_work) {   // workspace for NC chunks, allocated once per factor
    size_t freeb = 0, totb = 0;
    GP_CUDA(cudaMemGetInfo(&freeb, &totb));
    const int64_t cap = std::min<int64_t>((int64_t)4 << 30, (int64_t)(freeb / 4));
    int64_t nc = std::max<int64_t>(1, std::min<int64_t>(64, cap / per_chunk));
    if (ctx->budget) nc = std::max<int64_t>(1, std::min<int64_t>(nc, (int64_t)(ctx->budget - std::min(ctx->budget, ctx->held.load())) / per_chunk));
    f->var_nc = (int)nc;
    f->var_work = dalloc<uint8_t>(ctx, f->bufs, (size_t)(nc * per_chunk) + 256);
  }
  const int NC = (int)std::min<int64_t>(f->var_nc, want);
  VarWork<V> vw;
  vw.F = reinterpret_cast<V*>(f->var_work);
  vw.X = vw.F + FR * R;
  vw.cs = cs;
  vw.active = f->var_work + (size_t)f->var_nc * cs * sizeof(V);
  vw.ns = ns;
  double* part = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(vw.active + (size_t)f->var_nc * ns) + 15) &
                                           ~(uintptr_t)15);
  const tp::GridInfo g = tp::grid_of(ps);
  const gp_hyper& h0 = f->thetas_host[0];
  const double* theta = f->theta_dev + (int64_t)b * f->theta_stride;
  const double* Fb = f->F + (int64_t)b * n * h0.n1;
  const double* Cb = f->Cpt ? f->Cpt + (int64_t)b * n * 2 : nullptr;
  const size_t step_smem = (size_t)(T * (T + 1) + T * R) * sizeof(V);
  static_assert(sizeof(V) == 4 || sizeof(V) == 8, "working type");
  GP_CUDA(cudaFuncSetAttribute(k_var_step<St>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem));
  ProfScope ps_(ctx, KC_PREDICT);
  for (int64_t k0 = 0; k0 < m; k0 += (int64_t)NC * R) {
    const int64_t cnt = std::min<int64_t>(m - k0, (int64_t)NC * R);
    const int nc = (int)((cnt + R - 1) / R);
    GP_CUDA(cudaMemsetAsync(vw.active, 0, (size_t)nc * ns, st));
    for (int c = 0; c < nc; c++)
      GP_CUDA(cudaMemsetAsync(vw.X + c * cs, 0, (size_t)n * R * sizeof(V), st));
    k_var_mark<<<grid_for(cnt, 8), 256, 0, st>>>(d_Xt, m, k0, g, ps->X, ps->Us, ps->cell_perm, ps->cell_start, theta,
                                                h0.n1, h0.n2, h0.bump_dims, Fb, Cb, ps->pinv, dp, vw.active, ns,
                                                d_var);
    GP_CHECK_LAUNCH(ctx);
    k_var_zero<V><<<dim3(grid_for(ns, 8), nc), 256, 0, st>>>(dp, ns, vw);
    GP_CHECK_LAUNCH(ctx);
    k_var_scatter<V><<<grid_for(cnt, 8), 256, 0, st>>>(d_Xt, m, k0, g, ps->X, ps->Us, ps->cell_perm, ps->cell_start,
                                                       theta, h0.n1, h0.n2, h0.bump_dims, Fb, Cb, ps->pinv, dp, vw);
    GP_CHECK_LAUNCH(ctx);
    for (int32_t L = 0; L < sp.nlevels; L++) {
      const SymPlan::Level& lv = sp.levels[L];
      const int32_t nl = sp.lev_ptr[L + 1] - sp.lev_ptr[L];
      if (L > 0) {
        k_var_gather<V><<<dim3(nl, nc), 256, 0, st>>>(dp.lev_sn + sp.lev_ptr[L], dp, vw);
        GP_CHECK_LAUNCH(ctx);
      }
      if (lv.nsmall > 0) {
        k_var_small<St><<<dim3(lv.nsmall, nc), 256, 0, st>>>(dp.small_list + lv.small_off, dp, store, b, vw);
        GP_CHECK_LAUNCH(ctx);
      }
      for (const auto& stp : lv.steps) {
        k_var_step<St><<<dim3((unsigned)(stp.nfront + stp.trsm_total), nc), 256, step_smem, st>>>(
            dp.large_fronts + stp.fr_off, dp.step_pre + stp.pre_off, stp.nfront, stp.kb, dp, store, b, vw);
        GP_CHECK_LAUNCH(ctx);
      }
    }
    k_var_sumsq<V><<<dim3(SUM_CTAS, nc), 256, 0, st>>>(n, vw, part);
    GP_CHECK_LAUNCH(ctx);
    k_var_final<<<nc, R, 0, st>>>(part, SUM_CTAS, m, k0, d_var);
    GP_CHECK_LAUNCH(ctx);
  }
}

}  // namespace

void variance_run(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_Xt, int64_t m, double* d_var) {
  const SymPlan& sp = f->ps->sp;
  if (f->prec == GP_FP64) {
    fa::StoreF64 store{f->panels, sp.panel_entries, f->dinv, sp.diag_entries};
    variance_impl(ctx, f, store, b, d_Xt, m, d_var);
  } else {
    fa::StoreMix store{f->panels32, f->diag, sp.panel32_entries, sp.diag_entries, f->dinv32};
    variance_impl(ctx, f, store, b, d_Xt, m, d_var);
  }
}
