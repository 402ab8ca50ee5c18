// values.cu -- steps A3 (bump features) and A4 (kernel values of the pattern, scattered into the supernodal
// panels), plus the one-off map from CSR entries to panel offsets.
//
// A3: f_i(x) = sum_{j=1..n2} g_ij(x), g(x) = a exp{b [1 - (1 - |x-h|^2/r^2)^{-1}]} for |x-h|^2 < r^2 and 0
//     otherwise (Sec. 2.1, Eq. bumpFcn and the sum of bumps), over the leading bump_dims coordinates.
// A4: C_z(x_i, x_j) = core_var f0(q_c) [s0 f0(q_0) + sum_i f_i(x_i) f_i(x_j)] + tau^2 [i = j]
//     (Eq. C_sparse, C_y = C_core x C_sparse, Eq. Zcov), f0(q) = (1-q)^8 (35 q^3 + 25 q^2 + 8 q + 1) for q < 1
//     (Eq. compSupp, cubic coefficient as printed). q_c uses the core radii (the cached u = x / core_radius,
//     exactly the pattern's differences), q_0 the Wendland radii r0 (reused when r0 = core radius).
//     One warp per pattern row; every entry writes the CSR value (for refinement residuals) and, when it lies
//     in the lower triangle of P C_z P^T, its panel slot.
#include "gp_internal.cuh"
#include "testpoint.cuh"

namespace {

__device__ __forceinline__ double wendland(double q) {
  if (!(q < 1.0)) return 0.0;
  double t = 1.0 - q;
  double t2 = t * t, t4 = t2 * t2, t8 = t4 * t4;
  double poly = ((35.0 * q + 25.0) * q + 8.0) * q + 1.0;
  return t8 * poly;
}

__global__ void k_features(const double* __restrict__ X, int64_t n, int d, const double* __restrict__ theta,
                           int64_t tstride, int n1, int n2, int bd, double* __restrict__ F, double* __restrict__ Cpt) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (k >= n) return;
  if (Cpt) tp::core_point(theta + (int64_t)b * tstride, X + k * d, d, Cpt + ((int64_t)b * n + k) * 2);
  const double* th = theta + (int64_t)b * tstride + TH_BUMPS;
  const int per = bd + 3;
  double x[3] = {0, 0, 0};
  for (int c = 0; c < bd; c++) x[c] = X[k * d + c];
  double* out = F + ((int64_t)b * n + k) * n1;
  for (int i = 0; i < n1; i++) {
    double acc = 0.0;
    for (int j = 0; j < n2; j++) {
      const double* p = th + (int64_t)(i * n2 + j) * per;
      double s = 0.0;
      for (int c = 0; c < bd; c++) {
        double dc = x[c] - p[c];
        s = __dadd_rn(s, __dmul_rn(dc, dc));
      }
      double r = p[bd + 2], rr = r * r;
      double g = 0.0;
      if (s < rr) {
        double t = s / rr;
        g = p[bd] * exp(p[bd + 1] * (1.0 - 1.0 / (1.0 - t)));
      }
      acc += g;
    }
    out[i] = acc;
  }
}

// Warp per row of the pattern; B proposals per entry (geometry shared). MIXED: lower entries go to the
// FP32 row-major panels or, inside a 64 x 64 diagonal block, to the FP64 diagonal tiles (dest flag bit).
template <bool MIXED>
__global__ void k_values(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n, int d,
                         const double* __restrict__ U, const double* __restrict__ X,
                         const double* __restrict__ theta, int64_t tstride, int B, int n1,
                         const double* __restrict__ F, const double* __restrict__ Cpt,
                         const int64_t* __restrict__ dest, int64_t nnz,
                         int64_t panel_entries, double* __restrict__ val, double* __restrict__ panels,
                         float* __restrict__ p32, double* __restrict__ diag, int64_t diag_entries) {
  int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  double ui[3] = {0, 0, 0}, xi[3] = {0, 0, 0};
  for (int k = 0; k < d; k++) {
    ui[k] = U[i * d + k];
    xi[k] = X[i * d + k];
  }
  for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
    int32_t j = col[e];
    double q2 = 0.0;
    for (int k = 0; k < d; k++) {
      double dk = __dsub_rn(ui[k], U[(int64_t)j * d + k]);
      q2 = __dadd_rn(q2, __dmul_rn(dk, dk));
    }
    double wc = wendland(__dsqrt_rn(q2));
    int64_t de = dest[e];
    for (int b = 0; b < B; b++) {
      const double* th = theta + (int64_t)b * tstride;
      double v = 0.0;
      if (th[TH_KIND] != 0.0) {   // non-compact core: C_core(x_i, x_j) C_sparse, f0 of q0 from u = x / r0
        double acc = th[TH_S0] * wc;
        const double* Fi = F + ((int64_t)b * n + i) * n1;
        const double* Fj = F + ((int64_t)b * n + j) * n1;
        for (int k = 0; k < n1; k++) acc += Fi[k] * Fj[k];
        if (acc != 0.0)
          v = tp::core_paciorek(Cpt + ((int64_t)b * n + i) * 2, Cpt + ((int64_t)b * n + j) * 2, xi,
                                X + (int64_t)j * d, d) * acc;
      } else if (wc != 0.0) {
        double w0 = wc;
        bool same = true;
        for (int k = 0; k < d; k++) same = same && th[TH_R0 + k] == th[TH_CRAD + k];
        if (!same) {
          double s = 0.0;
          for (int k = 0; k < d; k++) {
            double dk = __dsub_rn(__ddiv_rn(xi[k], th[TH_R0 + k]), __ddiv_rn(X[(int64_t)j * d + k], th[TH_R0 + k]));
            s = __dadd_rn(s, __dmul_rn(dk, dk));
          }
          w0 = wendland(__dsqrt_rn(s));
        }
        double acc = th[TH_S0] * w0;
        const double* Fi = F + ((int64_t)b * n + i) * n1;
        const double* Fj = F + ((int64_t)b * n + j) * n1;
        for (int k = 0; k < n1; k++) acc += Fi[k] * Fj[k];
        v = (th[TH_CORE_VAR] * wc) * acc;
      }
      if (j == i) v += th[TH_NOISE];
      val[(int64_t)b * nnz + e] = v;
      if (MIXED) {
        if (de >= 0) {
          if (de & DIAG_FLAG) diag[(int64_t)b * diag_entries + (de & ~DIAG_FLAG)] = v;
          else p32[(int64_t)b * panel_entries + de] = (float)v;
        }
      } else if (de >= 0) {
        panels[(int64_t)b * panel_entries + de] = v;
      }
    }
  }
}

__global__ void k_inverse_perm(const int32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ pinv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pinv[perm[i]] = (int32_t)i;
}

// dest[e] = panel offset of entry e = (i, j) when pinv[i] >= pinv[j], else -1.
__global__ void k_dest(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n,
                       const int32_t* __restrict__ pinv, DevPlan dp, int64_t* __restrict__ dest) {
  int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  int32_t pi = pinv[i];
  for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
    int32_t pj = pinv[col[e]];
    if (pi < pj) {
      dest[e] = -1;
      continue;
    }
    int32_t s = dp.sn_of_col[pj];
    int32_t f = dp.sn_first[s], w = dp.w[s], r = dp.r[s];
    int64_t m = (int64_t)w + r;
    int64_t lr;
    if (pi < f + w) {
      lr = pi - f;
    } else {
      const int32_t* R = dp.frows + dp.frow_off[s] + w;
      int lo = 0, hi = r;   // first index with R[idx] >= pi
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (R[mid] < pi) lo = mid + 1;
        else hi = mid;
      }
      if (lo == r || R[lo] != pi) {   // cannot happen for a consistent plan; never write outside the panel
        dest[e] = -1;
        continue;
      }
      lr = w + lo;
    }
    dest[e] = dp.loff[s] + (int64_t)(pj - f) * m + lr;
  }
}

}  // namespace

void compute_dest_map(gp_ctx* ctx, gp_pointset* ps) {
  const int64_t n = ps->n;
  k_inverse_perm<<<grid_for(n, 256), 256, 0, ctx->stream>>>(ps->perm, n, ps->pinv);
  GP_CHECK_LAUNCH(ctx);
  ps->dest = dalloc<int64_t>(ctx, ps->bufs, ps->nnz);
  k_dest<<<grid_for(n * 32, 256), 256, 0, ctx->stream>>>(ps->rowptr, ps->col, n, ps->pinv, ps->dp, ps->dest);
  GP_CHECK_LAUNCH(ctx);
}

void values_run(gp_ctx* ctx, gp_factor_t* f) {
  gp_pointset* ps = f->ps;
  const int64_t n = ps->n;
  const gp_hyper& h0 = f->thetas_host[0];
  dim3 gf(grid_for(n, 128), f->B);
  if (h0.n1 > 0 || f->Cpt) {
    k_features<<<gf, 128, 0, ctx->stream>>>(ps->X, n, ps->d, f->theta_dev, f->theta_stride, h0.n1, h0.n2,
                                            h0.bump_dims, f->F, f->Cpt);
    GP_CHECK_LAUNCH(ctx);
  }
  GP_CUDA(cudaMemsetAsync(f->panels, 0, sizeof(double) * (size_t)f->B * ps->sp.panel_entries, ctx->stream));
  ProfScope ps_(ctx, KC_VALUES);
  k_values<false><<<grid_for(n * 32, 256), 256, 0, ctx->stream>>>(
      ps->rowptr, ps->col, n, ps->d, ps->U, ps->X, f->theta_dev, f->theta_stride, f->B, h0.n1, f->F, f->Cpt,
      ps->dest, ps->nnz, ps->sp.panel_entries, f->val, f->panels, nullptr, nullptr, 0);
  GP_CHECK_LAUNCH(ctx);
}

void values_run_mixed(gp_ctx* ctx, gp_factor_t* f) {
  gp_pointset* ps = f->ps;
  const SymPlan& sp = ps->sp;
  const int64_t n = ps->n;
  const gp_hyper& h0 = f->thetas_host[0];
  dim3 gf(grid_for(n, 128), f->B);
  if (h0.n1 > 0 || f->Cpt) {
    k_features<<<gf, 128, 0, ctx->stream>>>(ps->X, n, ps->d, f->theta_dev, f->theta_stride, h0.n1, h0.n2,
                                            h0.bump_dims, f->F, f->Cpt);
    GP_CHECK_LAUNCH(ctx);
  }
  GP_CUDA(cudaMemsetAsync(f->panels32, 0, sizeof(float) * (size_t)f->B * sp.panel32_entries, ctx->stream));
  GP_CUDA(cudaMemsetAsync(f->diag, 0, sizeof(double) * (size_t)f->B * sp.diag_entries, ctx->stream));
  ProfScope ps_(ctx, KC_VALUES);
  k_values<true><<<grid_for(n * 32, 256), 256, 0, ctx->stream>>>(
      ps->rowptr, ps->col, n, ps->d, ps->U, ps->X, f->theta_dev, f->theta_stride, f->B, h0.n1, f->F, f->Cpt,
      ps->dest32, ps->nnz, sp.panel32_entries, f->val, nullptr, f->panels32, f->diag, sp.diag_entries);
  GP_CHECK_LAUNCH(ctx);
}
