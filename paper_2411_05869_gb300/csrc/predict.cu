// predict.cu -- step A12: predictive mean m*_k = mu*_k + sum_j C_y(x*_k, x_j) alpha_j (Sec. 3.2), where the
// sum runs over the training points in the 3^d cells around x*_k (C_y vanishes beyond the core support, so
// these are all the nonzero terms) and no noise term enters (C_{y,z} = C_y off the observation diagonal).
// One warp per test point: bump features of x* first, then the lanes stride over each cell's points with a
// fixed lane assignment and a fixed shuffle tree, so the sum is reproducible.
#include <cmath>

#include "gp_internal.cuh"

namespace {

__device__ __forceinline__ double wendland(double q) {
  if (!(q < 1.0)) return 0.0;
  double t = 1.0 - q;
  double t2 = t * t, t4 = t2 * t2, t8 = t4 * t4;
  double poly = ((35.0 * q + 25.0) * q + 8.0) * q + 1.0;
  return t8 * poly;
}

struct GridInfo {
  int d;
  long long c0[3], nc[3];
  double rho[3];
};

__global__ void k_predict(const double* __restrict__ Xt, int64_t m, const double* __restrict__ mu, GridInfo g,
                          const double* __restrict__ X, const double* __restrict__ Us,
                          const int32_t* __restrict__ cell_perm, const int64_t* __restrict__ cell_start,
                          const double* __restrict__ theta, int n1, int n2, int bd, const double* __restrict__ F,
                          const double* __restrict__ alpha, double* __restrict__ mean) {
  __shared__ double fs[8][GP_MAX_N1];
  __shared__ double gs[8][64];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  int64_t k = (int64_t)blockIdx.x * 8 + wi;
  if (k >= m) return;   // whole warps exit together
  const int d = g.d;
  double xs[3] = {0, 0, 0}, us[3] = {0, 0, 0};
  for (int c = 0; c < d; c++) {
    xs[c] = Xt[k * d + c];
    us[c] = xs[c] / g.rho[c];
  }
  // bump features f_i(x*) = sum_j g_ij(x*): lanes evaluate bumps, lane i sums its family in j order
  const int nb = n1 * n2, per = bd + 3;
  for (int base = 0; base < nb; base += 64) {
    for (int q = lane; q < 64; q += 32) {
      int ij = base + q;
      double gval = 0.0;
      if (ij < nb) {
        const double* p = theta + TH_BUMPS + (int64_t)ij * per;
        double s = 0.0;
        for (int c = 0; c < bd; c++) {
          double dc = xs[c] - p[c];
          s = __dadd_rn(s, __dmul_rn(dc, dc));
        }
        double r = p[bd + 2], rr = r * r;
        if (s < rr) {
          double t = s / rr;
          gval = p[bd] * exp(p[bd + 1] * (1.0 - 1.0 / (1.0 - t)));
        }
      }
      gs[wi][q] = gval;
    }
    __syncwarp();
    if (lane < n1) {
      double acc = base == 0 ? 0.0 : fs[wi][lane];
      for (int j = 0; j < n2; j++) {
        int ij = lane * n2 + j;
        if (ij >= base && ij < base + 64) acc += gs[wi][ij - base];
      }
      fs[wi][lane] = acc;
    }
    __syncwarp();
  }
  bool same = true;
  for (int c = 0; c < d; c++) same = same && theta[TH_R0 + c] == theta[TH_CRAD + c];
  double total = 0.0;
  bool inside = true;
  long long ci[3] = {0, 0, 0};
  for (int c = 0; c < d; c++) {
    double fl = floor(us[c]);
    if (!(fl >= (double)(g.c0[c] - 2) && fl <= (double)(g.c0[c] + g.nc[c] + 1))) inside = false;
    else ci[c] = (long long)fl - g.c0[c];
  }
  if (inside) {
    int ncell = 1;
    for (int c = 0; c < d; c++) ncell *= 3;
    for (int t = 0; t < ncell; t++) {
      long long cc[3] = {0, 0, 0};
      int tt = t;
      bool ok = true;
      for (int c = 0; c < d; c++) {
        cc[c] = ci[c] + (tt % 3) - 1;
        tt /= 3;
        if (cc[c] < 0 || cc[c] >= g.nc[c]) ok = false;
      }
      if (!ok) continue;
      long long cell = 0;
      for (int c = d - 1; c >= 0; c--) cell = cell * g.nc[c] + cc[c];
      for (int64_t q = cell_start[cell] + lane; q < cell_start[cell + 1]; q += 32) {
        double q2 = 0.0;
        for (int c = 0; c < d; c++) {
          double dk = __dsub_rn(us[c], Us[q * d + c]);
          q2 = __dadd_rn(q2, __dmul_rn(dk, dk));
        }
        double wc = wendland(__dsqrt_rn(q2));
        if (wc == 0.0) continue;
        int32_t j = cell_perm[q];
        double w0 = wc;
        if (!same) {
          double s = 0.0;
          for (int c = 0; c < d; c++) {
            double dk = __dsub_rn(__ddiv_rn(xs[c], theta[TH_R0 + c]), __ddiv_rn(X[(int64_t)j * d + c], theta[TH_R0 + c]));
            s = __dadd_rn(s, __dmul_rn(dk, dk));
          }
          w0 = wendland(__dsqrt_rn(s));
        }
        double acc = theta[TH_S0] * w0;
        for (int i = 0; i < n1; i++) acc += fs[wi][i] * F[(int64_t)j * n1 + i];
        total += (theta[TH_CORE_VAR] * wc) * acc * alpha[j];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  if (lane == 0) mean[k] = (mu ? mu[k] : 0.0) + total;
}

}  // namespace

void predict_run(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_Xt, int64_t m, const double* d_mu, double* d_mean) {
  gp_pointset* ps = f->ps;
  const gp_hyper& h0 = f->thetas_host[0];
  GridInfo g{};
  g.d = ps->d;
  for (int c = 0; c < 3; c++) {
    g.c0[c] = ps->c0[c];
    g.nc[c] = ps->nc[c];
    g.rho[c] = ps->rho[c];
  }
  const double* theta = f->theta_dev + (int64_t)b * f->theta_stride;
  const double* F = f->F + (int64_t)b * ps->n * h0.n1;
  ProfScope ps_(ctx, KC_PREDICT);
  k_predict<<<grid_for(m, 8), 256, 0, ctx->stream>>>(d_Xt, m, d_mu, g, ps->X, ps->Us, ps->cell_perm, ps->cell_start,
                                                     theta, h0.n1, h0.n2, h0.bump_dims, F,
                                                     f->alpha + (int64_t)b * ps->n, d_mean);
  GP_CHECK_LAUNCH(ctx);
}
