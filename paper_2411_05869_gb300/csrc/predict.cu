// predict.cu -- step A12: predictive mean m*_k = mu*_k + sum_j C_y(x*_k, x_j) alpha_j (Sec. 3.2), where the
// sum runs over the training points in the 3^d cells around x*_k (C_y vanishes beyond the core support, so
// these are all the nonzero terms) and no noise term enters (C_{y,z} = C_y off the observation diagonal).
// One warp per test point: bump features of x* first, then the lanes stride over each cell's points with a
// fixed lane assignment and a fixed shuffle tree, so the sum is reproducible.
#include "gp_internal.cuh"
#include "testpoint.cuh"

namespace {

__global__ void k_predict(const double* __restrict__ Xt, int64_t m, const double* __restrict__ mu, tp::GridInfo g,
                          const double* __restrict__ X, const double* __restrict__ Us,
                          const int32_t* __restrict__ cell_perm, const int64_t* __restrict__ cell_start,
                          const double* __restrict__ theta, int n1, int n2, int bd, const double* __restrict__ F,
                          const double* __restrict__ Cpt, const double* __restrict__ alpha,
                          double* __restrict__ mean) {
  __shared__ double fs[8][GP_MAX_N1];
  __shared__ double gs[8][64];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  int64_t k = (int64_t)blockIdx.x * 8 + wi;
  if (k >= m) return;   // whole warps exit together
  const tp::TestPoint p = tp::load_features(Xt, k, g, theta, n1, n2, bd, fs[wi], gs[wi]);
  double total = 0.0;
  tp::for_each_neighbour(p, g, X, Us, cell_perm, cell_start, theta, n1, fs[wi], F, Cpt,
                         [&](int32_t j, double cy) { total += cy * alpha[j]; });
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  if (lane == 0) mean[k] = (mu ? mu[k] : 0.0) + total;
}

}  // namespace

void predict_run(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_Xt, int64_t m, const double* d_mu, double* d_mean) {
  gp_pointset* ps = f->ps;
  const gp_hyper& h0 = f->thetas_host[0];
  const tp::GridInfo g = tp::grid_of(ps);
  const double* theta = f->theta_dev + (int64_t)b * f->theta_stride;
  const double* F = f->F + (int64_t)b * ps->n * h0.n1;
  ProfScope ps_(ctx, KC_PREDICT);
  k_predict<<<grid_for(m, 8), 256, 0, ctx->stream>>>(d_Xt, m, d_mu, g, ps->X, ps->Us, ps->cell_perm, ps->cell_start,
                                                     theta, h0.n1, h0.n2, h0.bump_dims, F,
                                                     f->Cpt ? f->Cpt + (int64_t)b * ps->n * 2 : nullptr,
                                                     f->alpha + (int64_t)b * ps->n, d_mean);
  GP_CHECK_LAUNCH(ctx);
}
