// testpoint.cuh -- the terms of C_y(x*, x_j) for one test point x* and its training neighbours (Sec. 3.2), shared by
// the predictive mean and the predictive variance. One warp per test point: the bump features f_i(x*) first, then
// the lanes stride over the training points of the 3^d cells of the unit grid in u = x / core_radius around x*
// with a fixed lane assignment (C_y vanishes beyond the core support, so these hold every nonzero term):
//   C_y(x*, x_j) = core_var f0(q_c) [s0 f0(q_0) + sum_i f_i(x*) f_i(x_j)]   (Eq. C_sparse, C_y = C_core x C_sparse)
// with q_c from the cached u of the cell order and q_0 from x / r0 when r0 differs from the core radius.
#pragma once
#include <cmath>

#include "gp_internal.cuh"

namespace tp {

__device__ __forceinline__ double wendland(double q) {
  if (!(q < 1.0)) return 0.0;
  double t = 1.0 - q;
  double t2 = t * t, t4 = t2 * t2, t8 = t4 * t4;
  double poly = ((35.0 * q + 25.0) * q + 8.0) * q + 1.0;
  return t8 * poly;
}

// The non-compact core of App. B (Eq. PScov), smoothness 3/2: per point sigma(x) and Sigma(x) (log-linear in the
// coordinates), then C_core(x, x') = sigma sigma' (Sigma Sigma')^(d/4) / ((Sigma + Sigma') / 2)^(d/2) M(sqrt(Q)),
// Q = |x - x'|^2 / ((Sigma + Sigma') / 2), M(t) = (1 + sqrt(3) t) exp(-sqrt(3) t). Separately rounded operations.
__device__ __forceinline__ void core_point(const double* __restrict__ th, const double* __restrict__ x, int d,
                                           double* out) {
  double ls = log(th[TH_SIG0]), lS = log(th[TH_SIGMA0]);
  for (int k = 0; k < d; k++) {
    ls = __dadd_rn(ls, __dmul_rn(th[TH_PHIS + k], x[k]));
    lS = __dadd_rn(lS, __dmul_rn(th[TH_PHIS2 + k], x[k]));
  }
  out[0] = exp(ls);
  out[1] = exp(lS);
}
__device__ __forceinline__ double core_paciorek(const double* ci, const double* cj, const double* xi,
                                                const double* xj, int d) {
  const double avg = __dmul_rn(__dadd_rn(ci[1], cj[1]), 0.5);
  const double pref = __ddiv_rn(__dmul_rn(__dmul_rn(ci[0], cj[0]), pow(__dmul_rn(ci[1], cj[1]), d / 4.0)),
                                pow(avg, d / 2.0));
  double r2 = 0.0;
  for (int k = 0; k < d; k++) {
    const double dk = __dsub_rn(xi[k], xj[k]);
    r2 = __dadd_rn(r2, __dmul_rn(dk, dk));
  }
  const double st = __dmul_rn(sqrt(3.0), __dsqrt_rn(__ddiv_rn(r2, avg)));
  return __dmul_rn(pref, __dmul_rn(__dadd_rn(1.0, st), exp(-st)));
}

struct GridInfo {
  int d;
  long long c0[3], nc[3];
  double rho[3];
};

inline GridInfo grid_of(const gp_pointset* ps) {
  GridInfo g{};
  g.d = ps->d;
  for (int c = 0; c < 3; c++) {
    g.c0[c] = ps->c0[c];
    g.nc[c] = ps->nc[c];
    g.rho[c] = ps->rho[c];
  }
  return g;
}

// The warp's test point: coordinates, scaled coordinates and bump features (fs: the warp's n1 slots, gs: 64
// scratch slots, both in shared memory).
struct TestPoint {
  double xs[3], us[3];
};

__device__ __forceinline__ TestPoint load_features(const double* __restrict__ Xt, int64_t k, const GridInfo& g,
                                                   const double* __restrict__ theta, int n1, int n2, int bd,
                                                   double* fs, double* gs) {
  const int lane = threadIdx.x & 31;
  const int d = g.d;
  TestPoint p{{0, 0, 0}, {0, 0, 0}};
  for (int c = 0; c < d; c++) {
    p.xs[c] = Xt[k * d + c];
    p.us[c] = p.xs[c] / g.rho[c];
  }
  // f_i(x*) = sum_j g_ij(x*): lanes evaluate bumps, lane i sums its family in j order
  const int nb = n1 * n2, per = bd + 3;
  for (int base = 0; base < nb; base += 64) {
    for (int q = lane; q < 64; q += 32) {
      int ij = base + q;
      double gval = 0.0;
      if (ij < nb) {
        const double* b = theta + TH_BUMPS + (int64_t)ij * per;
        double s = 0.0;
        for (int c = 0; c < bd; c++) {
          double dc = p.xs[c] - b[c];
          s = __dadd_rn(s, __dmul_rn(dc, dc));
        }
        double r = b[bd + 2], rr = r * r;
        if (s < rr) {
          double t = s / rr;
          gval = b[bd] * exp(b[bd + 1] * (1.0 - 1.0 / (1.0 - t)));
        }
      }
      gs[q] = gval;
    }
    __syncwarp();
    if (lane < n1) {
      double acc = base == 0 ? 0.0 : fs[lane];
      for (int j = 0; j < n2; j++) {
        int ij = lane * n2 + j;
        if (ij >= base && ij < base + 64) acc += gs[ij - base];
      }
      fs[lane] = acc;
    }
    __syncwarp();
  }
  return p;
}

// Calls fn(j, cy) for every training point j (original index) with C_y(x*, x_j) != 0, lane by lane (lane `lane`
// of the warp visits the cells' points lane, lane + 32, ...). With the non-compact core (theta kind 1, Cpt the
// training points' sigma and Sigma) every training point is visited: C_sparse decides which terms are nonzero.
template <class Fn>
__device__ __forceinline__ void for_each_neighbour(const TestPoint& p, const GridInfo& g,
                                                   const double* __restrict__ X, const double* __restrict__ Us,
                                                   const int32_t* __restrict__ cell_perm,
                                                   const int64_t* __restrict__ cell_start,
                                                   const double* __restrict__ theta, int n1, const double* fs,
                                                   const double* __restrict__ F, const double* __restrict__ Cpt,
                                                   Fn&& fn) {
  const int lane = threadIdx.x & 31;
  const int d = g.d;
  if (theta[TH_KIND] != 0.0) {
    double cs[2];
    core_point(theta, p.xs, d, cs);
    const int64_t n = cell_start[g.nc[0] * g.nc[1] * g.nc[2]];
    for (int64_t q = lane; q < n; q += 32) {
      double q2 = 0.0;
      for (int c = 0; c < d; c++) {
        double dk = __dsub_rn(p.us[c], Us[q * d + c]);
        q2 = __dadd_rn(q2, __dmul_rn(dk, dk));
      }
      const int32_t j = cell_perm[q];
      double acc = theta[TH_S0] * wendland(__dsqrt_rn(q2));
      for (int i = 0; i < n1; i++) acc += fs[i] * F[(int64_t)j * n1 + i];
      if (acc == 0.0) continue;
      fn(j, core_paciorek(cs, Cpt + (int64_t)j * 2, p.xs, X + (int64_t)j * d, d) * acc);
    }
    return;
  }
  bool same = true;
  for (int c = 0; c < d; c++) same = same && theta[TH_R0 + c] == theta[TH_CRAD + c];
  bool inside = true;
  long long ci[3] = {0, 0, 0};
  for (int c = 0; c < d; c++) {
    double fl = floor(p.us[c]);
    if (!(fl >= (double)(g.c0[c] - 2) && fl <= (double)(g.c0[c] + g.nc[c] + 1))) inside = false;
    else ci[c] = (long long)fl - g.c0[c];
  }
  if (!inside) return;
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
        double dk = __dsub_rn(p.us[c], Us[q * d + c]);
        q2 = __dadd_rn(q2, __dmul_rn(dk, dk));
      }
      double wc = wendland(__dsqrt_rn(q2));
      if (wc == 0.0) continue;
      int32_t j = cell_perm[q];
      double w0 = wc;
      if (!same) {
        double s = 0.0;
        for (int c = 0; c < d; c++) {
          double dk = __dsub_rn(__ddiv_rn(p.xs[c], theta[TH_R0 + c]), __ddiv_rn(X[(int64_t)j * d + c], theta[TH_R0 + c]));
          s = __dadd_rn(s, __dmul_rn(dk, dk));
        }
        w0 = wendland(__dsqrt_rn(s));
      }
      double acc = theta[TH_S0] * w0;
      for (int i = 0; i < n1; i++) acc += fs[i] * F[(int64_t)j * n1 + i];
      fn(j, (theta[TH_CORE_VAR] * wc) * acc);
    }
  }
}

}  // namespace tp
