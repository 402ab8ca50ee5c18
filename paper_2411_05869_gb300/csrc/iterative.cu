// iterative.cu -- the paper's own computation of the log-likelihood above 100k points (Sec. 3.3), as a comparison
// for the exact factorization: the log-determinant by stochastic Lanczos quadrature and the quadratic form by a
// MINRES solve, both on the CSR values of C_z that the factor's value step (A4) computed:
//   log det C_z ~ (1/P) sum_p |v_p|^2 sum_i U_{1i}^2 log theta_i   (T_k = U diag(theta) U^T, k Lanczos steps from
//                                                                    v_p / |v_p|, no reorthogonalisation;
//                                                                    Ubaru, Chen and Saad, 2017)
//   alpha ~ C_z^{-1} r by MINRES (Paige and Saunders, 1975), Lanczos form with Givens rotations, from a given
//   start, stopped when the residual estimate falls to tol |r|;
//   log p ~ -1/2 log det - 1/2 r^T alpha - n/2 log(2 pi).
// The P probe vectors run side by side (an n x P block, probes contiguous per row): one sparse product of the
// block per Lanczos step. Every sum has a fixed order (warp per row, fixed-shape block reductions), so results are
// reproducible. The small eigenproblems of T_k are solved on the device by the cyclic Jacobi method (Golub and Van
// Loan, Sec. 8.5), tracking only the first row of the eigenvector matrix.
#include <algorithm>
#include <cmath>

#include "gp_internal.cuh"

namespace {

constexpr int NPART = 512;    // partial sums per reduction (grid of the reduction kernels)

// Y[i][p] = sum_e val[e] X[col[e]][p] for p < P (warp per row, lane p, entries in order).
__global__ void k_spmm(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, int64_t n, int P, const double* __restrict__ X,
                       double* __restrict__ Y) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double acc = 0.0;
  if (lane < P)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) acc += val[e] * X[(int64_t)col[e] * P + lane];
  if (lane < P) Y[i * P + lane] = acc;
}

// y = C x for one vector (warp per row, lanes over the row's entries, fixed shuffle tree).
__global__ void k_spmv(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, int64_t n, const double* __restrict__ x,
                       double* __restrict__ y) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double acc = 0.0;
  for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) acc += val[e] * x[col[e]];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[i] = acc;
}

// Partial column dots part[blk][p] = sum over this block's rows of A[i][p] B[i][p] (A may be B), rows
// blk * 8 + (t >> 5) stepping by NPART * 8. Also applies, first, the Lanczos update
// W[i][p] -= a[p] Qc[i][p] + b[p] Qp[i][p] when Qc is given (and dots the updated W with itself).
__global__ void k_coldot(int64_t n, int P, double* __restrict__ A, const double* __restrict__ B,
                         const double* __restrict__ Qc, const double* __restrict__ Qp,
                         const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double sp[8][32];
  const int lane = threadIdx.x & 31, r8 = threadIdx.x >> 5;
  double acc = 0.0;
  if (lane < P) {
    for (int64_t i = (int64_t)blockIdx.x * 8 + r8; i < n; i += (int64_t)gridDim.x * 8) {
      const int64_t o = i * P + lane;
      double w = A[o];
      if (Qc) {
        w = w - a[lane] * Qc[o] - (Qp ? b[lane] * Qp[o] : 0.0);
        A[o] = w;
        acc += w * w;
      } else {
        acc += w * B[o];
      }
    }
  }
  sp[r8][lane] = acc;
  __syncthreads();
  if (r8 == 0) {
    double s = 0.0;
    for (int q = 0; q < 8; q++) s += sp[q][lane];
    part[(int64_t)blockIdx.x * 32 + lane] = s;
  }
}

// out[p] = sum_blk part[blk][p] in block order; mode 1: out[p] = sqrt of that.
__global__ void k_colsum(const double* __restrict__ part, int nparts, int P, int mode, double* __restrict__ out) {
  const int p = threadIdx.x;
  if (p >= P) return;
  double s = 0.0;
  for (int q = 0; q < nparts; q++) s += part[(int64_t)q * 32 + p];
  out[p] = mode == 1 ? sqrt(s) : s;
}

// Q[i][p] = V[p][i]: the caller's probes (P x n) into the n x P block.
__global__ void k_probes_in(int64_t n, int P, const double* __restrict__ V, double* __restrict__ Q) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * P) return;
  const int64_t i = e / P;
  const int p = (int)(e % P);
  Q[e] = V[(int64_t)p * n + i];
}

// X[i][p] *= 1 / s[p] (s[p] = 0 leaves zeros).
__global__ void k_colscale(int64_t n, int P, double* __restrict__ X, const double* __restrict__ s) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * P) return;
  const double v = s[e % P];
  X[e] = v > 0.0 ? X[e] / v : 0.0;
}

// One CTA per probe: the eigenpairs of T_k (k <= 64; alpha[j][p], beta[j][p] for j < k - 1) by cyclic Jacobi
// sweeps in shared memory, then gam[p] = |v_p|^2 sum_i U_{1i}^2 log theta_i. The Lanczos process ends early where
// beta falls to 1e-14 of |alpha| (an invariant Krylov space); T is cut there. A non-positive Ritz value sets
// gam[p] to NaN.
__global__ void k_slq_quadrature(const double* __restrict__ alpha, const double* __restrict__ beta, int k, int P,
                                 const double* __restrict__ vnorm2, double* __restrict__ gam) {
  __shared__ double M[64][65];
  __shared__ double u[64];
  __shared__ double cs[3];
  __shared__ int kk_s;
  const int p = blockIdx.x, t = threadIdx.x;   // 64 threads
  if (t == 0) {
    int kk = 1;
    while (kk < k && beta[(kk - 1) * P + p] > 1e-14 * fabs(alpha[(kk - 1) * P + p])) kk++;
    kk_s = kk;
  }
  __syncthreads();
  const int kk = kk_s;
  for (int r = 0; r < kk; r++) {
    double v = 0.0;
    if (t < kk) {
      if (t == r) v = alpha[r * P + p];
      else if (t == r + 1) v = beta[r * P + p];
      else if (t + 1 == r) v = beta[t * P + p];
    }
    M[r][t] = v;
  }
  u[t] = t == 0 ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 60; sweep++) {
    // off-diagonal size (thread 0, fixed order)
    if (t == 0) {
      double off = 0.0, dia = 0.0;
      for (int r = 0; r < kk; r++)
        for (int c = 0; c < kk; c++) {
          if (r == c) dia += M[r][c] * M[r][c];
          else off += M[r][c] * M[r][c];
        }
      cs[2] = off <= 1e-30 * dia ? 1.0 : 0.0;
    }
    __syncthreads();
    if (cs[2] != 0.0) break;
    for (int a = 0; a < kk - 1; a++)
      for (int b = a + 1; b < kk; b++) {
        if (t == 0) {
          const double apq = M[a][b];
          double c = 1.0, s = 0.0;
          if (apq != 0.0) {
            const double tau = (M[b][b] - M[a][a]) / (2.0 * apq);
            const double tt = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
          cs[0] = c;
          cs[1] = s;
        }
        __syncthreads();
        const double c = cs[0], s = cs[1];
        if (s != 0.0) {
          // columns a, b of M <- M J (J: c on the diagonal, s at (a, b), -s at (b, a))
          if (t < kk) {
            const double ma = M[t][a], mb = M[t][b];
            M[t][a] = c * ma - s * mb;
            M[t][b] = s * ma + c * mb;
          }
          if (t == 0) {
            const double ua = u[a], ub = u[b];
            u[a] = c * ua - s * ub;
            u[b] = s * ua + c * ub;
          }
          __syncthreads();
          // rows a, b of M <- J^T M
          if (t < kk) {
            const double ma = M[a][t], mb = M[b][t];
            M[a][t] = c * ma - s * mb;
            M[b][t] = s * ma + c * mb;
          }
        }
        __syncthreads();
      }
  }
  if (t == 0) {
    double s = 0.0;
    bool ok = true;
    for (int i = 0; i < kk; i++) {
      const double th = M[i][i];
      ok = ok && th > 0.0;
      s += u[i] * u[i] * log(th);
    }
    gam[p] = ok ? vnorm2[p] * s : NAN;
  }
}

// out[0] = mean over p of gam[p] (fixed order).
__global__ void k_mean(const double* __restrict__ gam, int P, double* __restrict__ out) {
  double s = 0.0;
  for (int p = 0; p < P; p++) s += gam[p];
  out[0] = s / (double)P;
}

// ------------------------------------------------------------------------------------------ MINRES
struct MinresState {
  double beta;      // beta_j (|p| of the previous step; beta_1 = |r_0|)
  double c2, s2, c1, s1;
  double phibar;
  double bnorm;
  double tol;
  // this step's coefficients
  double alpha, beta_next, eps, delta, gamma, phi;
  int32_t done;     // 1: converged (later steps do nothing), 2: breakdown
  int32_t iters;
};

// x = b - x (r0 = b - C x0 from y = C x0 in x), and partial sums of r0^2 and b^2.
__global__ void k_minres_r0(int64_t n, const double* __restrict__ b, const double* __restrict__ y,
                            double* __restrict__ r, double* __restrict__ part) {
  __shared__ double s1[256], s2[256];
  double a1 = 0.0, a2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = b[i] - y[i];
    r[i] = v;
    a1 += v * v;
    a2 += b[i] * b[i];
  }
  s1[threadIdx.x] = a1;
  s2[threadIdx.x] = a2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x * 2] = s1[0];
    part[blockIdx.x * 2 + 1] = s2[0];
  }
}

__global__ void k_minres_init(const double* __restrict__ part, int nparts, double tol, MinresState* st) {
  double a = 0.0, b = 0.0;
  for (int q = 0; q < nparts; q++) {
    a += part[q * 2];
    b += part[q * 2 + 1];
  }
  MinresState s{};
  s.beta = sqrt(a);
  s.bnorm = sqrt(b);
  s.c2 = s.c1 = 1.0;
  s.s2 = s.s1 = 0.0;
  s.phibar = s.beta;
  s.tol = tol;
  s.done = s.beta <= tol * s.bnorm ? 1 : 0;
  s.iters = 0;
  *st = s;
}

// v = r / beta_1 (v_prev, d1, d2 cleared).
__global__ void k_minres_v1(int64_t n, const double* __restrict__ r, const MinresState* st, double* __restrict__ v,
                            double* __restrict__ vp, double* __restrict__ d1, double* __restrict__ d2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  v[i] = st->beta > 0.0 ? r[i] / st->beta : 0.0;
  vp[i] = 0.0;
  d1[i] = 0.0;
  d2[i] = 0.0;
}

// p = C v - beta_j v_prev in place (p holds C v), and partial sums of v . p (mode 0); or p -= alpha v and partial
// sums of p . p (mode 1).
__global__ void k_minres_vec(int64_t n, int mode, double* __restrict__ p, const double* __restrict__ v,
                             const double* __restrict__ vp, const MinresState* st, double* __restrict__ part) {
  __shared__ double sm[256];
  const double beta = st->beta, alpha = st->alpha;
  const bool skip = st->done != 0;
  double acc = 0.0;
  if (!skip)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      double w = p[i];
      if (mode == 0) {
        w = w - beta * vp[i];
        p[i] = w;
        acc += v[i] * w;
      } else {
        w = w - alpha * v[i];
        p[i] = w;
        acc += w * w;
      }
    }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// The step's scalars: mode 0 sums alpha_j; mode 1 sums |p|^2 into beta_{j+1}, then the rotations: column j of T
// through rotations j - 2 and j - 1, rotation j zeroing beta_{j+1}, the solution coefficient phi and the new
// residual estimate phibar.
__global__ void k_minres_scalars(const double* __restrict__ part, int nparts, int mode, MinresState* st) {
  MinresState s = *st;
  if (s.done) return;
  double a = 0.0;
  for (int q = 0; q < nparts; q++) a += part[q];
  if (mode == 0) {
    st->alpha = a;
    return;
  }
  s.beta_next = sqrt(a);
  s.eps = s.s2 * s.beta;
  const double dbar = s.c2 * s.beta;
  s.delta = s.c1 * dbar + s.s1 * s.alpha;
  const double gbar = -s.s1 * dbar + s.c1 * s.alpha;
  s.gamma = hypot(gbar, s.beta_next);
  if (s.gamma == 0.0) {
    st->done = 2;
    return;
  }
  const double c = gbar / s.gamma, sn = s.beta_next / s.gamma;
  s.phi = c * s.phibar;
  s.phibar = -sn * s.phibar;
  s.iters += 1;
  *st = s;
  // the rotations move down for the next step (the vector kernel reads eps, delta, gamma, phi of this step)
  st->c2 = s.c1;
  st->s2 = s.s1;
  st->c1 = c;
  st->s1 = sn;
}

// d = (v - delta d1 - eps d2) / gamma into d2's storage, x += phi d; v_next = p / beta_{j+1} into p's storage.
// Then beta_j <- beta_{j+1} and the converged flag.
__global__ void k_minres_update(int64_t n, double* __restrict__ x, const double* __restrict__ v,
                                double* __restrict__ p, const double* __restrict__ d1, double* __restrict__ d2,
                                const MinresState* st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || st->done) return;
  const double d = (v[i] - st->delta * d1[i] - st->eps * d2[i]) / st->gamma;
  d2[i] = d;
  x[i] += st->phi * d;
  p[i] = st->beta_next > 0.0 ? p[i] / st->beta_next : 0.0;
}

__global__ void k_minres_advance(MinresState* st, int maxiter) {
  if (st->done) return;
  st->beta = st->beta_next;
  if (fabs(st->phibar) <= st->tol * st->bnorm || st->beta_next == 0.0) st->done = 1;
  else if (st->iters >= maxiter) st->done = 3;
}

// Fixed-order dot x . y (one CTA of 1024 threads, thread-strided sums then a tree).
__global__ void __launch_bounds__(1024) k_dot1(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                                               double* __restrict__ out) {
  __shared__ double sm[1024];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 1024) a += x[i] * y[i];
  sm[threadIdx.x] = a;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sm[0];
}

}  // namespace

// Workspace (doubles): Lanczos 3 n P, MINRES 7 n, partials NPART * 32, alpha/beta 2 k P, scalars.
void iterative_run(gp_ctx* ctx, gp_factor_t* f, int b, const double* d_resid, const double* d_probes,
                   const double* d_x0, const gp_iterative_opts& o, gp_iterative_result* res) {
  gp_pointset* ps = f->ps;
  const int64_t n = ps->n, nnz = ps->nnz;
  const int P = o.probes, k = o.lanczos_steps;
  cudaStream_t st = ctx->stream;
  const size_t need = (size_t)(3 * n * P + 7 * n + NPART * 32 + 2 * k * P + 4 * P + 64) * sizeof(double) +
                      sizeof(MinresState) + 256;
  if (f->it_bytes < need) {   // grown on demand, held until gp_factor_free
    f->it_work = dalloc<uint8_t>(ctx, f->bufs, need);
    f->it_bytes = need;
  }
  double* w0 = reinterpret_cast<double*>(f->it_work);
  double* Qp = w0;
  double* Qc = Qp + n * P;
  double* W = Qc + n * P;
  double* x = W + n * P;
  double* r = x + n;
  double* v = r + n;
  double* vp = v + n;
  double* pp = vp + n;
  double* d1 = pp + n;
  double* d2 = d1 + n;
  double* part = d2 + n;
  double* alpha = part + NPART * 32;
  double* beta = alpha + k * P;
  double* vn2 = beta + k * P;
  double* gam = vn2 + P;
  double* scal = gam + P;   // [0] logdet, [1] quad, [2] true residual^2, [3] |r|^2
  MinresState* ms = reinterpret_cast<MinresState*>(scal + 2 * P + 64);
  const double* val = f->val + (int64_t)b * nnz;
  const unsigned rows_grid = grid_for(n * 32, 256);
  const unsigned el_grid = grid_for(n, 256);
  // ---- stochastic Lanczos quadrature, P probes side by side
  k_probes_in<<<grid_for(n * P, 256), 256, 0, st>>>(n, P, d_probes, Qc);
  GP_CHECK_LAUNCH(ctx);
  k_coldot<<<NPART, 256, 0, st>>>(n, P, Qc, Qc, nullptr, nullptr, nullptr, nullptr, part);
  GP_CHECK_LAUNCH(ctx);
  k_colsum<<<1, 32, 0, st>>>(part, NPART, P, 0, vn2);
  GP_CHECK_LAUNCH(ctx);
  k_colsum<<<1, 32, 0, st>>>(part, NPART, P, 1, gam);   // |v_p| (scratch)
  GP_CHECK_LAUNCH(ctx);
  k_colscale<<<grid_for(n * P, 256), 256, 0, st>>>(n, P, Qc, gam);
  GP_CHECK_LAUNCH(ctx);
  GP_CUDA(cudaMemsetAsync(Qp, 0, sizeof(double) * (size_t)n * P, st));
  for (int j = 0; j < k; j++) {
    k_spmm<<<rows_grid, 256, 0, st>>>(ps->rowptr, ps->col, val, n, P, Qc, W);
    GP_CHECK_LAUNCH(ctx);
    k_coldot<<<NPART, 256, 0, st>>>(n, P, W, Qc, nullptr, nullptr, nullptr, nullptr, part);   // alpha_j
    GP_CHECK_LAUNCH(ctx);
    k_colsum<<<1, 32, 0, st>>>(part, NPART, P, 0, alpha + (int64_t)j * P);
    GP_CHECK_LAUNCH(ctx);
    if (j == k - 1) break;
    k_coldot<<<NPART, 256, 0, st>>>(n, P, W, nullptr, Qc, j > 0 ? Qp : nullptr, alpha + (int64_t)j * P,
                                    j > 0 ? beta + (int64_t)(j - 1) * P : nullptr, part);   // W update, |W|^2
    GP_CHECK_LAUNCH(ctx);
    k_colsum<<<1, 32, 0, st>>>(part, NPART, P, 1, beta + (int64_t)j * P);
    GP_CHECK_LAUNCH(ctx);
    k_colscale<<<grid_for(n * P, 256), 256, 0, st>>>(n, P, W, beta + (int64_t)j * P);
    GP_CHECK_LAUNCH(ctx);
    double* t = Qp;   // (Qp, Qc, W) <- (Qc, W, Qp)
    Qp = Qc;
    Qc = W;
    W = t;
  }
  k_slq_quadrature<<<P, 64, 0, st>>>(alpha, beta, k, P, vn2, gam);
  GP_CHECK_LAUNCH(ctx);
  k_mean<<<1, 1, 0, st>>>(gam, P, scal);
  GP_CHECK_LAUNCH(ctx);
  // ---- MINRES from x0
  if (d_x0) GP_CUDA(cudaMemcpyAsync(x, d_x0, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st));
  else GP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, st));
  k_spmv<<<rows_grid, 256, 0, st>>>(ps->rowptr, ps->col, val, n, x, pp);
  GP_CHECK_LAUNCH(ctx);
  k_minres_r0<<<NPART, 256, 0, st>>>(n, d_resid, pp, r, part);
  GP_CHECK_LAUNCH(ctx);
  k_minres_init<<<1, 1, 0, st>>>(part, NPART, o.tol, ms);
  GP_CHECK_LAUNCH(ctx);
  k_minres_v1<<<el_grid, 256, 0, st>>>(n, r, ms, v, vp, d1, d2);
  GP_CHECK_LAUNCH(ctx);
  MinresState hs{};
  for (int it = 0; it < o.max_iter;) {
    const int chunk = std::min(16, o.max_iter - it);
    for (int q = 0; q < chunk; q++) {
      k_spmv<<<rows_grid, 256, 0, st>>>(ps->rowptr, ps->col, val, n, v, pp);
      GP_CHECK_LAUNCH(ctx);
      k_minres_vec<<<NPART, 256, 0, st>>>(n, 0, pp, v, vp, ms, part);
      GP_CHECK_LAUNCH(ctx);
      k_minres_scalars<<<1, 1, 0, st>>>(part, NPART, 0, ms);
      GP_CHECK_LAUNCH(ctx);
      k_minres_vec<<<NPART, 256, 0, st>>>(n, 1, pp, v, vp, ms, part);
      GP_CHECK_LAUNCH(ctx);
      k_minres_scalars<<<1, 1, 0, st>>>(part, NPART, 1, ms);
      GP_CHECK_LAUNCH(ctx);
      k_minres_update<<<el_grid, 256, 0, st>>>(n, x, v, pp, d1, d2, ms);
      GP_CHECK_LAUNCH(ctx);
      k_minres_advance<<<1, 1, 0, st>>>(ms, o.max_iter);
      GP_CHECK_LAUNCH(ctx);
      // (vp, v, pp) <- (v, pp, vp); (d2, d1) <- (d1, d2): the new d was written into d2's storage
      double* t = vp;
      vp = v;
      v = pp;
      pp = t;
      t = d2;
      d2 = d1;
      d1 = t;
    }
    it += chunk;
    GP_CUDA(cudaMemcpyAsync(&hs, ms, sizeof(MinresState), cudaMemcpyDeviceToHost, st));
    GP_CUDA(cudaStreamSynchronize(st));
    if (hs.done) break;
  }
  // The pointer rotations above assume every launched step advanced; steps after convergence leave every vector
  // untouched (their kernels return at once), so x holds the last update either way.
  // ---- quadratic form and the true residual
  k_dot1<<<1, 1024, 0, st>>>(n, d_resid, x, scal + 1);
  GP_CHECK_LAUNCH(ctx);
  k_spmv<<<rows_grid, 256, 0, st>>>(ps->rowptr, ps->col, val, n, x, pp);
  GP_CHECK_LAUNCH(ctx);
  k_minres_r0<<<NPART, 256, 0, st>>>(n, d_resid, pp, r, part);
  GP_CHECK_LAUNCH(ctx);
  k_minres_init<<<1, 1, 0, st>>>(part, NPART, o.tol, ms + 1);
  GP_CHECK_LAUNCH(ctx);
  double h[2];
  MinresState fin{};
  GP_CUDA(cudaMemcpyAsync(h, scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaMemcpyAsync(&fin, ms + 1, sizeof(MinresState), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaMemcpyAsync(&hs, ms, sizeof(MinresState), cudaMemcpyDeviceToHost, st));
  GP_CUDA(cudaStreamSynchronize(st));
  res->logdet = h[0];
  res->quad = h[1];
  res->loglik = -0.5 * h[0] - 0.5 * h[1] - 0.5 * (double)n * std::log(2.0 * 3.14159265358979323846);
  res->minres_iters = hs.iters;
  res->minres_relres = hs.bnorm > 0.0 ? std::fabs(hs.phibar) / hs.bnorm : 0.0;
  res->true_relres = fin.bnorm > 0.0 ? fin.beta / fin.bnorm : 0.0;
  res->converged = hs.done == 1 ? 1 : 0;
}
