// solve.cu -- steps A8-A11: supernodal forward and backward solves with the multifrontal factor, the
// quadratic form, the log-determinant, FP64 iterative refinement (mixed precision) and the log-likelihood
//   log p(z | beta, theta) = -1/2 log det C_z - 1/2 r^T C_z^{-1} r - n/2 log(2 pi)      (Sec. 3.3)
// with log det C_z = 2 sum_j log L_jj.
//
// Forward (levels ascending): the front vector of supernode s (m entries, own columns then the rows below)
// starts as the permuted right-hand side on its columns, receives every child's update vector through the
// child's relative indices (children in order), then x = L11^{-1} f_1 and f_2 -= L21 x; f_2 is the update
// vector handed to the parent. Backward (levels descending): t = x - L21^T alpha'(rows below), then
// L11^T z = t. Fronts of order <= 96 use one CTA; larger ones advance 64 columns per launch, every CTA
// multiplying by the inverted 64 x 64 diagonal block (formed by the factorization) and applying the result
// to its own 64-row (or 64-column) tile.
// The kernels read the factor through an accessor: FP64 column-major panels (GP_FP64) or FP32 row-major
// panels with FP64 diagonal tiles (GP_MIXED). In GP_FP64 the solves run in FP64 and the quadratic form is
// |L^{-1} P r|^2. In GP_MIXED the solves run in FP32 (FP32 inverses, FP32 vectors): they only precondition
// the FP64 refinement of alpha (residual r - C alpha from the FP64 CSR values, correction through the same
// factor) until |r - C alpha| / |r| <= 1e-12 or 10 sweeps; the quadratic form is r^T alpha in FP64 and the
// log-determinant is summed in FP64 from the FP64 diagonal tiles.
// Sums use fixed-shape trees, so results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <vector>

#include "factor_access.cuh"
#include "gp_internal.cuh"

namespace {

constexpr int T = GP_TILE;
using fa::AccF64;
using fa::AccMix;
using fa::StoreF64;
using fa::StoreMix;
using fa::find_front;

template <class V>
__global__ void k_rhs(const double* __restrict__ rhs, const int32_t* __restrict__ perm, int64_t n, DevPlan dp,
                      V* __restrict__ work, int64_t ws) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (j >= n) return;
  int32_t s = dp.sn_of_col[j];
  work[(int64_t)b * ws + dp.frow_off[s] + (j - dp.sn_first[s])] = (V)rhs[(int64_t)b * n + perm[j]];
}

// Children's update vectors into the front vector of each supernode of the list.
template <class V>
__global__ void k_fwd_gather(const int32_t* __restrict__ list, DevPlan dp, V* __restrict__ work, int64_t ws) {
  int32_t s = list[blockIdx.x];
  V* W = work + (int64_t)blockIdx.y * ws;
  V* fv = W + dp.frow_off[s];
  for (int32_t q = dp.ch_ptr[s]; q < dp.ch_ptr[s + 1]; q++) {
    int32_t c = dp.ch_idx[q];
    const V* uc = W + dp.frow_off[c] + dp.w[c];
    const int32_t* rel = dp.relidx + dp.relidx_off[c];
    for (int32_t a = threadIdx.x; a < dp.r[c]; a += blockDim.x) fv[rel[a]] += uc[a];
    __syncthreads();
  }
}

// Forward elimination of a whole (small) front by one CTA.
template <class St>
__global__ void k_fwd_small(const int32_t* __restrict__ list, DevPlan dp, St store, typename St::V* __restrict__ work,
                            int64_t ws, int64_t xv_off) {
  using V = typename St::V;
  __shared__ V xs;
  __shared__ V rdg[GP_SMALL_M];   // 1 / L_jj, formed in parallel ahead of the substitution
  int32_t s = list[blockIdx.x];
  int b = blockIdx.y;
  auto A = store.acc(dp, s, b);
  V* fv = work + (int64_t)b * ws + dp.frow_off[s];
  V* xv = work + (int64_t)b * ws + xv_off + dp.sn_first[s];
  const int w = dp.w[s];
  const int64_t m = (int64_t)w + dp.r[s];
  for (int j = threadIdx.x; j < w; j += blockDim.x) rdg[j] = V(1) / A.L(j, j);
  __syncthreads();
  for (int j = 0; j < w; j++) {
    if (threadIdx.x == 0) {
      xs = fv[j] * rdg[j];
      fv[j] = xs;
      xv[j] = xs;
    }
    __syncthreads();
    V x = xs;
    for (int64_t i = j + 1 + threadIdx.x; i < m; i += blockDim.x) fv[i] -= A.L(i, j) * x;
    __syncthreads();
  }
}

// The pieces of a forward step, shared by the single and the paired launches.
// x = inv(L_JJ) f_J for a block of width bw: inv is the block's 64 x 64 inverse, fb (shared) holds f_J; the
// product is split four ways over l and combined in a fixed order.
template <class V>
__device__ __forceinline__ void fwd_block_solve(const V* __restrict__ inv, const V* fb, V* x, V* LiT, V (*part)[T],
                                                int bw) {
#pragma unroll
  for (int u = 0; u < T * T / 256; u++) {
    const int q = threadIdx.x + u * 256;
    LiT[(q & 63) * (T + 1) + (q >> 6)] = inv[q];
  }
  __syncthreads();
  {   // the inverse is lower triangular with zeros above (and past bw), so every l enters
    const int g = threadIdx.x >> 6, q = threadIdx.x & 63;
    V acc = 0;
#pragma unroll
    for (int l = g * 16; l < g * 16 + 16; l++) acc += LiT[l * (T + 1) + q] * fb[l];
    part[g][q] = acc;
  }
  __syncthreads();
  if (threadIdx.x < T) {
    const int q = threadIdx.x;
    x[q] = q < bw ? (part[0][q] + part[1][q]) + (part[2][q] + part[3][q]) : V(0);
  }
  __syncthreads();
}

// acc_i = L[i, c0 .. c0 + bw) x for the rows [r0, rend) (at most 64), handed to sink(i, acc) by one thread per
// row. Row-major panels: a half-warp reads one row's 64 entries as 16 float4, four rows per half-warp with all
// loads in flight, a fixed shuffle tree per row; column-major: thread per row.
template <class St, class Sink>
__device__ __forceinline__ void fwd_rows(const typename St::Acc& A, int64_t r0, int64_t rend, int c0, int bw,
                                         const typename St::V* x, Sink&& sink) {
  using V = typename St::V;
  if constexpr (St::kRowMajor) {
    // columns past bw are zero in x and the row is padded to ldw (a multiple of 4): whole float4 reads are safe
    const int hw = threadIdx.x >> 4, l = (threadIdx.x & 15) * 4;
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int64_t i = r0 + hw + 16 * u;
      v[u] = (i < rend && l < bw) ? *reinterpret_cast<const float4*>(A.P + i * A.ldw + c0 + l)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      V acc = (V)v[u].x * x[l] + (V)v[u].y * x[l + 1] + (V)v[u].z * x[l + 2] + (V)v[u].w * x[l + 3];
      for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const int64_t i = r0 + hw + 16 * u;
      if (i < rend && (threadIdx.x & 15) == 0) sink(i, acc);
    }
  } else {
    for (int64_t i = r0 + threadIdx.x; i < rend; i += blockDim.x) {
      V acc = 0;
      for (int l = 0; l < bw; l++) acc += A.L(i, c0 + l) * x[l];
      sink(i, acc);
    }
  }
}

// Forward, block column kb of every large front of a step, one launch: every CTA forms x_J = inv(L_JJ) f_J
// (a 64 x 64 product with the inverted diagonal block); tasks [0, nfront) write x_J to x (the front vector's
// block stays untouched, others read it), the rest (64-row tile prefix) apply f_i -= L[i, J] x_J to one tile.
template <class St>
__global__ void __launch_bounds__(256) k_fwd_step(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre,
                                                  int nfront, int kb, DevPlan dp, St store,
                                                  typename St::V* __restrict__ work, int64_t ws, int64_t xv_off) {
  using V = typename St::V;
  __shared__ V LiT[T * (T + 1)];   // LiT[l][q] = inv[q][l]
  __shared__ V fb[T], x[T], part[4][T];
  const int64_t t = blockIdx.x;
  const bool writer = t < nfront;
  const int fi = writer ? (int)t : find_front(pre, nfront, t - nfront);
  const int32_t s = fronts[fi];
  const int b = blockIdx.y;
  auto A = store.acc(dp, s, b);
  V* fv = work + (int64_t)b * ws + dp.frow_off[s];
  const int w = dp.w[s];
  const int64_t m = (int64_t)w + dp.r[s];
  const int c0 = kb * T, bw = min(T, w - c0), c1 = c0 + bw;
  if (threadIdx.x < T) fb[threadIdx.x] = threadIdx.x < bw ? fv[c0 + threadIdx.x] : V(0);
  fwd_block_solve(store.inv(dp, s, b) + (int64_t)kb * T * T, fb, x, LiT, part, bw);
  if (writer) {
    V* xv = work + (int64_t)b * ws + xv_off + dp.sn_first[s];
    if (threadIdx.x < bw) xv[c0 + threadIdx.x] = x[threadIdx.x];
    return;
  }
  const int64_t r0 = c1 + (t - nfront - pre[fi]) * T, rend = imin64(r0 + T, m);
  fwd_rows<St>(A, r0, rend, c0, bw, x, [&](int64_t i, V acc) { fv[i] -= acc; });
}

// Forward, block columns kb and kb + 1 in one launch (the chain of forward steps is the sweep's latency). The
// fronts [0, n2) of the list have block kb + 1: every CTA forms x1 = inv(L_11) f_1, f_2' = f_2 - L_21 x1 and
// x2 = inv(L_22) f_2' itself (the same operations, in the same order, as two single steps), then a writer
// stores x1, x2 and a tile task applies f_i -= L_i1 x1, then f_i -= L_i2 x2 to 64 rows after block kb + 1.
// Fronts past n2 take block kb alone, as a single step.
template <class St>
__global__ void __launch_bounds__(256) k_fwd_pair(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre,
                                                  int nfront, int n2, int kb, DevPlan dp, St store,
                                                  typename St::V* __restrict__ work, int64_t ws, int64_t xv_off) {
  using V = typename St::V;
  __shared__ V LiT[T * (T + 1)];   // LiT[l][q] = inv[q][l]
  __shared__ V fb[T], x1[T], x2[T], part[4][T], a1[T], a2[T];
  const int64_t t = blockIdx.x;
  const bool writer = t < nfront;
  const int fi = writer ? (int)t : find_front(pre, nfront, t - nfront);
  const int32_t s = fronts[fi];
  const int b = blockIdx.y;
  auto A = store.acc(dp, s, b);
  V* fv = work + (int64_t)b * ws + dp.frow_off[s];
  const int w = dp.w[s];
  const int64_t m = (int64_t)w + dp.r[s];
  const bool two = fi < n2;
  const int c0 = kb * T, bw1 = min(T, w - c0), c1 = c0 + bw1;
  const int bw2 = two ? min(T, w - c1) : 0, c2 = c1 + bw2;
  const V* inv = store.inv(dp, s, b) + (int64_t)kb * T * T;
  if (threadIdx.x < T) fb[threadIdx.x] = threadIdx.x < bw1 ? fv[c0 + threadIdx.x] : V(0);
  fwd_block_solve(inv, fb, x1, LiT, part, bw1);
  if (two) {
    fwd_rows<St>(A, c1, c2, c0, bw1, x1, [&](int64_t i, V acc) { a1[i - c1] = acc; });
    __syncthreads();
    if (threadIdx.x < T) fb[threadIdx.x] = threadIdx.x < bw2 ? fv[c1 + threadIdx.x] - a1[threadIdx.x] : V(0);
    fwd_block_solve(inv + T * T, fb, x2, LiT, part, bw2);
  }
  if (writer) {
    V* xv = work + (int64_t)b * ws + xv_off + dp.sn_first[s];
    if (threadIdx.x < bw1) xv[c0 + threadIdx.x] = x1[threadIdx.x];
    if (threadIdx.x < bw2) xv[c1 + threadIdx.x] = x2[threadIdx.x];
    return;
  }
  const int64_t r0 = c2 + (t - nfront - pre[fi]) * T, rend = imin64(r0 + T, m);
  fwd_rows<St>(A, r0, rend, c0, bw1, x1, [&](int64_t i, V acc) { a1[i - r0] = acc; });
  if (two) fwd_rows<St>(A, r0, rend, c1, bw2, x2, [&](int64_t i, V acc) { a2[i - r0] = acc; });
  __syncthreads();
  if (threadIdx.x < T && r0 + threadIdx.x < rend) {
    V v = fv[r0 + threadIdx.x];
    v -= a1[threadIdx.x];
    if (two) v -= a2[threadIdx.x];
    fv[r0 + threadIdx.x] = v;
  }
}

// Backward, small fronts (one CTA each): t_j = x_j - sum_{a < r} L[w + a, j] alpha'(R_s[a]) (warp per
// column), then L11^T z = t by substitution; z is written to alpha'.
template <class St>
__global__ void k_bwd_prep(const int32_t* __restrict__ list, int solve_small, DevPlan dp, St store,
                           typename St::V* __restrict__ work, int64_t ws, int64_t apv_off, int64_t xv_off) {
  using V = typename St::V;
  __shared__ V zs;
  __shared__ V rdg[GP_SMALL_M];
  int32_t s = list[blockIdx.x];
  int b = blockIdx.y;
  auto A = store.acc(dp, s, b);
  V* W = work + (int64_t)b * ws;
  V* fv = W + dp.frow_off[s];
  V* apv = W + apv_off;
  const int w = dp.w[s], r = dp.r[s];
  const int32_t* R = dp.frows + dp.frow_off[s] + w;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < w; j += nw) {
    V acc = 0;
    for (int a = lane; a < r; a += 32) acc += A.L(w + a, j) * apv[R[a]];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) fv[j] = W[xv_off + dp.sn_first[s] + j] - acc;
  }
  if (!solve_small) return;
  for (int j = threadIdx.x; j < w; j += blockDim.x) rdg[j] = V(1) / A.L(j, j);
  __syncthreads();
  const int32_t first = dp.sn_first[s];
  for (int j = w - 1; j >= 0; j--) {
    if (threadIdx.x == 0) {
      zs = fv[j] * rdg[j];
      fv[j] = zs;
      apv[first + j] = zs;
    }
    __syncthreads();
    V z = zs;
    for (int k = threadIdx.x; k < j; k += blockDim.x) fv[k] -= A.L(j, k) * z;
    __syncthreads();
  }
}

// Backward, large fronts: t_j = x_j - sum_a L[w + a, j] alpha'(R_s[a]) for the 64-column stripe of each task
// (a task per (front, stripe) over all of a level's large fronts), in two launches: partial sums over chunks of
// BP_CH rows (grid: task x chunk), then a fixed-order sum of the chunks per task.
// Row-major: 64 threads across the stripe's columns x 4 row groups, eight loads in flight per thread;
// column-major: a warp per column.
constexpr int BP_CH = 128;

template <class St>
__global__ void __launch_bounds__(256) k_bwd_prep_part(const int32_t* __restrict__ fronts,
                                                       const int32_t* __restrict__ kbs, int ntask, int nch,
                                                       DevPlan dp, St store, const typename St::V* __restrict__ work,
                                                       int64_t ws, int64_t apv_off, typename St::V* __restrict__ part) {
  using V = typename St::V;
  __shared__ V ps[4][T];
  const int task = blockIdx.x, chunk = blockIdx.y, b = blockIdx.z;
  const int32_t s = fronts[task];
  const int j0 = kbs[task] * T;
  const int w = dp.w[s], r = dp.r[s];
  const int a0 = chunk * BP_CH;
  if (a0 >= r) return;
  const int a1 = min(r, a0 + BP_CH);
  auto A = store.acc(dp, s, b);
  const V* apv = work + (int64_t)b * ws + apv_off;
  const int nj = min(T, w - j0);
  const int32_t* R = dp.frows + dp.frow_off[s] + w;
  V* out = part + (((int64_t)b * ntask + task) * nch + chunk) * T;
  if constexpr (St::kRowMajor) {
    const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
    V acc = 0;
    if (c < nj) {
      for (int a = a0 + g; a < a1; a += 32) {
        V lv[8], av[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
          const int aa = a + 4 * e;
          lv[e] = aa < a1 ? (V)A.P[(int64_t)(w + aa) * A.ldw + j0 + c] : V(0);
          av[e] = aa < a1 ? apv[R[aa]] : V(0);
        }
#pragma unroll
        for (int e = 0; e < 8; e++) acc += lv[e] * av[e];
      }
    }
    ps[g][c] = acc;
    __syncthreads();
    if (g == 0) out[c] = ((ps[0][c] + ps[1][c]) + ps[2][c]) + ps[3][c];
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int jj = warp; jj < T; jj += nw) {
      V acc = 0;
      if (jj < nj)
        for (int a = a0 + lane; a < a1; a += 32) acc += A.L(w + a, j0 + jj) * apv[R[a]];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) out[jj] = acc;
    }
  }
}

template <class V>
__global__ void k_bwd_prep_sum(const int32_t* __restrict__ fronts, const int32_t* __restrict__ kbs, int ntask,
                               int nch, DevPlan dp, V* __restrict__ work, int64_t ws, int64_t xv_off,
                               const V* __restrict__ part) {
  const int task = blockIdx.x, b = blockIdx.y, c = threadIdx.x;
  const int32_t s = fronts[task];
  const int j0 = kbs[task] * T;
  const int nj = min(T, dp.w[s] - j0);
  if (c >= nj) return;
  const int nc = (dp.r[s] + BP_CH - 1) / BP_CH;
  const V* p = part + ((int64_t)b * ntask + task) * nch * T + c;
  V acc = 0;
  for (int k = 0; k < nc; k++) acc += p[(int64_t)k * T];
  V* W = work + (int64_t)b * ws;
  W[dp.frow_off[s] + j0 + c] = W[xv_off + dp.sn_first[s] + j0 + c] - acc;
}

// The pieces of a backward step, shared by the single and the paired launches.
// z = inv(L_JJ)^T t_J for a block of width bw: inv is the block's 64 x 64 inverse (row-major into Li), tb
// (shared) holds t_J; z_q = sum_{l >= q} inv[l][q] t_l (zeros above the diagonal and past bw), split four ways
// over l and combined in a fixed order.
template <class V>
__device__ __forceinline__ void bwd_block_solve(const V* __restrict__ inv, const V* tb, V* z, V* Li, V (*part)[T],
                                                int bw) {
#pragma unroll
  for (int u = 0; u < T * T / 256; u++) {
    const int q = threadIdx.x + u * 256;
    Li[(q >> 6) * (T + 1) + (q & 63)] = inv[q];
  }
  __syncthreads();
  const int g = threadIdx.x >> 6, q = threadIdx.x & 63;
  {
    V acc = 0;
#pragma unroll
    for (int l = g * 16; l < g * 16 + 16; l++) acc += Li[l * (T + 1) + q] * tb[l];
    part[g][q] = acc;
  }
  __syncthreads();
  if (threadIdx.x < T) {
    const int k = threadIdx.x;
    z[k] = k < bw ? (part[0][k] + part[1][k]) + (part[2][k] + part[3][k]) : V(0);
  }
  __syncthreads();
}

// sum_k = sum_l L[r0 + l, k0 + k] z_l over the bw rows of a block (k < 64; returned to threads k < 64), split
// four ways over l (16 independent loads per thread in flight) and combined in a fixed order.
template <class St>
__device__ __forceinline__ typename St::V bwd_tile_sum(const typename St::Acc& A, int r0, int bw, int k0,
                                                       const typename St::V* z, typename St::V (*part)[T]) {
  using V = typename St::V;
  const int g = threadIdx.x >> 6, q = threadIdx.x & 63;
  V acc = 0;
  if constexpr (St::kRowMajor) {   // row r0 + l is contiguous over the tile's columns
    V v[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
      const int l = g * 16 + e;
      v[e] = l < bw ? (V)A.P[(int64_t)(r0 + l) * A.ldw + k0 + q] : V(0);
    }
#pragma unroll
    for (int e = 0; e < 16; e++) acc += v[e] * z[g * 16 + e];
  } else {
    for (int e = 0; e < 16; e++) {
      const int l = g * 16 + e;
      if (l < bw) acc += A.L(r0 + l, k0 + q) * z[l];
    }
  }
  __syncthreads();   // part is reused
  part[g][q] = acc;
  __syncthreads();
  V sum = 0;
  if (threadIdx.x < T) {
    const int k = threadIdx.x;
    sum = (part[0][k] + part[1][k]) + (part[2][k] + part[3][k]);
  }
  return sum;
}

// Backward, block column kb of every large front of a step, one launch: every CTA forms
// z_J = inv(L_JJ)^T t_J; task 0 of a front writes z_J to alpha', tasks 1..kb apply t_k -= L[J, k]^T z_J to
// one 64-column tile of the earlier columns k < c0.
template <class St>
__global__ void __launch_bounds__(256) k_bwd_step(const int32_t* __restrict__ fronts, int nfront, int kb, DevPlan dp,
                                                  St store, typename St::V* __restrict__ work, int64_t ws,
                                                  int64_t apv_off) {
  using V = typename St::V;
  __shared__ V Li[T * (T + 1)];   // the inverse block (row-major)
  __shared__ V tb[T], z[T], part[4][T];
  const int64_t t = blockIdx.x;
  const int fi = (int)(t / (kb + 1));
  const int task = (int)(t % (kb + 1));
  const int32_t s = fronts[fi];
  const int b = blockIdx.y;
  auto A = store.acc(dp, s, b);
  V* W = work + (int64_t)b * ws;
  V* fv = W + dp.frow_off[s];
  const int w = dp.w[s];
  const int c0 = kb * T, bw = min(T, w - c0);
  if (threadIdx.x < T) tb[threadIdx.x] = threadIdx.x < bw ? fv[c0 + threadIdx.x] : V(0);
  bwd_block_solve(store.inv(dp, s, b) + (int64_t)kb * T * T, tb, z, Li, part, bw);
  if (task == 0) {
    V* apv = W + apv_off;
    if (threadIdx.x < bw) apv[dp.sn_first[s] + c0 + threadIdx.x] = z[threadIdx.x];
    return;
  }
  const int k0 = (task - 1) * T;   // columns [k0, k0 + 64) < c0
  const V sum = bwd_tile_sum<St>(A, c0, bw, k0, z, part);
  if (threadIdx.x < T) fv[k0 + threadIdx.x] -= sum;
}

// Backward, block columns kb + 1 and kb in one launch (the chain of backward steps is the sweep's latency). The
// fronts [0, n2) of step kb's list have block kb + 1: every CTA forms z2 = inv(L_22)^T t_2,
// t_1' = t_1 - L_21^T z2 and z1 = inv(L_11)^T t_1' itself (the same operations, in the same order, as two
// single steps); task 0 writes z1, z2 to alpha', tasks 1..kb apply t_k -= L[2, k]^T z2, then t_k -= L[1, k]^T z1
// to one 64-column tile k < c0. Fronts past n2 take block kb alone, as a single step.
template <class St>
__global__ void __launch_bounds__(256) k_bwd_pair(const int32_t* __restrict__ fronts, int nfront, int n2, int kb,
                                                  DevPlan dp, St store, typename St::V* __restrict__ work,
                                                  int64_t ws, int64_t apv_off) {
  using V = typename St::V;
  __shared__ V Li[T * (T + 1)];
  __shared__ V tb[T], z1[T], z2[T], part[4][T];
  const int64_t t = blockIdx.x;
  const int fi = (int)(t / (kb + 1));
  const int task = (int)(t % (kb + 1));
  const int32_t s = fronts[fi];
  const int b = blockIdx.y;
  auto A = store.acc(dp, s, b);
  V* W = work + (int64_t)b * ws;
  V* fv = W + dp.frow_off[s];
  const int w = dp.w[s];
  const bool two = fi < n2;
  const int c0 = kb * T, bw1 = min(T, w - c0), c1 = c0 + bw1;
  const int bw2 = two ? min(T, w - c1) : 0;
  const V* inv = store.inv(dp, s, b) + (int64_t)kb * T * T;
  V t1 = 0;
  if (two) {
    if (threadIdx.x < T) tb[threadIdx.x] = threadIdx.x < bw2 ? fv[c1 + threadIdx.x] : V(0);
    bwd_block_solve(inv + T * T, tb, z2, Li, part, bw2);
    const V sum = bwd_tile_sum<St>(A, c1, bw2, c0, z2, part);   // block kb's columns
    if (threadIdx.x < T) t1 = fv[c0 + threadIdx.x] - sum;
  } else if (threadIdx.x < T) {
    t1 = fv[c0 + threadIdx.x];
  }
  if (threadIdx.x < T) tb[threadIdx.x] = threadIdx.x < bw1 ? t1 : V(0);
  bwd_block_solve(inv, tb, z1, Li, part, bw1);
  if (task == 0) {
    V* apv = W + apv_off + dp.sn_first[s];
    if (threadIdx.x < bw1) apv[c0 + threadIdx.x] = z1[threadIdx.x];
    if (threadIdx.x < bw2) apv[c1 + threadIdx.x] = z2[threadIdx.x];
    return;
  }
  const int k0 = (task - 1) * T;
  V v = 0;
  if (threadIdx.x < T) v = fv[k0 + threadIdx.x];
  if (two) {
    const V sum2 = bwd_tile_sum<St>(A, c1, bw2, k0, z2, part);
    v -= sum2;
  }
  const V sum1 = bwd_tile_sum<St>(A, c0, bw1, k0, z1, part);
  v -= sum1;
  if (threadIdx.x < T) fv[k0 + threadIdx.x] = v;
}

// Per-block partial sums: log L_jj and x_j^2 (x = forward solution on own columns).
template <class St>
__global__ void k_partials(int64_t n, DevPlan dp, St store, const typename St::V* __restrict__ work, int64_t ws,
                           int64_t xv_off, double* __restrict__ red, int64_t rs, int nblk) {
  __shared__ double sa[1024], sb[1024];
  int b = blockIdx.y;
  int64_t j = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  double la = 0.0, lb = 0.0;
  if (j < n) {
    int32_t s = dp.sn_of_col[j];
    int64_t jl = j - dp.sn_first[s];
    auto A = store.acc(dp, s, b);
    la = log(A.Ld(jl, jl));
    double x = (double)work[(int64_t)b * ws + xv_off + j];
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

// Fixed-order sum of nblk partials (two series a, b) per proposal.
__global__ void k_sum2(const double* __restrict__ red, int64_t rs, int nblk, double* __restrict__ out) {
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
    out[2 * b] = ta;
    out[2 * b + 1] = tb;
  }
}

__global__ void k_finish(int B, int64_t n, const double* __restrict__ s_logdet, const double* __restrict__ s_quad,
                         const int32_t* __restrict__ notpd, const int32_t* __restrict__ tc_err,
                         double* __restrict__ out) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double logdet = 2.0 * s_logdet[2 * b];
  double quad = s_quad[2 * b + 1];
  double ll = -0.5 * logdet - 0.5 * quad - 0.5 * (double)n * log(2.0 * 3.14159265358979323846);
  if (notpd[b] != 0x7fffffff) ll = -INFINITY;
  if (tc_err && *tc_err) ll = NAN;
  out[b] = ll;
}

template <class V>
__global__ void k_alpha(const V* __restrict__ work, int64_t ws, int64_t apv_off, const int32_t* __restrict__ perm,
                        int64_t n, double* __restrict__ alpha) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (j < n) alpha[(int64_t)b * n + perm[j]] = (double)work[(int64_t)b * ws + apv_off + j];
}

// res = r - C alpha (warp per CSR row, fixed lane order) and per-block sums of res^2, r^2 and r . alpha.
__global__ void k_residual(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n,
                           int64_t nnz, const double* __restrict__ val, const double* __restrict__ alpha,
                           const double* __restrict__ resid, double* __restrict__ res, double* __restrict__ red,
                           int64_t rs, int nblk) {
  __shared__ double s1[8], s2[8], s3[8];
  int b = blockIdx.y;
  int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  const double* a = alpha + (int64_t)b * n;
  if (i < n) {
    const double* v = val + (int64_t)b * nnz;
    for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) acc += v[e] * a[col[e]];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  double rr = 0.0, ri = 0.0, ra = 0.0;
  if (i < n && lane == 0) {
    ri = resid[(int64_t)b * n + i];
    rr = ri - acc;
    ra = ri * a[i];
    if (res) res[(int64_t)b * n + i] = rr;
  }
  if (lane == 0) {
    s1[warp] = rr * rr;
    s2[warp] = ri * ri;
    s3[warp] = ra;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int q = 0; q < 8; q++) {
      a1 += s1[q];
      a2 += s2[q];
      a3 += s3[q];
    }
    red[(int64_t)b * rs + blockIdx.x] = a1;
    red[(int64_t)b * rs + nblk + blockIdx.x] = a2;
    red[(int64_t)b * rs + 2 * nblk + blockIdx.x] = a3;
  }
}

// Fixed-order reduction of the residual partials: err[b] = |res| / |r|, rdot[b] = r . alpha. Thread t sums
// partials t, t + 1024, ... in order (three independent chains), then one tree over the 1024 threads.
constexpr int RELRES_THREADS = 1024;
__global__ void __launch_bounds__(RELRES_THREADS) k_relres(const double* __restrict__ red, int64_t rs, int nblk,
                                                           double* __restrict__ err, double* __restrict__ rdot) {
  __shared__ double sa[RELRES_THREADS], sb[RELRES_THREADS], sc[RELRES_THREADS];
  const int b = blockIdx.x, t = threadIdx.x;
  const double* ra = red + (int64_t)b * rs;
  double ta = 0.0, tb = 0.0, tc = 0.0;
  for (int i = t; i < nblk; i += RELRES_THREADS) {
    ta += ra[i];
    tb += ra[nblk + i];
    tc += ra[2 * (int64_t)nblk + i];
  }
  sa[t] = ta;
  sb[t] = tb;
  sc[t] = tc;
  __syncthreads();
  for (int o = RELRES_THREADS / 2; o > 0; o >>= 1) {
    if (t < o) {
      sa[t] += sa[t + o];
      sb[t] += sb[t + o];
      sc[t] += sc[t + o];
    }
    __syncthreads();
  }
  if (t == 0) {
    if (err) err[b] = sb[0] > 0.0 ? sqrt(sa[0] / sb[0]) : sqrt(sa[0]);
    if (rdot) rdot[2 * b + 1] = sc[0];
  }
}

// The refinement loop's test on the device: continue while some proposal's |r - C alpha| / |r| exceeds 1e-12 (or
// is not finite) and fewer than 10 corrections have run. it[0] counts the corrections; a factorization whose
// bounded waits ran out (tc_err) stops the loop at once (its outputs become NaN).
__global__ void k_refine_test(const double* __restrict__ err, int B, int32_t* __restrict__ it,
                              unsigned long long* __restrict__ runs, const int32_t* __restrict__ tc_err, int reset,
                              cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  if (reset) it[0] = 0;
  double worst = 0.0;
  for (int b = 0; b < B; b++) worst = fmax(worst, isfinite(err[b]) ? err[b] : 1.0);
  const bool more = worst > 1e-12 && it[0] < 10 && !(tc_err && *tc_err);
  if (more) {
    it[0] += 1;
    runs[0] += 1;   // corrections run by the loop over the factor's life (launch accounting)
  }
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, int64_t cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) y[i] += x[i];
}

// Row chunks of the widest front among level L's large-front tasks (the backward partial-sum grid).
int bwd_chunks(const SymPlan& sp, int32_t L) {
  const auto& ll = sp.level_large[L];
  int nch = 1;
  for (int64_t q = 0; q < ll.count; q++) {
    const int32_t s = sp.large_fronts[ll.off + q];
    nch = std::max(nch, (int)((sp.sn_r[s] + BP_CH - 1) / BP_CH));
  }
  return nch;
}

template <class St>
void solve_impl(gp_ctx* ctx, gp_factor_t* f, const St& store, const double* rhs, double* alpha_out, bool partials) {
  gp_pointset* ps = f->ps;
  const SymPlan& sp = ps->sp;
  const DevPlan& dp = ps->dp;
  cudaStream_t st = ctx->stream;
  const int B = f->B;
  const int64_t n = ps->n, ws = f->work_stride;
  const int64_t apv_off = sp.sn_frow[sp.ns];   // work layout: front vectors, alpha' (n), x (n)
  const int64_t xv_off = apv_off + n;
  using V = typename St::V;
  V* work = reinterpret_cast<V*>(f->work);   // ws entries of V per proposal
  GP_CUDA(cudaMemsetAsync(f->work, 0, sizeof(V) * (size_t)B * ws, st));
  k_rhs<<<dim3(grid_for(n, 256), B), 256, 0, st>>>(rhs, ps->perm, n, dp, work, ws);
  GP_CHECK_LAUNCH(ctx);
  for (int32_t L = 0; L < sp.nlevels; L++) {
    const SymPlan::Level& lv = sp.levels[L];
    int32_t nl = sp.lev_ptr[L + 1] - sp.lev_ptr[L];
    if (L > 0) {
      k_fwd_gather<<<dim3(nl, B), 256, 0, st>>>(dp.lev_sn + sp.lev_ptr[L], dp, work, ws);
      GP_CHECK_LAUNCH(ctx);
    }
    if (lv.nsmall > 0) {
      k_fwd_small<St><<<dim3(lv.nsmall, B), 128, 0, st>>>(dp.small_list + lv.small_off, dp, store, work, ws,
                                                          xv_off);
      GP_CHECK_LAUNCH(ctx);
    }
    for (size_t q = 0; q < lv.steps.size();) {
      const auto& stp = lv.steps[q];
      if (q + 1 < lv.steps.size()) {   // block columns kb and kb + 1 together
        k_fwd_pair<St><<<dim3((unsigned)(stp.nfront + stp.pair_total), B), 256, 0, st>>>(
            dp.large_fronts + stp.fr_off, dp.pair_pre + stp.pair_pre_off, stp.nfront, stp.pair_n2, stp.kb, dp, store,
            work, ws, xv_off);
        q += 2;
      } else {
        k_fwd_step<St><<<dim3((unsigned)(stp.nfront + stp.trsm_total), B), 256, 0, st>>>(
            dp.large_fronts + stp.fr_off, dp.step_pre + stp.pre_off, stp.nfront, stp.kb, dp, store, work, ws,
            xv_off);
        q += 1;
      }
      GP_CHECK_LAUNCH(ctx);
    }
  }
  if (partials) {
    int nblk = (int)((n + 1023) / 1024);
    k_partials<St><<<dim3(nblk, B), 1024, 0, st>>>(n, dp, store, work, ws, xv_off, f->red, f->red_stride, nblk);
    GP_CHECK_LAUNCH(ctx);
  }
  for (int32_t L = sp.nlevels - 1; L >= 0; L--) {
    const SymPlan::Level& lv = sp.levels[L];
    if (lv.nsmall > 0) {
      k_bwd_prep<St><<<dim3(lv.nsmall, B), 256, 0, st>>>(dp.small_list + lv.small_off, 1, dp, store, work, ws,
                                                         apv_off, xv_off);
      GP_CHECK_LAUNCH(ctx);
    }
    if (!lv.steps.empty()) {
      const auto& ll = sp.level_large[L];   // one task per (large front, 64-column stripe)
      const int nch = bwd_chunks(sp, L);
      V* part = reinterpret_cast<V*>(f->bwd_part);
      k_bwd_prep_part<St><<<dim3((unsigned)ll.count, nch, B), 256, 0, st>>>(
          dp.large_fronts + ll.off, dp.large_kb + ll.off, (int)ll.count, nch, dp, store, work, ws, apv_off, part);
      GP_CHECK_LAUNCH(ctx);
      k_bwd_prep_sum<V><<<dim3((unsigned)ll.count, B), T, 0, st>>>(dp.large_fronts + ll.off, dp.large_kb + ll.off,
                                                                   (int)ll.count, nch, dp, work, ws, xv_off, part);
      GP_CHECK_LAUNCH(ctx);
      for (int q = (int)lv.steps.size() - 1; q >= 0;) {
        if (q >= 1) {   // block columns kb + 1 = q and kb = q - 1 together
          const auto& stp = lv.steps[q - 1];
          k_bwd_pair<St><<<dim3((unsigned)((int64_t)stp.nfront * (stp.kb + 1)), B), 256, 0, st>>>(
              dp.large_fronts + stp.fr_off, stp.nfront, lv.steps[q].nfront, stp.kb, dp, store, work, ws, apv_off);
          q -= 2;
        } else {
          const auto& stp = lv.steps[q];
          k_bwd_step<St><<<dim3((unsigned)((int64_t)stp.nfront * (stp.kb + 1)), B), 256, 0, st>>>(
              dp.large_fronts + stp.fr_off, stp.nfront, stp.kb, dp, store, work, ws, apv_off);
          q -= 1;
        }
        GP_CHECK_LAUNCH(ctx);
      }
    }
  }
  k_alpha<<<dim3(grid_for(n, 256), B), 256, 0, st>>>(work, ws, apv_off, ps->perm, n, alpha_out);
  GP_CHECK_LAUNCH(ctx);
}

// Residual of alpha for right-hand sides rhs: res (nullable) = rhs - C alpha; err[b] = |res|/|rhs|;
// rdot[2b+1] = rhs . alpha. Partials go to the workspace (free once alpha has been extracted).
void residual_impl(gp_ctx* ctx, gp_factor_t* f, const double* rhs, const double* alpha, double* res, double* err,
                   double* rdot) {
  gp_pointset* ps = f->ps;
  const int64_t n = ps->n;
  int nblk = (int)((n + 7) / 8);
  GP_REQUIRE(3 * (int64_t)nblk + 2 <= f->work_stride, "residual partials exceed the workspace");
  k_residual<<<dim3(nblk, f->B), 256, 0, ctx->stream>>>(ps->rowptr, ps->col, n, ps->nnz, f->val, alpha, rhs, res,
                                                        f->work, f->work_stride, nblk);
  GP_CHECK_LAUNCH(ctx);
  k_relres<<<f->B, RELRES_THREADS, 0, ctx->stream>>>(f->work, f->work_stride, nblk, err, rdot);
  GP_CHECK_LAUNCH(ctx);
}

}  // namespace

// Run `body` directly, or through a CUDA graph captured on first use (the launch sequence depends only on
// the plan; every pointer it uses belongs to the factor).
template <class F>
static void run_maybe_graph(gp_ctx* ctx, cudaGraphExec_t* gx, int64_t* nl, F&& body) {
  if (!use_graphs(ctx)) {
    body();
    return;
  }
  if (!*gx) *gx = capture_graph(ctx, body, nl);
  replay_graph(ctx, *gx, *nl);
}

// The mixed path's refinement (A11) as one executable graph, so that gp_loglik neither waits for the device nor
// reads back a residual: [residual, test] then a conditional WHILE node whose body is [correction solve, alpha +=
// correction, residual, test], then [final residual with r . alpha, log-likelihood]. The test kernel sets the loop's
// condition (cudaGraphSetConditional). The output pointers are baked into the graph, so it is rebuilt when they
// change. *nl receives the launches of one pass (the body counted once).
template <class St>
static cudaGraphExec_t build_refine_graph(gp_ctx* ctx, gp_factor_t* f, const St& store, double* res, double* cor,
                                          double* errv, double* s_log, double* s_quad, double* d_out, double* d_err,
                                          int64_t* nl) {
  const int B = f->B;
  const int64_t n = f->ps->n;
  cudaStream_t st = ctx->stream;
  const int64_t l0 = ctx->launches;
  cudaGraph_t g = nullptr, body = nullptr;
  GP_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  try {
    GP_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    int32_t* it = f->refine_it;
    // [residual, test]
    GP_CUDA(cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    residual_impl(ctx, f, f->rhs, f->alpha, res, errv, nullptr);
    k_refine_test<<<1, 32, 0, st>>>(errv, B, it, f->refine_runs, f->tiles_err, 1, h);
    GP_CHECK_LAUNCH(ctx);
    cudaGraph_t gg = nullptr;
    GP_CUDA(cudaStreamEndCapture(st, &gg));
    // the loop node after the captured nodes without successors
    size_t nn = 0;
    GP_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn), sinks;
    GP_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
    for (cudaGraphNode_t v : nodes) {
      size_t nd = 0;
      GP_CUDA(cudaGraphNodeGetDependentNodes(v, nullptr, nullptr, &nd));
      if (nd == 0) sinks.push_back(v);
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop = nullptr;
    GP_CUDA(cudaGraphAddNode(&loop, g, sinks.data(), nullptr, sinks.size(), &cp));
    body = cp.conditional.phGraph_out[0];
    // body: correction, alpha update, residual, test
    GP_CUDA(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const int64_t lb = ctx->launches;
    solve_impl(ctx, f, store, res, cor, false);
    k_axpy<<<grid_for((int64_t)B * n, 256), 256, 0, st>>>(f->alpha, cor, (int64_t)B * n);
    GP_CHECK_LAUNCH(ctx);
    residual_impl(ctx, f, f->rhs, f->alpha, res, errv, nullptr);
    k_refine_test<<<1, 32, 0, st>>>(errv, B, it, f->refine_runs, f->tiles_err, 0, h);
    GP_CHECK_LAUNCH(ctx);
    f->n_refine_body = ctx->launches - lb;
    GP_CUDA(cudaStreamEndCapture(st, &gg));
    // after the loop: r . alpha and the log-likelihood
    GP_CUDA(cudaStreamBeginCaptureToGraph(st, g, &loop, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    residual_impl(ctx, f, f->rhs, f->alpha, nullptr, d_err ? d_err : errv, s_quad);
    k_finish<<<grid_for(B, 128), 128, 0, st>>>(B, n, s_log, s_quad, f->notpd, f->tiles_err, d_out);
    GP_CHECK_LAUNCH(ctx);
    GP_CUDA(cudaStreamEndCapture(st, &gg));
  } catch (...) {
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(st, &junk);
    }
    cudaGetLastError();
    cudaGraphDestroy(g);
    ctx->launches = l0;
    throw;
  }
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) throw GpError{GP_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)};
  *nl = ctx->launches - l0 - f->n_refine_body;   // a replay counts the loop body only as it runs (below)
  ctx->launches = l0;
  f->refine_out = d_out;
  f->refine_err = d_err;
  return ex;
}

void loglik_run(gp_ctx* ctx, gp_factor_t* f, const double* d_resid, double* d_out, double* d_err) {
  ProfScope ps_(ctx, KC_SOLVE);   // the whole solve (with refinement) as one timed span
  gp_pointset* ps = f->ps;
  const int B = f->B;
  const int64_t n = ps->n;
  const int nblk = (int)((n + 1023) / 1024);
  // f->red: B x red_stride partials, then 4B sums
  double* sums = f->red + (size_t)B * f->red_stride;
  double* s_log = sums;            // [2b] = sum log L_jj, [2b+1] = sum x^2
  double* s_quad = sums + 2 * B;   // [2b+1] = r . alpha (mixed)
  // the solve graph reads the right-hand side from the factor's own buffer
  GP_CUDA(cudaMemcpyAsync(f->rhs, d_resid, sizeof(double) * (size_t)B * n, cudaMemcpyDeviceToDevice, ctx->stream));
  if (f->prec == GP_FP64) {
    StoreF64 store{f->panels, ps->sp.panel_entries, f->dinv, ps->sp.diag_entries};
    run_maybe_graph(ctx, &f->gx_solve, &f->n_solve, [&] {
      solve_impl(ctx, f, store, f->rhs, f->alpha, true);
      k_sum2<<<B, 256, 0, ctx->stream>>>(f->red, f->red_stride, nblk, s_log);
      GP_CHECK_LAUNCH(ctx);
    });
    k_finish<<<grid_for(B, 128), 128, 0, ctx->stream>>>(B, n, s_log, s_log, f->notpd, nullptr, d_out);
    GP_CHECK_LAUNCH(ctx);
    if (d_err) residual_impl(ctx, f, f->rhs, f->alpha, nullptr, d_err, nullptr);
    return;
  }
  StoreMix store{f->panels32, f->diag, ps->sp.panel32_entries, ps->sp.diag_entries, f->dinv32};
  run_maybe_graph(ctx, &f->gx_solve, &f->n_solve, [&] {
    solve_impl(ctx, f, store, f->rhs, f->alpha, true);
    k_sum2<<<B, 256, 0, ctx->stream>>>(f->red, f->red_stride, nblk, s_log);
    GP_CHECK_LAUNCH(ctx);
  });
  // A11: FP64 iterative refinement of alpha
  double* res = f->delta;                       // B x n residual
  double* cor = f->delta + (size_t)B * n;       // B x n correction
  double* errv = f->red;                        // B relative residuals (partials are consumed already)
  if (use_graphs(ctx)) {   // the whole refinement as one graph: the loop's test runs on the device
    if (f->gx_refine && (f->refine_out != d_out || f->refine_err != d_err)) {
      GP_CUDA(cudaGraphExecDestroy(f->gx_refine));
      f->gx_refine = nullptr;
    }
    if (!f->gx_refine) f->gx_refine = build_refine_graph(ctx, f, store, res, cor, errv, s_log, s_quad, d_out, d_err,
                                                         &f->n_refine);
    replay_graph(ctx, f->gx_refine, f->n_refine);
    return;
  }
  std::vector<double> herr(B);
  int32_t terr = 0;
  for (int it = 0; it < 10; it++) {
    residual_impl(ctx, f, f->rhs, f->alpha, res, errv, nullptr);
    d2h(ctx, herr.data(), errv, B);
    if (it == 0) d2h(ctx, &terr, f->tiles_err, 1);
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
    if (terr != 0) break;   // the factorization timed out: the outputs become NaN below
    double worst = 0.0;
    for (int b = 0; b < B; b++) worst = std::max(worst, std::isfinite(herr[b]) ? herr[b] : 1.0);
    if (worst <= 1e-12) break;
    run_maybe_graph(ctx, &f->gx_cor, &f->n_cor, [&] {
      solve_impl(ctx, f, store, res, cor, false);
      k_axpy<<<grid_for((int64_t)B * n, 256), 256, 0, ctx->stream>>>(f->alpha, cor, (int64_t)B * n);
      GP_CHECK_LAUNCH(ctx);
    });
  }
  residual_impl(ctx, f, f->rhs, f->alpha, nullptr, d_err ? d_err : errv, s_quad);
  k_finish<<<grid_for(B, 128), 128, 0, ctx->stream>>>(B, n, s_log, s_quad, f->notpd, f->tiles_err, d_out);
  GP_CHECK_LAUNCH(ctx);
  if (terr != 0) throw GpError{GP_ERR_TIMEOUT, "a bounded wait of the factorization's tensor-core updates ran out"};
}

// Entries (per proposal) of the backward partial-sum scratch: the largest level's tasks x row chunks x 64.
int64_t bwd_part_entries(const SymPlan& sp) {
  int64_t e = 64;
  for (int32_t L = 0; L < sp.nlevels; L++)
    if (sp.level_large[L].count > 0) e = std::max<int64_t>(e, sp.level_large[L].count * bwd_chunks(sp, L) * T);
  return e;
}
