// solve.cu -- steps A8-A11: supernodal forward and backward solves with the multifrontal factor, the
// quadratic form, the log-determinant, FP64 iterative refinement (mixed precision) and the log-likelihood
//   log p(z | beta, theta) = -1/2 log det C_z - 1/2 r^T C_z^{-1} r - n/2 log(2 pi)      (Sec. 3.3)
// with log det C_z = 2 sum_j log L_jj.
//
// Forward (levels ascending): the front vector of supernode s (m entries, own columns then the rows below)
// starts as the permuted right-hand side on its columns, receives every child's update vector through the
// child's relative indices (children in order), then x = L11^{-1} f_1 and f_2 -= L21 x; f_2 is the update
// vector handed to the parent. Backward (levels descending): t = x - L21^T alpha'(rows below), then
// L11^T z = t. Fronts of order <= 96 use one CTA; the larger fronts of a level take one launch per sweep, in
// tasks of 64 rows (forward) or 64 columns (backward) that wait for the blocks they need (k_fwd_flow,
// k_bwd_flow), each block solved with the inverted 64 x 64 diagonal block the factorization formed.
// The kernels read the factor through an accessor: FP64 column-major panels (GP_FP64) or FP32 row-major
// panels with FP64 diagonal tiles (GP_MIXED). In GP_FP64 the solves run in FP64 and the quadratic form is
// |L^{-1} P r|^2. In GP_MIXED the solves run in FP32 (FP32 inverses, FP32 vectors): they only precondition
// the FP64 refinement of alpha (residual r - C alpha from the FP64 CSR values, correction through the same
// factor) until |r - C alpha| / |r| <= 1e-10 (the factor's tolerance; 1e-12 before a prediction) or 10 sweeps;
// the quadratic form is alpha^T (2 r - C alpha) in FP64, exact to second order in the residual, and the
// log-determinant is summed in FP64 from the FP64 diagonal tiles.
// Sums use fixed-shape trees, so results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <type_traits>
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

// Children's update vectors into the front vector of each supernode of the list: CTA (x, y, z) takes rows
// [GATHER_ROWS y, GATHER_ROWS (y + 1)) of front list[x] for proposal z, and adds, child by child in child order,
// the entries whose relative index falls there (rel is increasing, so they are one range per child). Every row
// receives its children's entries in child order whatever the row split, so the sums do not depend on it.
constexpr int GATHER_ROWS = 1024;
__device__ __forceinline__ int32_t lower_bound_i32(const int32_t* __restrict__ a, int32_t n, int32_t key) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
template <class V>
__global__ void k_fwd_gather(const int32_t* __restrict__ list, DevPlan dp, V* __restrict__ work, int64_t ws) {
  const int32_t s = list[blockIdx.x];
  const int64_t m = (int64_t)dp.w[s] + dp.r[s];
  const int64_t lo = (int64_t)blockIdx.y * GATHER_ROWS;
  if (lo >= m) return;
  const int32_t rlo = (int32_t)lo, rhi = (int32_t)min(m, lo + GATHER_ROWS);
  V* W = work + (int64_t)blockIdx.z * ws;
  V* fv = W + dp.frow_off[s];
  __shared__ int32_t rng[2];
  for (int32_t q = dp.ch_ptr[s]; q < dp.ch_ptr[s + 1]; q++) {
    const int32_t c = dp.ch_idx[q];
    const V* uc = W + dp.frow_off[c] + dp.w[c];
    const int32_t* rel = dp.relidx + dp.relidx_off[c];
    if (threadIdx.x < 2) rng[threadIdx.x] = lower_bound_i32(rel, dp.r[c], threadIdx.x == 0 ? rlo : rhi);
    __syncthreads();
    const int32_t a0 = rng[0], a1 = rng[1];
    for (int32_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) fv[rel[a]] += uc[a];
    __syncthreads();   // this child's entries land before the next child's, and rng is free again
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

// ---------------------------------------------------------------------------------------------------------
// The large fronts of a level, one launch per sweep. Every CTA draws a ticket, the index of its task in the
// level's task list (tasks x proposals, proposals inner), and waits (bounded) only for blocks that tasks with
// lower tickets publish. A task that drew a ticket is running, so the lowest unfinished ticket never waits for
// an unfinished task and every wait ends.
//   forward task (s, i < nb): x_i = inv(L_ii) (f_i - sum_{J < i} L_iJ x_J), written to x and published (flag i);
//   forward task (s, i >= nb): f_R -= sum_{J < nb} L_RJ x_J for the 64 rows R = w + 64 (i - nb) + [0, 64)
//     below the front's columns (the update vector handed to the parent);
//   backward task (s, J): z_J = inv(L_JJ)^T (t_J - sum_{I > J} L_IJ^T z_I), with t_J = x_J - L_{R,J}^T alpha'(R)
//     as the level's partial-sum launches left it in the front vector, written to alpha' and published (flag J).
// A task publishes only after it has read every block it needs, so a published flag implies all flags before it
// (after it, backward): one acquire of the last block a task needs covers the rest once the chain has passed.
// A task reads the L tile of its next block while it waits for the current one. Every task sums its blocks in
// a fixed order (J ascending, I descending) with fixed-shape trees, so results do not depend on timing.

__device__ __forceinline__ int32_t ld_acquire_gpu(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int32_t* p, int32_t v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits (every calling thread polls; a converged warp makes one request per poll) until *flag != 0. A wait that
// runs out of polls or time sets *err and returns: the task goes on with what it has and the factor reports
// the timeout (its log-likelihoods become NaN). Once *err is set no wait of the factor waits any longer, so a
// launch ends soon after its first wait ran out.
__device__ __forceinline__ void wait_flag(const int32_t* flag, tcg::WaitLimit lim, int32_t* err) {
  if (ld_acquire_gpu(flag) != 0) return;
  const uint64_t t0 = tcg::global_ns();
  for (uint32_t it = 1; it < lim.polls; it++) {
    __nanosleep(20);
    if (ld_acquire_gpu(flag) != 0) return;
    if ((it & 15) == 15 && (tcg::global_ns() - t0 > lim.ns || ld_acquire_gpu(err) != 0)) break;
  }
  atomicExch(err, 1);
}

// The CTA's ticket (thread 0 draws it; all threads get it).
__device__ __forceinline__ int draw_ticket(int32_t* ticket, int* slot) {
  if (threadIdx.x == 0) *slot = atomicAdd(ticket, 1);
  __syncthreads();
  return *slot;
}

// y = M f for a 64 x 64 matrix staged in shared memory as Ms[l * (T + 1) + q] = M[q][l] (the forward solve's
// inverse, transposed) or = M[l][q] (the backward solve's inverse^T), f in shared memory; the product is split
// four ways over l and combined in a fixed order; y[q] = 0 for q >= bw.
template <class V>
__device__ __forceinline__ void block_apply(const V* Ms, const V* fvec, V* y, V (*part)[T], int bw) {
  const int g = threadIdx.x >> 6, q = threadIdx.x & 63;
  V acc = 0;
#pragma unroll
  for (int l = g * 16; l < g * 16 + 16; l++) acc += Ms[l * (T + 1) + q] * fvec[l];
  part[g][q] = acc;
  __syncthreads();
  if (threadIdx.x < T) y[threadIdx.x] = threadIdx.x < bw ? (part[0][q] + part[1][q]) + (part[2][q] + part[3][q]) : V(0);
  __syncthreads();
}

constexpr int FS = T + 1;   // row stride of the shared 64 x 64 tiles
// Dynamic shared memory of a flow kernel with SB blocks per chain task: the blocks' inverses and, for SB = 2,
// the tile between the two blocks.
template <class V, int SB>
constexpr size_t flow_smem_bytes() { return (SB == 1 ? 1 : 3) * (size_t)T * FS * sizeof(V); }
template <class V, int SB>
constexpr int flow_min_blocks() { return sizeof(V) == 4 ? (SB == 1 ? 4 : 2) : 1; }

// Forward, SB (1 or 2) blocks per chain task; rows below the columns in tasks of 64 SB rows.
template <class St, int SB>
__global__ void __launch_bounds__(256, flow_min_blocks<typename St::V, SB>())
    k_fwd_flow(const int2* __restrict__ tasks, int B, DevPlan dp, St store, typename St::V* __restrict__ work,
               int64_t ws, int64_t xv_off, int32_t* __restrict__ ticket, int32_t* __restrict__ flags, int64_t nfl,
               int32_t* __restrict__ err, tcg::WaitLimit lim) {
  using V = typename St::V;
  extern __shared__ __align__(16) unsigned char flow_sh[];
  V* Ms0 = reinterpret_cast<V*>(flow_sh);   // Ms_k[l][q] = inv(L_{i0+k})[q][l]
  V* Ms1 = Ms0 + T * FS;
  V* Tl = Ms1 + T * FS;                      // Tl[q][l] = L[64 (i0 + 1) + q, 64 i0 + l] (SB = 2)
  __shared__ V fsh[SB * T], tots[SB * T], fb[T], x[T], part[4][T];
  __shared__ int tk_s;
  const int tk = draw_ticket(ticket, &tk_s);
  const int2 task = tasks[tk / B];
  const int b = tk % B;
  const int32_t s = task.x;
  auto A = store.acc(dp, s, b);
  V* W = work + (int64_t)b * ws;
  V* fv = W + dp.frow_off[s];
  V* xs = W + xv_off + dp.sn_first[s];   // x on the front's columns
  const int w = dp.w[s];
  const int64_t m = (int64_t)w + dp.r[s];
  const int nb = (w + T - 1) / T, nbs = (nb + SB - 1) / SB;
  int32_t* fl = flags + (int64_t)b * nfl + dp.sn_fl[s];
  const bool own = task.y < nbs;
  const int i0 = own ? task.y * SB : 0;
  const int nblk = own ? min(SB, nb - i0) : 0;
  const int64_t r0 = own ? (int64_t)i0 * T : (int64_t)w + (int64_t)(task.y - nbs) * (SB * T);
  const int nr = (int)imin64(SB * T, (own ? (int64_t)w : m) - r0);   // rows of the task
  const int nJ = own ? i0 : nb;
  if (own) {   // the blocks' inverses, the tile between them and f, staged while the earlier blocks arrive
    for (int k = 0; k < nblk; k++) {
      const V* inv = store.inv(dp, s, b) + (int64_t)(i0 + k) * T * T;
      V* Ms = k == 0 ? Ms0 : Ms1;
#pragma unroll 4
      for (int u = 0; u < T * T / 256; u++) {
        const int q = threadIdx.x + u * 256;
        Ms[(q & 63) * FS + (q >> 6)] = inv[q];
      }
    }
    if (SB == 2 && nblk == 2) {
#pragma unroll 4
      for (int u = 0; u < T * T / 256; u++) {
        const int e = threadIdx.x + u * 256;
        const int q = St::kRowMajor ? e >> 6 : e & 63, l = St::kRowMajor ? e & 63 : e >> 6;
        Tl[q * FS + l] = T + q < nr ? (V)A.L(r0 + T + q, (int64_t)i0 * T + l) : V(0);
      }
    }
    if (threadIdx.x < SB * T) fsh[threadIdx.x] = threadIdx.x < nr ? fv[r0 + threadIdx.x] : V(0);
  }
  int ready = -1;   // blocks [0, ready] are known published
  auto need = [&](int J) {   // one acquire also covers the next 8 blocks when they are already out
    if (J <= ready) return;
    const int ahead = min(nJ - 1, J + 8);
    if (ld_acquire_gpu(fl + ahead) != 0) {
      ready = ahead;
      return;
    }
    wait_flag(fl + J, lim, err);
    ready = J;
  };
  // tots[q] = sum_{J < nJ} L[r0 + q, J] x_J for the task's rows
  if constexpr (St::kRowMajor) {
    // a half-warp reads one row's 64 entries of a tile as 16 float4: rows hw + 16 u of the task (u < RU); the
    // next tile is read while the current one is used, and so are its x values once they are known published;
    // a lane sums its four columns over all tiles, the row's 16 lanes are combined at the end
    constexpr int RU = SB * T / 16;
    const int hw = threadIdx.x >> 4, l = (threadIdx.x & 15) * 4;
    auto load = [&](int J, float4 (&v)[RU]) {
      const int c0 = J * T, bw = min(T, w - c0);
#pragma unroll
      for (int u = 0; u < RU; u++) {
        const int rr = hw + 16 * u;
        v[u] = (rr < nr && l < bw) ? *reinterpret_cast<const float4*>(A.P + (r0 + rr) * A.ldw + c0 + l)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto loadx = [&](int J, float (&xq)[4]) {
      const int c0 = J * T, bw = min(T, w - c0);
#pragma unroll
      for (int e = 0; e < 4; e++) xq[e] = l + e < bw ? __ldcg(xs + c0 + l + e) : 0.f;
    };
    float acc[RU];
#pragma unroll
    for (int u = 0; u < RU; u++) acc[u] = 0.f;
    float4 v[RU], vn[RU];
    float xq[4], xn[4];
    bool have_x = false;
    if (nJ > 0) load(0, v);
    for (int J = 0; J < nJ; J++) {
      if (J + 1 < nJ) load(J + 1, vn);
      need(J);
      if (!have_x) loadx(J, xq);
      const bool have_xn = J + 1 < nJ && J + 1 <= ready;
      if (have_xn) loadx(J + 1, xn);
#pragma unroll
      for (int u = 0; u < RU; u++) acc[u] += v[u].x * xq[0] + v[u].y * xq[1] + v[u].z * xq[2] + v[u].w * xq[3];
      if (J + 1 < nJ) {
#pragma unroll
        for (int u = 0; u < RU; u++) v[u] = vn[u];
#pragma unroll
        for (int e = 0; e < 4; e++) xq[e] = xn[e];
      }
      have_x = have_xn;
    }
#pragma unroll
    for (int u = 0; u < RU; u++) {   // the 16 lanes of a row: a fixed tree
      for (int o = 8; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
    }
    if ((threadIdx.x & 15) == 0) {
#pragma unroll
      for (int u = 0; u < RU; u++) tots[hw + 16 * u] = acc[u];
    }
  } else {
    // thread (g, q): row r0 + q (q < 64 SB), the columns 64 / G g + [0, 64 / G) of each tile (G = 256 / (64 SB))
    constexpr int NQ = SB * T, G = 256 / NQ, CW = T / G;
    const int g = threadIdx.x / NQ, q = threadIdx.x % NQ;
    V acc = 0;
    for (int J = 0; J < nJ; J++) {
      need(J);
      const int c0 = J * T, bw = min(T, w - c0);
      if (q < nr)
        for (int e = 0; e < CW; e++) {
          const int l = g * CW + e;
          if (l < bw) acc += A.L(r0 + q, c0 + l) * __ldcg(xs + c0 + l);
        }
    }
    V* pp = &part[0][0];   // 4 x 64 entries: G - 1 partial rows of NQ
    if (g > 0) pp[(g - 1) * NQ + q] = acc;
    __syncthreads();
    if (g == 0) {
      for (int k = 1; k < G; k++) acc += pp[(k - 1) * NQ + q];
      tots[q] = acc;
    }
  }
  __syncthreads();
  if (!own) {
    if (threadIdx.x < nr) fv[r0 + threadIdx.x] -= tots[threadIdx.x];
    return;
  }
  // block i0
  const int nr0 = min(T, nr);
  if (threadIdx.x < T) fb[threadIdx.x] = threadIdx.x < nr0 ? fsh[threadIdx.x] - tots[threadIdx.x] : V(0);
  __syncthreads();
  block_apply(Ms0, fb, x, part, nr0);
  if (threadIdx.x < nr0) xs[r0 + threadIdx.x] = x[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) st_release_gpu(fl + i0, 1);
  if (SB == 1 || nblk < 2) return;
  // block i0 + 1: f -= L[i0 + 1, i0] x_{i0}
  const int nr1 = nr - T;
  {
    const int g = threadIdx.x >> 6, q = threadIdx.x & 63;
    V a = 0;
#pragma unroll
    for (int l = g * 16; l < g * 16 + 16; l++) a += Tl[q * FS + l] * x[l];
    part[g][q] = a;
  }
  __syncthreads();
  if (threadIdx.x < T) {
    const int q = threadIdx.x;
    fb[q] = q < nr1 ? (fsh[T + q] - tots[T + q]) - ((part[0][q] + part[1][q]) + (part[2][q] + part[3][q])) : V(0);
  }
  __syncthreads();
  block_apply(Ms1, fb, x, part, nr1);
  if (threadIdx.x < nr1) xs[r0 + T + threadIdx.x] = x[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) st_release_gpu(fl + i0 + 1, 1);
}

// Backward, SB (1 or 2) blocks per chain task.
template <class St, int SB>
__global__ void __launch_bounds__(256, flow_min_blocks<typename St::V, SB>())
    k_bwd_flow(const int2* __restrict__ tasks, int B, DevPlan dp, St store, typename St::V* __restrict__ work,
               int64_t ws, int64_t apv_off, int32_t* __restrict__ ticket, int32_t* __restrict__ flags, int64_t nfl,
               int32_t* __restrict__ err, tcg::WaitLimit lim) {
  using V = typename St::V;
  extern __shared__ __align__(16) unsigned char flow_sh[];
  V* Ms0 = reinterpret_cast<V*>(flow_sh);   // Ms_k[l][q] = inv(L_{J0+k})[l][q]: z_q = sum_l inv[l][q] t_l
  V* Ms1 = Ms0 + T * FS;
  V* Tl = Ms1 + T * FS;                      // Tl[l][q] = L[64 (J0 + 1) + l, 64 J0 + q] (SB = 2)
  __shared__ V tsh[SB * T], psum[SB * T], tb[T], z[T], part[4][T];
  __shared__ V red[256 / (SB * T / 4)][SB * T];   // row groups x columns
  __shared__ int tk_s;
  const int tk = draw_ticket(ticket, &tk_s);
  const int2 task = tasks[tk / B];
  const int b = tk % B;
  const int32_t s = task.x;
  const int J0 = task.y * SB;
  auto A = store.acc(dp, s, b);
  V* W = work + (int64_t)b * ws;
  V* fv = W + dp.frow_off[s];
  V* zs = W + apv_off + dp.sn_first[s];   // alpha' on the front's columns
  const int w = dp.w[s];
  const int nb = (w + T - 1) / T;
  const int nblk = min(SB, nb - J0);
  const int c0 = J0 * T, nc = min(SB * T, w - c0);   // the task's columns
  int32_t* fl = flags + (int64_t)b * nfl + dp.sn_fl[s];
  for (int k = 0; k < nblk; k++) {
    const V* inv = store.inv(dp, s, b) + (int64_t)(J0 + k) * T * T;
    V* Ms = k == 0 ? Ms0 : Ms1;
#pragma unroll 4
    for (int u = 0; u < T * T / 256; u++) {
      const int q = threadIdx.x + u * 256;
      Ms[(q >> 6) * FS + (q & 63)] = inv[q];
    }
  }
  if (SB == 2 && nblk == 2) {
    const int bw1 = nc - T;
#pragma unroll 4
    for (int u = 0; u < T * T / 256; u++) {
      const int e = threadIdx.x + u * 256;
      const int l = St::kRowMajor ? e >> 6 : e & 63, q = St::kRowMajor ? e & 63 : e >> 6;
      Tl[l * FS + q] = l < bw1 ? (V)A.L((int64_t)c0 + T + l, c0 + q) : V(0);
    }
  }
  if (threadIdx.x < SB * T) tsh[threadIdx.x] = threadIdx.x < nc ? fv[c0 + threadIdx.x] : V(0);
  const int Itop = J0 + nblk;   // the blocks above the task: I = nb - 1 down to Itop
  int ready = nb;               // blocks [ready, nb) are known published
  auto need = [&](int I) {      // one acquire also covers the next 8 blocks when they are already out
    if (I >= ready) return;
    const int ahead = max(Itop, I - 8);
    if (ld_acquire_gpu(fl + ahead) != 0) {
      ready = ahead;
      return;
    }
    wait_flag(fl + I, lim, err);
    ready = I;
  };
  // warp k: rows RPT k + [0, RPT) of tile I; lane c: columns c0 + 4 c + [0, 4) (a warp reads RPT row segments of
  // 64 SB entries); the next tile is read while the current one is used, and so are its alpha' values once they
  // are known published
  constexpr int NQ4 = SB * T / 4, G = 256 / NQ4, RPT = T / G;
  const int g = threadIdx.x / NQ4, c4 = (threadIdx.x % NQ4) * 4;
  using V4 = typename std::conditional<sizeof(V) == 4, float4, double4>::type;
  auto load = [&](int I, V4 (&v)[RPT]) {
    const int bwI = min(T, w - I * T);
#pragma unroll
    for (int e = 0; e < RPT; e++) {
      const int l = g * RPT + e;
      const int64_t row = (int64_t)I * T + l;
      if (l < bwI && c4 < nc) {
        if constexpr (St::kRowMajor) {
          v[e] = *reinterpret_cast<const V4*>(A.P + row * A.ldw + c0 + c4);
        } else {
          v[e].x = A.L(row, c0 + c4);
          v[e].y = c4 + 1 < nc ? A.L(row, c0 + c4 + 1) : V(0);
          v[e].z = c4 + 2 < nc ? A.L(row, c0 + c4 + 2) : V(0);
          v[e].w = c4 + 3 < nc ? A.L(row, c0 + c4 + 3) : V(0);
        }
      } else {
        v[e].x = v[e].y = v[e].z = v[e].w = V(0);
      }
    }
  };
  auto loadz = [&](int I, V (&zq)[RPT]) {
    const int bwI = min(T, w - I * T);
#pragma unroll
    for (int e = 0; e < RPT; e++) {
      const int l = g * RPT + e;
      zq[e] = l < bwI ? __ldcg(zs + I * T + l) : V(0);
    }
  };
  V acc[4] = {0, 0, 0, 0};
  {
    V4 v[RPT], vn[RPT];
    V zq[RPT], zn[RPT];
    bool have_z = false;
    if (nb - 1 >= Itop) load(nb - 1, v);
    for (int I = nb - 1; I >= Itop; I--) {
      if (I - 1 >= Itop) load(I - 1, vn);
      need(I);
      if (!have_z) loadz(I, zq);
      const bool have_zn = I - 1 >= Itop && I - 1 >= ready;
      if (have_zn) loadz(I - 1, zn);
#pragma unroll
      for (int e = 0; e < RPT; e++) {
        acc[0] += v[e].x * zq[e];
        acc[1] += v[e].y * zq[e];
        acc[2] += v[e].z * zq[e];
        acc[3] += v[e].w * zq[e];
      }
      if (I - 1 >= Itop) {
#pragma unroll
        for (int e = 0; e < RPT; e++) {
          v[e] = vn[e];
          zq[e] = zn[e];
        }
      }
      have_z = have_zn;
    }
  }
  // psum[col] = sum over the row groups (warps) of the partial sums, in group order
  {
#pragma unroll
    for (int k = 0; k < 4; k++) red[g][c4 + k] = acc[k];
    __syncthreads();
    if (threadIdx.x < SB * T) {
      V t = 0;
      for (int k = 0; k < G; k++) t += red[k][threadIdx.x];
      psum[threadIdx.x] = t;
    }
    __syncthreads();
  }
  if (SB == 2 && nblk == 2) {   // block J0 + 1 first
    const int bw1 = nc - T;
    if (threadIdx.x < T) tb[threadIdx.x] = threadIdx.x < bw1 ? tsh[T + threadIdx.x] - psum[T + threadIdx.x] : V(0);
    __syncthreads();
    block_apply(Ms1, tb, z, part, bw1);
    if (threadIdx.x < bw1) zs[c0 + T + threadIdx.x] = z[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) st_release_gpu(fl + J0 + 1, 1);
    // block J0: t -= L[J0 + 1, J0]^T z_{J0 + 1}
    {
      const int gg = threadIdx.x >> 6, qq = threadIdx.x & 63;
      V a = 0;
#pragma unroll
      for (int l = gg * 16; l < gg * 16 + 16; l++) a += Tl[l * FS + qq] * z[l];
      part[gg][qq] = a;
    }
    __syncthreads();
    if (threadIdx.x < T) {
      const int qq = threadIdx.x;
      tb[qq] = (tsh[qq] - psum[qq]) - ((part[0][qq] + part[1][qq]) + (part[2][qq] + part[3][qq]));
    }
  } else if (threadIdx.x < T) {
    tb[threadIdx.x] = threadIdx.x < nc ? tsh[threadIdx.x] - psum[threadIdx.x] : V(0);
  }
  __syncthreads();
  const int bw0 = min(T, nc);
  block_apply(Ms0, tb, z, part, bw0);
  if (threadIdx.x < bw0) zs[c0 + threadIdx.x] = z[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) st_release_gpu(fl + J0, 1);
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
    ra = a[i] * (ri + rr);   // alpha_i (2 r_i - (C alpha)_i): the second-order form of r^T C^-1 r
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

// The refinement loop's test on the device: continue while some proposal's |r - C alpha| / |r| exceeds tol (or
// is not finite) and fewer than 10 corrections have run. it[0] counts the corrections; a factorization whose
// bounded waits ran out (tc_err) stops the loop at once (its outputs become NaN).
__global__ void k_refine_test(const double* __restrict__ err, int B, double tol, int32_t* __restrict__ it,
                              unsigned long long* __restrict__ runs, const int32_t* __restrict__ tc_err, int reset,
                              cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  if (reset) it[0] = 0;
  double worst = 0.0;
  for (int b = 0; b < B; b++) worst = fmax(worst, isfinite(err[b]) ? err[b] : 1.0);
  const bool more = worst > tol && it[0] < 10 && !(tc_err && *tc_err);
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

// Dynamic shared memory of the flow kernels (above the 48 KB default), set once per process.
template <class St, int SB>
void flow_attrs() {
  static const bool done = [] {
    const int bytes = (int)flow_smem_bytes<typename St::V, SB>();
    cudaFuncSetAttribute(k_fwd_flow<St, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_bwd_flow<St, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return true;
  }();
  (void)done;
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
  // tickets and readiness flags of the large fronts' tasks
  GP_CUDA(cudaMemsetAsync(f->flow_sync, 0, sizeof(int32_t) * (size_t)flow_sync_entries(sp, B), st));
  int32_t* fwd_flags = f->flow_sync + 2 * sp.nlevels;
  int32_t* bwd_flags = fwd_flags + (int64_t)B * sp.n_fl;
  flow_attrs<St, 1>();
  flow_attrs<St, 2>();
  k_rhs<<<dim3(grid_for(n, 256), B), 256, 0, st>>>(rhs, ps->perm, n, dp, work, ws);
  GP_CHECK_LAUNCH(ctx);
  for (int32_t L = 0; L < sp.nlevels; L++) {
    const SymPlan::Level& lv = sp.levels[L];
    int32_t nl = sp.lev_ptr[L + 1] - sp.lev_ptr[L];
    if (L > 0) {
      int64_t mmax = 1;   // row chunks of the level's largest front
      for (int32_t q = sp.lev_ptr[L]; q < sp.lev_ptr[L + 1]; q++) {
        const int32_t s = sp.lev_sn[q];
        mmax = std::max<int64_t>(mmax, (int64_t)sp.sn_w[s] + sp.sn_r[s]);
      }
      const unsigned nch = (unsigned)((mmax + GATHER_ROWS - 1) / GATHER_ROWS);
      k_fwd_gather<<<dim3(nl, nch, B), 256, 0, st>>>(dp.lev_sn + sp.lev_ptr[L], dp, work, ws);
      GP_CHECK_LAUNCH(ctx);
    }
    if (lv.nsmall > 0) {
      k_fwd_small<St><<<dim3(lv.nsmall, B), 128, 0, st>>>(dp.small_list + lv.small_off, dp, store, work, ws,
                                                          xv_off);
      GP_CHECK_LAUNCH(ctx);
    }
    const int64_t nt = sp.flow_fwd_ptr[L + 1] - sp.flow_fwd_ptr[L];
    if (nt > 0) {
      const auto kf = lv.flow_sb == 2 ? k_fwd_flow<St, 2> : k_fwd_flow<St, 1>;
      const size_t sm = lv.flow_sb == 2 ? flow_smem_bytes<V, 2>() : flow_smem_bytes<V, 1>();
      kf<<<(unsigned)(nt * B), 256, sm, st>>>(dp.flow_fwd + sp.flow_fwd_ptr[L], B, dp, store, work, ws, xv_off,
                                              f->flow_sync + 2 * L, fwd_flags, sp.n_fl, f->tiles_err, f->wait_lim);
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
      const int64_t nt = sp.flow_bwd_ptr[L + 1] - sp.flow_bwd_ptr[L];
      const auto kb = lv.flow_sb == 2 ? k_bwd_flow<St, 2> : k_bwd_flow<St, 1>;
      const size_t sm = lv.flow_sb == 2 ? flow_smem_bytes<V, 2>() : flow_smem_bytes<V, 1>();
      kb<<<(unsigned)(nt * B), 256, sm, st>>>(dp.flow_bwd + sp.flow_bwd_ptr[L], B, dp, store, work, ws, apv_off,
                                              f->flow_sync + 2 * L + 1, bwd_flags, sp.n_fl, f->tiles_err,
                                              f->wait_lim);
      GP_CHECK_LAUNCH(ctx);
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
// correction, residual, test], then, if finish, [final residual with the quadratic form, log-likelihood] into
// d_out / d_err (gp_loglik passes the factor's own result buffer, so one graph serves every caller). The test kernel
// sets the loop's condition (cudaGraphSetConditional); the loop stops at relative residual tol. *nl receives the
// launches of one pass (the body counted once).
template <class St>
static cudaGraphExec_t build_refine_graph(gp_ctx* ctx, gp_factor_t* f, const St& store, double* res, double* cor,
                                          double* errv, double* s_log, double* s_quad, double* d_out, double* d_err,
                                          int64_t* nl, double tol, bool finish) {
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
    k_refine_test<<<1, 32, 0, st>>>(errv, B, tol, it, f->refine_runs, f->tiles_err, 1, h);
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
    k_refine_test<<<1, 32, 0, st>>>(errv, B, tol, it, f->refine_runs, f->tiles_err, 0, h);
    GP_CHECK_LAUNCH(ctx);
    f->n_refine_body = ctx->launches - lb;
    GP_CUDA(cudaStreamEndCapture(st, &gg));
    if (finish) {   // after the loop: the quadratic form and the log-likelihood
      GP_CUDA(cudaStreamBeginCaptureToGraph(st, g, &loop, nullptr, 1, cudaStreamCaptureModeThreadLocal));
      residual_impl(ctx, f, f->rhs, f->alpha, nullptr, d_err ? d_err : errv, s_quad);
      k_finish<<<grid_for(B, 128), 128, 0, st>>>(B, n, s_log, s_quad, f->notpd, f->tiles_err, d_out);
      GP_CHECK_LAUNCH(ctx);
      GP_CUDA(cudaStreamEndCapture(st, &gg));
    }
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
  if (finish) {
    f->refine_out = d_out;
    f->refine_err = d_err;
  }
  return ex;
}

// Host-driven refinement of alpha (the legacy default stream, where graphs are not used) until every proposal's
// relative residual is at most tol or 10 corrections have run; *terr receives the factorization's timeout flag.
template <class St>
static void refine_host_loop(gp_ctx* ctx, gp_factor_t* f, const St& store, double* res, double* cor, double* errv,
                             double tol, int32_t* terr) {
  const int B = f->B;
  const int64_t n = f->ps->n;
  std::vector<double> herr(B);
  *terr = 0;
  for (int it = 0; it < 10; it++) {
    residual_impl(ctx, f, f->rhs, f->alpha, res, errv, nullptr);
    d2h(ctx, herr.data(), errv, B);
    if (it == 0) d2h(ctx, terr, f->tiles_err, 1);
    GP_CUDA(cudaStreamSynchronize(ctx->stream));
    if (*terr != 0) break;   // the factorization timed out: the outputs become NaN
    double worst = 0.0;
    for (int b = 0; b < B; b++) worst = std::max(worst, std::isfinite(herr[b]) ? herr[b] : 1.0);
    if (worst <= tol) break;
    run_maybe_graph(ctx, &f->gx_cor, &f->n_cor, [&] {
      solve_impl(ctx, f, store, res, cor, false);
      k_axpy<<<grid_for((int64_t)B * n, 256), 256, 0, ctx->stream>>>(f->alpha, cor, (int64_t)B * n);
      GP_CHECK_LAUNCH(ctx);
    });
  }
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
    // the graph writes the factor's own result buffer (so one graph serves every caller's output pointers), and
    // plain copies move the results out
    double* g_out = f->ll_buf;
    double* g_err = f->ll_buf + B;
    if (!f->gx_refine) f->gx_refine = build_refine_graph(ctx, f, store, res, cor, errv, s_log, s_quad, g_out, g_err,
                                                         &f->n_refine, f->refine_tol, true);
    replay_graph(ctx, f->gx_refine, f->n_refine);
    GP_CUDA(cudaMemcpyAsync(d_out, g_out, sizeof(double) * B, cudaMemcpyDeviceToDevice, ctx->stream));
    if (d_err) GP_CUDA(cudaMemcpyAsync(d_err, g_err, sizeof(double) * B, cudaMemcpyDeviceToDevice, ctx->stream));
    f->alpha_tol = f->refine_tol;
    return;
  }
  int32_t terr = 0;
  refine_host_loop(ctx, f, store, res, cor, errv, f->refine_tol, &terr);
  f->alpha_tol = f->refine_tol;
  residual_impl(ctx, f, f->rhs, f->alpha, nullptr, d_err ? d_err : errv, s_quad);
  k_finish<<<grid_for(B, 128), 128, 0, ctx->stream>>>(B, n, s_log, s_quad, f->notpd, f->tiles_err, d_out);
  GP_CHECK_LAUNCH(ctx);
  if (terr != 0) throw GpError{GP_ERR_TIMEOUT, "a bounded wait of the factorization's tensor-core updates ran out"};
}

// alpha of a GP_MIXED factor refined to a relative residual of at most ALPHA_TOL before a prediction uses it:
// gp_loglik may stop its refinement earlier (GP_OPT_REFINE_EXP), since its second-order quadratic form does not
// need more. Runs the remaining corrections, if any (a residual and its test when there are none).
constexpr double ALPHA_TOL = 1e-12;
void refine_alpha_for_predict(gp_ctx* ctx, gp_factor_t* f) {
  if (f->prec != GP_MIXED || f->alpha_tol <= ALPHA_TOL) return;
  gp_pointset* ps = f->ps;
  const int64_t n = ps->n;
  StoreMix store{f->panels32, f->diag, ps->sp.panel32_entries, ps->sp.diag_entries, f->dinv32};
  double* res = f->delta;
  double* cor = f->delta + (size_t)f->B * n;
  double* errv = f->red;
  if (use_graphs(ctx)) {
    if (!f->gx_tail)
      f->gx_tail = build_refine_graph(ctx, f, store, res, cor, errv, nullptr, nullptr, nullptr, nullptr, &f->n_tail,
                                      ALPHA_TOL, false);
    replay_graph(ctx, f->gx_tail, f->n_tail);
  } else {
    int32_t terr = 0;
    refine_host_loop(ctx, f, store, res, cor, errv, ALPHA_TOL, &terr);
  }
  f->alpha_tol = ALPHA_TOL;
}

// Entries (per proposal) of the backward partial-sum scratch: the largest level's tasks x row chunks x 64.
int64_t bwd_part_entries(const SymPlan& sp) {
  int64_t e = 64;
  for (int32_t L = 0; L < sp.nlevels; L++)
    if (sp.level_large[L].count > 0) e = std::max<int64_t>(e, sp.level_large[L].count * bwd_chunks(sp, L) * T);
  return e;
}
