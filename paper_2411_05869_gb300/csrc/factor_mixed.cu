// factor_mixed.cu -- step A7 in mixed precision (GP_MIXED): the multifrontal supernodal Cholesky of
// P C_z P^T with the off-diagonal supernode updates on FP16 or TF32 tensor cores (tcgen05, FP32 accumulation in
// tensor memory) and every diagonal 64 x 64 block kept, updated and factored in FP64 (optionally factored in
// FP32 from its FP64 accumulation).
//
// Storage per proposal: FP32 panels row-major (row i of supernode s at loff32 + i * ldw, K = column index
// contiguous, as the tensor-core operands want), FP64 diagonal tiles (tile t of s at doff + t * 4096, row-major
// 64 x 64), FP32 update matrices (row-major r x r). Entries (i, j) of a front with i, j < w in the same 64-block
// live in the FP64 tile, every other panel entry in FP32.
// Per level: zero the update matrices, extend-add the children (FP32 sums into the parent's FP32 entries and
// FP64 tiles), factor fronts of order <= 96 wholly in FP64 shared memory, and step the large fronts 64 columns
// at a time: POTRF of the diagonal tile (FP64, with the FP32 inverse of its factor), TRSM of the
// rows below in FP32, then the updates F[i, j] -= sum_l L[i, l] L[j, l] on the tensor cores (left-looking
// 128 x 64 strips per block, 256 x 256 CTA-pair tiles at a group's end), each FP32 operand split into two FP16
// parts of the entry times a power of two (or two TF32 parts), three products per step (the pair holds the entry
// to about 2^-22 of it), with the tile results added in FP64 to the diagonal tiles and in FP32 elsewhere.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "gp_internal.cuh"
#include "tc_gemm.cuh"

void values_run_mixed(gp_ctx* ctx, gp_factor_t* f);

namespace {

constexpr int T = GP_TILE;

struct MixFront {
  int32_t w, r, ldw;
  int64_t m;
  float* P;     // FP32 panel (m x ldw)
  double* D;    // FP64 diagonal tiles
  float* Uu;    // FP32 update matrix (r x r)
};

__device__ __forceinline__ MixFront mix_front(const DevPlan& dp, int32_t s, float* p32, double* dg, float* u32) {
  MixFront fr;
  fr.w = dp.w[s];
  fr.r = dp.r[s];
  fr.ldw = dp.ldw[s];
  fr.m = (int64_t)fr.w + fr.r;
  fr.P = p32 + dp.loff32[s];
  fr.D = dg + dp.doff[s];
  fr.Uu = u32 + dp.uoff[s];
  return fr;
}

__device__ __forceinline__ bool in_diag(const MixFront& fr, int64_t i, int64_t j) {
  return i < fr.w && (i >> 6) == (j >> 6);
}
__device__ __forceinline__ double* diag_at(const MixFront& fr, int64_t i, int64_t j) {
  return fr.D + (i >> 6) * (T * T) + (i & 63) * T + (j & 63);
}
__device__ __forceinline__ double mix_get(const MixFront& fr, int64_t i, int64_t j) {
  if (j < fr.w) return in_diag(fr, i, j) ? *diag_at(fr, i, j) : (double)fr.P[i * fr.ldw + j];
  return (double)fr.Uu[(i - fr.w) * fr.r + (j - fr.w)];
}
__device__ __forceinline__ void mix_set(const MixFront& fr, int64_t i, int64_t j, double v) {
  if (j < fr.w) {
    if (in_diag(fr, i, j)) *diag_at(fr, i, j) = v;
    else fr.P[i * fr.ldw + j] = (float)v;
  } else {
    fr.Uu[(i - fr.w) * fr.r + (j - fr.w)] = (float)v;
  }
}
__device__ __forceinline__ void mix_add(const MixFront& fr, int64_t i, int64_t j, float v) {
  if (j < fr.w) {
    if (in_diag(fr, i, j)) *diag_at(fr, i, j) += (double)v;
    else fr.P[i * fr.ldw + j] += v;
  } else {
    fr.Uu[(i - fr.w) * fr.r + (j - fr.w)] += v;
  }
}

__device__ __forceinline__ double checked_sqrt(double d, int32_t* notpd, int32_t col) {
  if (!(d > 0.0)) {
    atomicMin(notpd, col);
    return 1.0;
  }
  return sqrt(d);
}

// Row a and column b of entry e of a lower triangle stored by rows (e = a (a + 1) / 2 + b, b <= a).
__device__ __forceinline__ void tri_decode(int64_t e, int64_t& a, int64_t& b) {
  int64_t r = (int64_t)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= e) r++;
  while (r * (r + 1) / 2 > e) r--;
  a = r;
  b = e - r * (r + 1) / 2;
}

// The update matrices' lower triangles (row a, columns b <= a; nothing reads or writes the upper ones) are zeroed
// and extend-added in chunks of GP_EA_CHUNK entries in row order, one CTA per (supernode, chunk): every thread
// has work however short the rows are (the small fronts' update matrices are thousands of short rows). Thread t
// takes the chunk's entries t, t + 256, ..., EA_G of them at a time with all their loads in flight, stepping
// (row, column) along instead of decoding every entry.
constexpr int EA_THREADS = 256, EA_PER = GP_EA_CHUNK / EA_THREADS, EA_G = 4;
__device__ __forceinline__ void tri_step(int64_t e, int64_t& a, int64_t& b) {   // entry e = the previous + 256
  b += EA_THREADS;
  if (b > a) tri_decode(e, a, b);
}

__global__ void __launch_bounds__(EA_THREADS) k_zero_updates32(const int2* __restrict__ tab, DevPlan dp,
                                                               float* __restrict__ upd, int64_t UE) {
  const int2 task = tab[blockIdx.x];
  const int32_t s = task.x;
  float* U = upd + (int64_t)blockIdx.y * UE + dp.uoff[s];
  const int64_t r = dp.r[s], E = r * (r + 1) / 2;
  int64_t e = (int64_t)task.y * GP_EA_CHUNK + threadIdx.x, a, b;
  if (e >= E) return;
  tri_decode(e, a, b);
  for (int k = 0; k < EA_PER && e < E; k++) {
    U[a * r + b] = 0.f;
    e += EA_THREADS;
    if (e < E) tri_step(e, a, b);
  }
}

// Entries a, b <= a of the child's update matrix into the parent front (row rel[a], column rel[b]). The targets of
// distinct entries are distinct (rel is increasing) and a launch takes one child of each parent, so no two
// threads of a launch touch one target.
__global__ void __launch_bounds__(EA_THREADS) k_extend_add32(const int2* __restrict__ tab, DevPlan dp,
                                                             float* __restrict__ p32, double* __restrict__ dg,
                                                             float* __restrict__ u32, int64_t P32E, int64_t DE,
                                                             int64_t UE) {
  const int2 task = tab[blockIdx.x];
  const int32_t c = task.x;
  const int bp = blockIdx.y;
  float* pp = p32 + (int64_t)bp * P32E;
  double* pd = dg + (int64_t)bp * DE;
  float* pu = u32 + (int64_t)bp * UE;
  const int32_t p = dp.sn_parent[c];
  const int64_t rc = dp.r[c], E = rc * (rc + 1) / 2;
  const float* Uc = pu + dp.uoff[c];
  const int32_t* rel = dp.relidx + dp.relidx_off[c];
  const MixFront fp = mix_front(dp, p, pp, pd, pu);
  int64_t e = (int64_t)task.y * GP_EA_CHUNK + threadIdx.x, a = 0, b = 0;
  if (e >= E) return;
  tri_decode(e, a, b);
  for (int k0 = 0; k0 < EA_PER && e < E; k0 += EA_G) {
    int32_t tr[EA_G], cc[EA_G];
    float vv[EA_G];
#pragma unroll
    for (int k = 0; k < EA_G; k++) {
      tr[k] = -1;
      if (e < E) {
        tr[k] = rel[a];
        cc[k] = rel[b];
        vv[k] = Uc[a * rc + b];
        e += EA_THREADS;
        if (e < E) tri_step(e, a, b);
      }
    }
    float old[EA_G];
#pragma unroll
    for (int k = 0; k < EA_G; k++)   // a row below the parent's columns: its update-matrix row or FP32 panel row
      if (tr[k] >= fp.w)
        old[k] = cc[k] >= fp.w ? fp.Uu[(int64_t)(tr[k] - fp.w) * fp.r + (cc[k] - fp.w)]
                               : fp.P[(int64_t)tr[k] * fp.ldw + cc[k]];
#pragma unroll
    for (int k = 0; k < EA_G; k++) {
      if (tr[k] < 0) continue;
      if (tr[k] >= fp.w) {
        float* t = cc[k] >= fp.w ? fp.Uu + (int64_t)(tr[k] - fp.w) * fp.r + (cc[k] - fp.w)
                                 : fp.P + (int64_t)tr[k] * fp.ldw + cc[k];
        *t = old[k] + vv[k];
      } else {   // a row of the parent's columns: panel or FP64 diagonal tile
        mix_add(fp, tr[k], cc[k], vv[k]);
      }
    }
  }
}

// Fronts of order <= GP_SMALL_M: the whole partial factorization in FP64 shared memory.
__global__ void k_small_front32(const int32_t* __restrict__ list, DevPlan dp, float* __restrict__ p32,
                                double* __restrict__ dg, float* __restrict__ u32, int64_t P32E, int64_t DE,
                                int64_t UE, int32_t* __restrict__ notpd) {
  extern __shared__ double A[];
  int32_t s = list[blockIdx.x];
  int b = blockIdx.y;
  MixFront fr = mix_front(dp, s, p32 + (int64_t)b * P32E, dg + (int64_t)b * DE, u32 + (int64_t)b * UE);
  const int m = (int)fr.m, w = fr.w;
  const int32_t first = dp.sn_first[s];
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t % m, j = t / m;
    if (i >= j) A[t] = mix_get(fr, i, j);
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
    // trailing lower triangle: 8 columns x 32 rows of threads (blockDim = 256)
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int j = k + 1 + ty; j < m; j += 8) {
      const double ajk = A[k * m + j];
      for (int i = j + tx; i < m; i += 32) A[j * m + i] -= A[k * m + i] * ajk;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t % m, j = t / m;
    if (i >= j) mix_set(fr, i, j, A[t]);
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

// POTRF of the 64 x 64 diagonal tiles. A tile accumulates its assembled values and every update in FP64. On the
// factorization's critical path it is eliminated in FP32 (the tile rounded once to FP32) for the FP32 inverse
// of its factor, which the FP32 TRSM of the rows below and the FP32 solves use, like every other off-diagonal
// operand of this path. The factor of the tile itself (L_11, whose diagonal gives the log-determinant) is
// computed in FP64 from the FP64 tile by one batched launch over all diagonal tiles after the last level (the
// tiles are final once their block step has run, and no later step reads L_11); with GP_OPT_DIAG_FP32 the FP32
// elimination stores its L_11 instead. Right-looking, with the tile in registers: thread (tr, tc) of a 16 x 16 grid
// holds the entries (tr + 16 p, tc + 16 q), p, q < 4, of the tile and of X = inv(U), U the unit lower factor
// (A = U diag(d) U^T, U_ik = a_ik / d_k with a_ik column k as updated through column k - 1). The pivots
// d_k = L_kk^2 stay unscaled: column k enters through s_j = a_jk / d_k as a_ij -= a_ik s_j (j > k), and the
// same step eliminates below X's row k: X_ij -= U_ik X_kj (i > k, j <= k), the forward elimination of the
// identity. Two columns per step and one barrier per step (the step's fixed costs -- barrier, shared-memory
// round trip, reciprocal -- are what a column costs here): every thread reads columns k and k + 1 and rows k,
// k + 1 of X as published by their holders, forms column k + 1's and row k + 1's updates by column k itself, and
// applies both. Then L_ik = a_ik / sqrt(d_k), inv(L)_ij = X_ij / sqrt(d_i). X is eliminated in FP32 only.
constexpr int POTRF_THREADS = 256;

// 1 / d by Newton's iteration r <- r + r (1 - d r) from the hardware's FP32 approximate reciprocal: one step in
// FP32 (within about an ulp), two in FP64 (the error squares per step: about 2^-23 -> 2^-46 -> below an FP64 ulp).
// The pivots are normal numbers well inside the FP32 range (a tile's entries are covariances of order one).
__device__ __forceinline__ float rcp_seed(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}
__device__ __forceinline__ float recip_nr(float d) {
  const float r = rcp_seed(d);
  return fmaf(r, fmaf(-d, r, 1.f), r);
}
__device__ __forceinline__ double recip_nr(double d) {
  double r = (double)rcp_seed((float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  return fma(r, fma(-d, r, 1.0), r);
}
__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }

// The factorization of one tile by the CTA's 256 threads in arithmetic R: D the FP64 tile (in: the accumulated
// entries; out, if STORE_L: L), DI its FP32 inverse tile (out, if INV), bw its width, first the global column of
// its first column (a failed pivot records the smallest such column in *flag).
template <class R, bool INV, bool STORE_L>
__device__ __forceinline__ void potrf_tile(double* __restrict__ D, float* __restrict__ DI, int bw, int32_t first,
                                           int32_t* __restrict__ flag) {
  __shared__ R col[2][2][T];      // columns k, k + 1 after the updates of columns < k (double-buffered)
  __shared__ float xrow[2][2][T]; // rows k, k + 1 of X after the eliminations of rows < k (double-buffered)
  __shared__ R piv[T];            // pivots d_k
  __shared__ R rd[T];             // 1 / d_k
  __shared__ R sc[T];             // 1 / L_kk
  const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
  __syncthreads();   // an earlier call's readers of the shared arrays are done
  R a[4][4];
  float x[4][4];
  uint32_t own = 0;   // bit 4 p + q: entry (tr + 16 p, tc + 16 q) is in the lower triangle of the bw x bw tile
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int i = tr + 16 * p, j = tc + 16 * q;
      const bool in = j <= i && i < bw;
      a[p][q] = in ? (R)D[i * T + j] : R(0);
      x[p][q] = i == j ? 1.f : 0.f;
      own |= (in ? 1u : 0u) << (4 * p + q);
    }
  if (tc < 2) {
#pragma unroll
    for (int p = 0; p < 4; p++) col[0][tc][tr + 16 * p] = a[p][0];
  }
  if (tr < 2) {
#pragma unroll
    for (int q = 0; q < 4; q++) xrow[0][tr][tc + 16 * q] = x[0][q];
  }
  // Four phases of 16 columns: in phase m columns below 16 m are final, so only the tile's entries of column
  // groups q >= m and row groups p >= q take part (entries above the diagonal inside a diagonal block, and rows
  // past bw, are updated but never read), and only X's entries of row groups p >= m and column groups q <= m.
#pragma unroll
  for (int m = 0; m < 4; m++) {
    const int kend = min(16 * (m + 1), bw);
    for (int k = 16 * m; k < kend; k += 2) {
      __syncthreads();
      const int buf = k & 2 ? 1 : 0;
      const R* ca = col[buf][0];       // column k
      const R* cb = col[buf][1];       // column k + 1 (not yet updated by column k)
      const float* xa = xrow[buf][0];  // row k of X (final)
      const float* xb = xrow[buf][1];  // row k + 1 of X (not yet eliminated by row k)
      const bool two = k + 1 < bw;
      R d0 = ca[k];
      if (!(d0 > R(0))) {
        if (tid == 0) atomicMin(flag, first + k);
        d0 = R(1);
      }
      const R r0 = recip_nr(d0);
      const R s01 = two ? ca[k + 1] * r0 : R(0);   // U_{k+1, k}
      R d1 = two ? fma(-ca[k + 1], s01, cb[k + 1]) : R(1);
      if (!(d1 > R(0))) {
        if (tid == 0) atomicMin(flag, first + k + 1);
        d1 = R(1);
      }
      const R r1 = recip_nr(d1);
      if (tid == 0) {
        piv[k] = d0;
        rd[k] = r0;
        if (two) {
          piv[k + 1] = d1;
          rd[k + 1] = r1;
        }
      }
      R ci0[4], ci1[4], sj0[4], sj1[4];
      float xa4[4], xb4[4];
#pragma unroll
      for (int p = m; p < 4; p++) {
        ci0[p] = ca[tr + 16 * p];
        ci1[p] = fma(-ci0[p], s01, cb[tr + 16 * p]);
      }
#pragma unroll
      for (int q = m; q < 4; q++) {
        const R v = ca[tc + 16 * q];
        sj0[q] = v * r0;
        sj1[q] = fma(-v, s01, cb[tc + 16 * q]) * r1;
      }
      const float s01f = (float)s01;
      if (INV) {
#pragma unroll
        for (int q = 0; q <= m; q++) {
          xa4[q] = xa[tc + 16 * q];
          xb4[q] = fmaf(-s01f, xa4[q], xb[tc + 16 * q]);   // row k + 1 of X, eliminated by row k
        }
      }
      const int jm = tc + 16 * m;   // this thread's column of group m
      const int im = tr + 16 * m;   // this thread's row of group m
#pragma unroll
      for (int q = m; q < 4; q++)
#pragma unroll
        for (int p = q; p < 4; p++) {
          if (q > m || jm > k) a[p][q] = fma(-ci0[p], sj0[q], a[p][q]);
          if (two && (q > m || jm > k + 1)) a[p][q] = fma(-ci1[p], sj1[q], a[p][q]);
        }
      if (INV) {
#pragma unroll
        for (int p = m; p < 4; p++) {
          const float u0 = (float)(ci0[p] * r0), u1 = (float)(ci1[p] * r1);   // U_ik, U_i,k+1
#pragma unroll
          for (int q = 0; q <= m; q++) {
            if (p > m || im > k) x[p][q] = fmaf(-u0, xa4[q], x[p][q]);
            if (two && (p > m || im > k + 1)) x[p][q] = fmaf(-u1, xb4[q], x[p][q]);
          }
        }
      }
      const int k2 = k + 2;
      if (k2 < bw) {
        const int qb = k2 >> 4;
        if ((tc >> 1) == ((k2 & 15) >> 1)) {   // publish columns k + 2 and k + 3
          const int h = tc & 1;
          R* cn = col[buf ^ 1][h];
#pragma unroll
          for (int p = m; p < 4; p++) {
            const int i = tr + 16 * p;
            R v = a[p][m];
            if (m < 3 && qb == m + 1) v = a[p][m < 3 ? m + 1 : m];
            if (i >= k2 + h && i < bw) cn[i] = v;
          }
        }
        if (INV && (tr >> 1) == ((k2 & 15) >> 1)) {   // publish rows k + 2 and k + 3 of X
          const int h = tr & 1;
          float* xn = xrow[buf ^ 1][h];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            float v = x[m][q];
            if (m < 3 && qb == m + 1) v = x[m < 3 ? m + 1 : m][q];
            xn[tc + 16 * q] = v;
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid < T) sc[tid] = tid < bw ? sqrt_r(piv[tid]) * rd[tid] : R(1);   // sqrt(d) / d = 1 / L_kk
  __syncthreads();
#pragma unroll
  for (int p = 0; p < 4; p++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int i = tr + 16 * p, j = tc + 16 * q;
      float li = 0.f;
      if (own >> (4 * p + q) & 1) {
        if (STORE_L) D[i * T + j] = i == j ? (double)sqrt_r(piv[i]) : (double)(a[p][q] * sc[j]);
        li = x[p][q] * (float)sc[i];
      }
      if (INV) DI[i * T + j] = li;
    }
}

// The FP32 elimination of diagonal tile kb of each front of a step (its inverse; L_11 too if STORE_L).
template <bool STORE_L>
__global__ void __launch_bounds__(POTRF_THREADS) k_potrf_diag(const int32_t* __restrict__ fronts, int kb, DevPlan dp,
                                                              double* __restrict__ dg, int64_t DE,
                                                              int32_t* __restrict__ notpd, float* __restrict__ dinv32) {
  const int32_t s = fronts[blockIdx.x];
  const int b = blockIdx.y;
  const int64_t off = (int64_t)b * DE + dp.doff[s] + (int64_t)kb * T * T;
  potrf_tile<float, true, STORE_L>(dg + off, dinv32 + off, min(T, dp.w[s] - kb * T), dp.sn_first[s] + kb * T,
                                   notpd + b);
}

// L_11 of every diagonal tile of the large fronts in FP64 (tile t of the launch: front fronts[t], block kb[t];
// proposal blockIdx.y), from the FP64 tile as the factorization left it.
__global__ void __launch_bounds__(POTRF_THREADS) k_potrf_tiles64(const int32_t* __restrict__ fronts,
                                                                 const int32_t* __restrict__ kbs, DevPlan dp,
                                                                 double* __restrict__ dg, int64_t DE,
                                                                 int32_t* __restrict__ notpd) {
  const int32_t s = fronts[blockIdx.x], kb = kbs[blockIdx.x];
  const int b = blockIdx.y;
  const int64_t off = (int64_t)b * DE + dp.doff[s] + (int64_t)kb * T * T;
  potrf_tile<double, false, true>(dg + off, nullptr, min(T, dp.w[s] - kb * T), dp.sn_first[s] + kb * T, notpd + b);
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// FP32 TRSM of the rows below diagonal tile kb as a product with the inverse the POTRF left behind:
// X = B L^{-T}, X[r][j] = sum_{l <= j} B[r][l] Inv[j][l], one CTA of 256 threads per 64-row tile, each thread a
// 4 x 4 block of X (no dependency chains, unlike a column-by-column substitution). The L entries are written
// with the low parts of their TF32 pairs (tf32_lo), the tensor-core operands of the updates.
constexpr int TS = T + 4;   // transposed shared tiles, rows 16-byte aligned for vector reads

// dst[l][r] = src[r][l] for a 64 x 64 block at src (row stride lds), rows >= nr and columns >= nc read as zero;
// all 16 loads of a thread in flight at once.
__device__ __forceinline__ void load_tile_t(float* dst, const float* __restrict__ src, int64_t lds, int nr, int nc) {
  float v[16];
#pragma unroll
  for (int u = 0; u < 16; u++) {
    const int q = threadIdx.x + u * 256, i = q >> 6, j = q & 63;
    v[u] = (i < nr && j < nc) ? src[i * lds + j] : 0.f;
  }
#pragma unroll
  for (int u = 0; u < 16; u++) {
    const int q = threadIdx.x + u * 256, i = q >> 6, j = q & 63;
    dst[j * TS + i] = v[u];
  }
}

// acc[e][f] = sum_{l < kl} BT[l][tr + e] CT[l][tc + f] (thread: rows tr..tr+3 x columns tc..tc+3, one 16-byte
// read of each operand per l).
__device__ __forceinline__ void prod_tile(const float* BT, const float* CT, int kl, float (&acc)[4][4]) {
  const int tr = (threadIdx.x >> 4) * 4, tc = (threadIdx.x & 15) * 4;
#pragma unroll
  for (int e = 0; e < 4; e++)
#pragma unroll
    for (int f = 0; f < 4; f++) acc[e][f] = 0.f;
  for (int l = 0; l < kl; l++) {
    const float4 bq = *reinterpret_cast<const float4*>(BT + l * TS + tr);
    const float4 cq = *reinterpret_cast<const float4*>(CT + l * TS + tc);
    const float bv4[4] = {bq.x, bq.y, bq.z, bq.w}, cv4[4] = {cq.x, cq.y, cq.z, cq.w};
#pragma unroll
    for (int e = 0; e < 4; e++)
#pragma unroll
      for (int f = 0; f < 4; f++) acc[e][f] = fmaf(bv4[e], cv4[f], acc[e][f]);
  }
}

// The TF32 operand pair of an L entry x: the high part is x itself as the TF32 MMAs read it (they ignore the low
// 13 mantissa bits, i.e. truncate), the low part lo = x - trunc_tf32(x), exact in FP32 and rounded to TF32 here.
__device__ __forceinline__ float tf32_lo(float x) {
  return tf32_rn(x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u));
}

// The FP16 operand pairs (GP_OPT_SPLIT_F16) of proposal b are those of its L entries times 2^k, k =
// 12 - floor(E / 2) for max_i C_ii in [2^E, 2^(E+1)): |L_ij| <= sqrt(C_ii) < 2^(floor(E/2) + 1), so every scaled
// entry is below 2^13, well inside FP16's range (2^16). A pair holds its scaled entry y to within 2^-22 |y|, or
// 2^-25 absolute below 2^-3 (where the low part is subnormal), i.e. to 2^-38 of the bound. k is clamped to +-126
// (2^k and 2^-k are normal FP32 numbers).
__device__ __forceinline__ int f16_scale_exp(const unsigned long long* __restrict__ dmax, int b) {
  const int E = (int)((dmax[b] >> 52) & 0x7ff) - 1023;
  const int fl = E >= 0 ? E / 2 : -((1 - E) / 2);   // floor(E / 2)
  return min(126, max(-126, 12 - fl));
}
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }   // |k| <= 126

// The FP16 pair of a scaled entry y: hi = y rounded to FP16, lo = y - hi (exact in FP32) rounded to FP16.
__device__ __forceinline__ void f16_pair(float y, __half& hi, __half& lo) {
  hi = __float2half_rn(y);
  lo = __float2half_rn(y - __half2float(hi));
}

// Where store_x puts the tensor-core operands: dmax null for the TF32 pairs' low parts (the high part is the
// panel entry itself), else the FP16 pairs of proposal b (scale from dmax[b]) in a front region of m rows.
struct OpSplit {
  const unsigned long long* dmax;
  int b;
  int64_t m;
};

// Rows tr..tr+3 x columns tc..tc+3 of X into the front's panel at P + o (row stride ldw, o = row0 ldw + col0)
// and their tensor-core operands into the front's operand region L, for rows < nr and columns < bw.
// TF32 pairs: the low parts at L + o; the padding columns of a row (from the front's width up to ldw, inside the
// last 4-column group) get a zero low part: the region is reused by the fronts of other levels, and the updates
// read those columns (times a zero high part). FP16 pairs (op.dmax set): rows of ldh = ldw rounded up to 8
// halves, the high parts at (half*)L + row ldh + column and the low parts m ldh halves further; the padding
// columns up to ldh get zero pairs (the updates read them, and FP16 pairs have no zero high part elsewhere).
__device__ __forceinline__ void store_x(const float (&acc)[4][4], float* __restrict__ P, float* __restrict__ L,
                                        int64_t row0, int col0, int ldw, int nr, int bw, const OpSplit& op) {
  const int tr = (threadIdx.x >> 4) * 4, tc = (threadIdx.x & 15) * 4;
  if (op.dmax) {
    const float sc = pow2f(f16_scale_exp(op.dmax, op.b));
    const int ldh = (ldw + 7) & ~7, bw8 = (bw + 7) & ~7;
    __half* H = reinterpret_cast<__half*>(L);
    const int64_t lo_off = op.m * ldh;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int i = tr + e;
      if (i >= nr || tc >= bw8) continue;
      const int64_t o = row0 * ldw + col0 + (int64_t)i * ldw + tc;
      const int64_t oh = (row0 + i) * ldh + col0 + tc;   // 8-byte aligned: ldh, col0 and tc are x4
      __align__(8) __half hv[4], lv[4];
      if (tc + 4 <= bw) {
        *reinterpret_cast<float4*>(P + o) = make_float4(acc[e][0], acc[e][1], acc[e][2], acc[e][3]);
#pragma unroll
        for (int f = 0; f < 4; f++) f16_pair(acc[e][f] * sc, hv[f], lv[f]);
      } else {   // the front's last columns and the padding after them
#pragma unroll
        for (int f = 0; f < 4; f++) {
          hv[f] = __float2half_rn(0.f);
          lv[f] = hv[f];
          if (tc + f < bw) {
            P[o + f] = acc[e][f];
            f16_pair(acc[e][f] * sc, hv[f], lv[f]);
          }
        }
      }
      *reinterpret_cast<uint2*>(H + oh) = *reinterpret_cast<const uint2*>(hv);
      *reinterpret_cast<uint2*>(H + lo_off + oh) = *reinterpret_cast<const uint2*>(lv);
    }
    return;
  }
  const int64_t o0 = row0 * ldw + col0;
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int i = tr + e;
    if (i >= nr) continue;
    const int64_t o = o0 + (int64_t)i * ldw + tc;   // 16-byte aligned: ldw, the columns, tc and the offsets are x4
    if (tc + 4 <= bw) {
      const float4 x = make_float4(acc[e][0], acc[e][1], acc[e][2], acc[e][3]);
      *reinterpret_cast<float4*>(P + o) = x;
      *reinterpret_cast<float4*>(L + o) = make_float4(tf32_lo(x.x), tf32_lo(x.y), tf32_lo(x.z), tf32_lo(x.w));
    } else if (tc < bw) {   // the front's last columns (bw < 64 only at its last block) and the padding after them
      float lo[4];
#pragma unroll
      for (int f = 0; f < 4; f++) {
        lo[f] = 0.f;
        if (tc + f < bw) {
          P[o + f] = acc[e][f];
          lo[f] = tf32_lo(acc[e][f]);
        }
      }
      *reinterpret_cast<float4*>(L + o) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

// acc -> BT[l][r] (the transposed form prod_tile reads).
__device__ __forceinline__ void stash_t(const float (&acc)[4][4], float* BT) {
  const int tr = (threadIdx.x >> 4) * 4, tc = (threadIdx.x & 15) * 4;
#pragma unroll
  for (int e = 0; e < 4; e++)
#pragma unroll
    for (int f = 0; f < 4; f++) BT[(tc + f) * TS + tr + e] = acc[e][f];
}

__global__ void __launch_bounds__(256) k_trsm32(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre,
                                                int nfront, int kb, DevPlan dp, float* __restrict__ p32,
                                                float* __restrict__ opl, int64_t LOE,
                                                const float* __restrict__ dinv32, int64_t P32E, int64_t DE,
                                                const unsigned long long* __restrict__ dmax) {
  __shared__ __align__(16) float BsT[T * TS];   // BsT[l][r] = B[r][l]
  __shared__ __align__(16) float IsT[T * TS];   // IsT[l][j] = Inv[j][l]
  int64_t t = blockIdx.x;
  int fi = find_front(pre, nfront, t);
  int32_t s = fronts[fi];
  int b = blockIdx.y;
  const int64_t ob = (int64_t)b * P32E + dp.loff32[s];
  const float* DI = dinv32 + (int64_t)b * DE + dp.doff[s] + (int64_t)kb * T * T;
  const int w = dp.w[s], ldw = dp.ldw[s];
  const int64_t m = (int64_t)w + dp.r[s];
  const int c0 = kb * T, bw = min(T, w - c0), c1 = c0 + bw;
  const int64_t r0 = c1 + (t - pre[fi]) * T;
  const int nr = (int)imin64(T, m - r0);
  load_tile_t(IsT, DI, T, T, T);   // zero outside the lower bw x bw triangle
  load_tile_t(BsT, p32 + ob + r0 * ldw + c0, ldw, nr, bw);
  __syncthreads();
  float acc[4][4];
  prod_tile(BsT, IsT, bw, acc);
  store_x(acc, p32 + ob, opl + (int64_t)b * LOE + dp.lo_off[s], r0, c0, ldw, nr, bw, OpSplit{dmax, b, m});
}

// Block columns kb and kb + 1 at once (the mixed path's block steps in pairs, for an even group width): fronts
// [0, n2) of the list have block kb + 1. POTRF of tile kb; then, for those fronts, L_21 = A_21 inv(L_11)^T (the
// 64 rows of block kb + 1 in block column kb, with their TF32 pair), A_22 -= L_21 L_21^T into the FP64 tile of
// block kb + 1 (FP32 products, as the tensor-core updates give it), and the POTRF of that tile. One CTA per front.
template <bool STORE_L>
__global__ void __launch_bounds__(POTRF_THREADS) k_potrf_pair(const int32_t* __restrict__ fronts, int n2, int kb,
                                                              DevPlan dp, float* __restrict__ p32,
                                                              float* __restrict__ opl, int64_t LOE,
                                                              double* __restrict__ dg, float* __restrict__ dinv32,
                                                              int64_t P32E, int64_t DE, int32_t* __restrict__ notpd,
                                                              const unsigned long long* __restrict__ dmax) {
  __shared__ __align__(16) float BsT[T * TS];
  __shared__ __align__(16) float IsT[T * TS];
  const int fi = blockIdx.x;
  const int32_t s = fronts[fi];
  const int b = blockIdx.y;
  const int w = dp.w[s], ldw = dp.ldw[s];
  const int c0 = kb * T, bw1 = min(T, w - c0), c1 = c0 + bw1;
  const int64_t off = (int64_t)b * DE + dp.doff[s] + (int64_t)kb * T * T;
  const int32_t first = dp.sn_first[s] + c0;
  potrf_tile<float, true, STORE_L>(dg + off, dinv32 + off, bw1, first, notpd + b);
  if (fi >= n2) return;
  const int bw2 = min(T, w - c1);
  const int64_t ob = (int64_t)b * P32E + dp.loff32[s];
  __syncthreads();   // the inverse tile is in global memory, written by this CTA
  load_tile_t(IsT, dinv32 + off, T, T, T);
  load_tile_t(BsT, p32 + ob + (int64_t)c1 * ldw + c0, ldw, bw2, bw1);
  __syncthreads();
  float acc[4][4];
  prod_tile(BsT, IsT, bw1, acc);   // L_21
  store_x(acc, p32 + ob, opl + (int64_t)b * LOE + dp.lo_off[s], c1, c0, ldw, bw2, bw1,
          OpSplit{dmax, b, (int64_t)w + dp.r[s]});
  __syncthreads();
  stash_t(acc, BsT);   // BsT[l][r] = L_21[r][l]; rows past bw2 hold zeros
  __syncthreads();
  float g[4][4];
  prod_tile(BsT, BsT, bw1, g);   // g = L_21 L_21^T
  double* D2 = dg + off + T * T;
  const int tr = (threadIdx.x >> 4) * 4, tc = (threadIdx.x & 15) * 4;
#pragma unroll
  for (int e = 0; e < 4; e++)
#pragma unroll
    for (int f = 0; f < 4; f++) {
      const int i = tr + e, j = tc + f;
      if (j <= i && i < bw2) D2[i * T + j] -= (double)g[e][f];
    }
  potrf_tile<float, true, STORE_L>(D2, dinv32 + off + T * T, bw2, first + T, notpd + b);   // begins with a barrier
}

// The TRSM of a pair of block columns kb, kb + 1: for each 64-row tile below the pair (below block kb alone for
// fronts past n2), X_1 = B_1 inv(L_11)^T, B_2' = B_2 - X_1 L_21^T, X_2 = B_2' inv(L_22)^T.
__global__ void __launch_bounds__(256, 3) k_trsm32_pair(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre,
                                                     int nfront, int n2, int kb, DevPlan dp, float* __restrict__ p32,
                                                     float* __restrict__ opl, int64_t LOE,
                                                     const float* __restrict__ dinv32, int64_t P32E, int64_t DE,
                                                     const unsigned long long* __restrict__ dmax) {
  __shared__ __align__(16) float BsT[T * TS];
  __shared__ __align__(16) float IsT[T * TS];
  int64_t t = blockIdx.x;
  int fi = find_front(pre, nfront, t);
  int32_t s = fronts[fi];
  int b = blockIdx.y;
  const int64_t ob = (int64_t)b * P32E + dp.loff32[s];
  const float* DI = dinv32 + (int64_t)b * DE + dp.doff[s] + (int64_t)kb * T * T;
  const int w = dp.w[s], ldw = dp.ldw[s];
  const int64_t m = (int64_t)w + dp.r[s];
  const bool two = fi < n2;
  const int c0 = kb * T, bw1 = min(T, w - c0), c1 = c0 + bw1;
  const int bw2 = two ? min(T, w - c1) : 0, c2 = c1 + bw2;
  const int64_t r0 = c2 + (t - pre[fi]) * T;
  const int nr = (int)imin64(T, m - r0);
  float* P = p32 + ob;
  float* Lo = opl + (int64_t)b * LOE + dp.lo_off[s];
  load_tile_t(IsT, DI, T, T, T);
  load_tile_t(BsT, P + r0 * ldw + c0, ldw, nr, bw1);
  __syncthreads();
  float acc[4][4];
  prod_tile(BsT, IsT, bw1, acc);   // X_1
  store_x(acc, P, Lo, r0, c0, ldw, nr, bw1, OpSplit{dmax, b, m});
  if (!two) return;
  __syncthreads();
  stash_t(acc, BsT);                                            // BsT[l][r] = X_1[r][l]
  load_tile_t(IsT, P + (int64_t)c1 * ldw + c0, ldw, bw2, bw1);  // IsT[l][j] = L_21[j][l]
  __syncthreads();
  prod_tile(BsT, IsT, bw1, acc);   // X_1 L_21^T
  __syncthreads();
  load_tile_t(BsT, P + r0 * ldw + c1, ldw, nr, bw2);   // B_2
  load_tile_t(IsT, DI + T * T, T, T, T);              // inv(L_22)
  __syncthreads();
  {
    const int tr = (threadIdx.x >> 4) * 4, tc = (threadIdx.x & 15) * 4;
#pragma unroll
    for (int e = 0; e < 4; e++)
#pragma unroll
      for (int f = 0; f < 4; f++) acc[e][f] = BsT[(tc + f) * TS + tr + e] - acc[e][f];   // B_2' (zero past nr, bw2)
    __syncthreads();
    stash_t(acc, BsT);
  }
  __syncthreads();
  prod_tile(BsT, IsT, bw2, acc);   // X_2
  store_x(acc, P, Lo, r0, c1, ldw, nr, bw2, OpSplit{dmax, b, m});
}

// ---------------------------------------------------------------------------------------------------------
// Trailing updates on the tensor cores: F[i, j] -= sum_{l in K} L[i, l] L[j, l] over 128 x TN tiles, j <= i.
// Modes (block column kb = columns [c0, c1), in the (64 G)-column group [g0, gend), G = the plan's group):
//   3: left-looking, before the block's POTRF: rows >= c0 x the block's columns, 128 x 64 tiles, K = [g0, c0)
//      (the group's earlier blocks); 4: the same for block columns kb and kb + 1 at once, 128 x 128 tiles;
//   2: group end: rows/columns >= gend, tiles on and below the diagonal (the plan's tile width: 256 x 256 per
//      CTA pair, or 128 x 128), K = the whole group [g0, gend).
// The operands are a pair (hi, lo) per L entry, and each tile accumulates A_lo B_hi^T + A_hi B_lo^T + A_hi B_hi^T
// (the split of Ootomo and Yokota, 2022), FP32 accumulation:
//   F16 (the default): hi and lo are FP16, the entry times 2^k rounded and the remainder rounded (the pair holds
//     the entry to 2^-22 of it; the dropped lo lo term is at most 2^-22 of a product), both written by the TRSM
//     into the level's operand workspace; kind::f16 MMAs take 16 K per instruction, so an operand chunk of 128
//     bytes per row holds 64 K and a step costs half the instructions and half the operand bytes of TF32; the
//     epilogue scales the tile back by 2^-2k (exact).
//   TF32: hi is the FP32 panel entry itself, read through the TF32 MMA's truncation of the low 13 mantissa bits,
//     and lo the rounded remainder the TRSM writes into the workspace (the pair holds the entry to 2^-22 of it;
//     the dropped lo lo term, up to 2^-20 of a product with the truncated high part, is the larger error; one
//     TF32 pass keeps 11 significant bits).
// The wide tiles of mode 2 halve
// the MMA instructions and cut the operand bytes per flop by a quarter (the L2 -> SM operand stream is what
// bounds this kernel). Mode 2 runs in clusters of two CTAs on the tile pairs (rows 2p and 2p + 1 of 128, the same
// 256 columns) as one 256 x 256 CTA-pair MMA: each CTA loads its own 128 A rows and its half of the 256 B rows,
// so a stage costs each CTA two thirds of the operand bytes of an unpaired 128 x 256 tile and holds 64 KB, which
// leaves room for a three-stage ring; the even CTA issues the MMAs once both CTAs' bytes have landed on its
// barrier, and its commits free the stage and hand the accumulator halves to both CTAs.
//
// One persistent CTA per SM walks the launch's tiles (all fronts, all proposals) with three roles:
//   warp 0 (one lane): TMA loads of 128-row operand chunks (128 bytes per row: 64 FP16 or 32 TF32 entries) into
//                      a ring of 128-byte-swizzled tiles;
//   warp 1 (one lane): tcgen05.mma, 12 instructions per chunk, into one of two TMEM accumulators;
//   warps 2-9: the epilogue, which drains the other accumulator (tcgen05.ld -> swizzled 32 x 32 shared slab ->
//              coalesced read-modify-write of the front, 32 loads in flight per lane) while the next tile's
//              MMAs run.
// A tile whose A rows are a block of its B rows (on the diagonal) loads only B. Waits are bounded; a wait that
// runs out sets *err and the CTA winds down.
constexpr int UW_THREADS = 320;
constexpr int UW_EPI = 8 * 32 * 32 * 4;  // a 32 x 32 FP32 slab per epilogue warp
constexpr int UW_BAR = 256;
template <int TN, bool PAIR = false>
struct UW {
  static constexpr int STAGES = TN == 256 && !PAIR ? 2 : 3;
  static constexpr int OPA = 128 * 32 * 4;        // A operand chunk: 128 rows x 32 FP32 (128-byte rows)
  // B rows held by this CTA (whole 128-row boxes; N = TN are used; a CTA pair holds half of B in each CTA)
  static constexpr int BROWS = PAIR ? TN / 2 : (TN < 128 ? 128 : TN);
  static constexpr int OPB = BROWS * 32 * 4;      // B operand chunk
  static constexpr int STAGE = 2 * OPA + 2 * OPB; // A_hi, A_lo, B_hi, B_lo
  static constexpr int SMEM = STAGES * STAGE + UW_EPI + UW_BAR + 1024;
  static constexpr uint32_t TMEM_COLS = 2 * TN;   // two FP32 accumulators of TN columns
};

// Bit mask of the integers below x, 0 <= x <= 32.
__device__ __forceinline__ uint32_t below32(int x) { return x >= 32 ? 0xffffffffu : ((1u << x) - 1u); }

struct UTile {
  int32_t s, slot;
  int b, w, r, ldw, K, kc;
  int64_t m, i0, j0, jlim;
};

// Tile tt of a launch: proposal, front (prefix search), then its position. Mode 2 with TN = 256 (paired): tile
// pair p (rows 2p and 2p + 1 of 128) holds p + 1 tiles of 256 columns; CTA `rank` of the pair takes row 2p + rank.
// Modes 3 and 4 may cover part of the strip's 128-row tiles (mode + 8 part): part 0 all of them, part 1 only the
// first (the rows of the step's diagonal tiles, one tile per front: pre is not read), part 2 the others (pre
// counts a front's tiles after its first).
template <int TN, bool PAIR>
__device__ __forceinline__ UTile decode_tile(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre,
                                             int nfront, int64_t total, int kb, int mode_part, int group,
                                             const DevPlan& dp, const int32_t* __restrict__ slot_of, int64_t tt,
                                             int rank) {
  UTile u;
  const int mode = mode_part & 7, part = mode_part >> 3;
  u.b = (int)(tt / total);
  const int64_t t = tt - (int64_t)u.b * total;
  const int fi = part == 1 ? (int)t : find_front(pre, nfront, t);
  u.s = fronts[fi];
  u.slot = slot_of[u.s];
  u.w = dp.w[u.s];
  u.r = dp.r[u.s];
  u.ldw = dp.ldw[u.s];
  u.m = (int64_t)u.w + u.r;
  const int c0 = kb * T, bw = min(T, u.w - c0), c1 = c0 + bw;
  const int g0 = (kb / group) * group * T, gend = min(g0 + group * T, u.w);
  (void)bw;
  const int64_t loc = part == 1 ? 0 : t - pre[fi];
  int64_t I, J, base;
  if (mode >= 3) {   // 4: the strip of block columns kb and kb + 1 (the block steps in pairs)
    I = part == 2 ? loc + 1 : loc;
    J = 0;
    base = c0;
    u.jlim = mode == 4 ? min(c0 + 2 * T, u.w) : c1;
    u.K = c0 - g0;
    u.kc = g0;
  } else {
    if (TN == 128) {
      I = (int64_t)((sqrtf(8.f * (float)loc + 1.f) - 1.f) * 0.5f);
      while ((I + 1) * (I + 2) / 2 <= loc) I++;
      while (I * (I + 1) / 2 > loc) I--;
      J = loc - I * (I + 1) / 2;
    } else if (PAIR) {
      int64_t p = (int64_t)((sqrtf(8.f * (float)loc + 1.f) - 1.f) * 0.5f);
      while ((p + 1) * (p + 2) / 2 <= loc) p++;
      while (p * (p + 1) / 2 > loc) p--;
      J = loc - p * (p + 1) / 2;
      I = 2 * p + rank;
    } else {
      int64_t p = (int64_t)((sqrtf(4.f * (float)loc + 1.f) - 1.f) * 0.5f);
      while ((p + 1) * (p + 2) <= loc) p++;
      while (p * (p + 1) > loc) p--;
      const int64_t rem = loc - p * (p + 1);
      I = 2 * p + (rem > p ? 1 : 0);
      J = rem > p ? rem - (p + 1) : rem;
    }
    base = gend;
    u.jlim = u.m;
    u.K = gend - g0;
    u.kc = g0;
  }
  u.i0 = base + I * 128;
  u.j0 = base + J * TN;
  return u;
}

template <int TN, bool PAIR, bool F16>
__global__ void __launch_bounds__(UW_THREADS, 1)
    k_update_ws(const int32_t* __restrict__ fronts, const int64_t* __restrict__ pre, int nfront, int64_t total,
                int64_t ntiles, int kb, int mode, int group, DevPlan dp, const uint8_t* __restrict__ tmaps,
                const int32_t* __restrict__ slot_of, float* __restrict__ p32, double* __restrict__ dg,
                float* __restrict__ u32, int64_t P32E, int64_t DE, int64_t UE, int32_t* __restrict__ err,
                tcg::WaitLimit lim, const unsigned long long* __restrict__ dmax) {
  using C = UW<TN, PAIR>;
  constexpr int NS = C::STAGES;
  constexpr int KCH = F16 ? 64 : 32;   // K per operand chunk: one 128-byte row of FP16 or of TF32 entries
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* epi = reinterpret_cast<float*>(smem + NS * C::STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NS * C::STAGE + UW_EPI);
  uint64_t* full = bars;                // [NS] operands landed
  uint64_t* empty = bars + NS;          // [NS] MMAs done reading
  uint64_t* tfull = bars + 2 * NS;      // [2] accumulator complete
  uint64_t* tempty = bars + 2 * NS + 2; // [2] accumulator drained
  uint64_t* drain = bars + 2 * NS + 4;    // the MMA issuer's last commit (winding down)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  uint32_t* issued_s = tslot + 2;         // operand chunks this CTA's producer issued
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = tcg::smem_u32(smem);
  if (threadIdx.x == 0) {
    for (int q = 0; q < NS; q++) {
      tcg::mbar_init(&full[q], 1);
      tcg::mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; q++) {
      tcg::mbar_init(&tfull[q], 1);
      tcg::mbar_init(&tempty[q], PAIR ? 16 : 8);   // paired: both CTAs' epilogue warps drain the even CTA's MMAs
    }
    tcg::mbar_init(drain, 1);
    *issued_s = 0;
    *abort_flag = *(volatile int32_t*)err != 0;   // an earlier launch of this factorization failed: skip the tiles
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    if (PAIR) tcg::tmem_alloc2(tslot, C::TMEM_COLS);
    else tcg::tmem_alloc(tslot, C::TMEM_COLS);
  }
  tcg::tc_fence_before();
  if (PAIR) tcg::cluster_sync();   // the peer's barriers are initialised before anything reaches them
  else __syncthreads();
  tcg::tc_fence_after();
  const uint32_t tmem = *tslot;
  const int rank = PAIR ? (int)tcg::cluster_ctarank() : 0;
  const int64_t t_first = PAIR ? (int64_t)tcg::cluster_id_x() : (int64_t)blockIdx.x;
  const int64_t t_step = PAIR ? (int64_t)tcg::cluster_count_x() : (int64_t)gridDim.x;
  auto fail = [&]() {
    *abort_flag = 1;
    atomicExch(err, 1);
  };
  // which 128-row block of this CTA's B holds the A rows (-1: none, A is loaded)
  auto a_in_b = [rank](const UTile& u) -> int {
    if (PAIR) return u.i0 == u.j0 + 128 * rank ? 0 : -1;   // a diagonal pair: each CTA's A half is its B half
    if (u.i0 == u.j0) return 0;
    if (TN == 256 && u.i0 == u.j0 + 128) return 1;
    return -1;
  };

  if (warp == 0) {
    if (lane == 0) {   // TMA producer
      uint32_t st = 0, ph = 0, issued = 0;
      for (int64_t tt = t_first; tt < ntiles && !*abort_flag; tt += t_step) {
        const UTile u = decode_tile<TN, PAIR>(fronts, pre, nfront, total, kb, mode, group, dp, slot_of, tt, rank);
        const uint8_t* mh = tmaps + (int64_t)u.slot * 256;
        const uint8_t* ml = mh + 128;
        tcg::tmap_acquire(mh);
        tcg::tmap_acquire(ml);
        const bool shared_a = a_in_b(u) >= 0;
        const int nch = (u.K + KCH - 1) / KCH;
        for (int c = 0; c < nch; c++) {
          if (!tcg::mbar_wait(&empty[st], ph ^ 1, lim)) {
            fail();
            break;
          }
          const uint32_t sa = sbase + st * C::STAGE, sb = sa + 2 * C::OPA;
          const int x = u.kc + c * KCH;
          if (PAIR) {   // this CTA's A rows and half of B, counted on the even CTA's barrier
            const uint32_t fb = tcg::mapa_shared(tcg::smem_u32(&full[st]), 0);
            if (rank == 0) tcg::mbar_arrive_expect_tx(&full[st], 2 * ((shared_a ? 0 : 2 * C::OPA) + 2 * C::OPB));
            if (!shared_a) {
              tcg::tma_load_3d_2sm(sa, mh, x, (int)u.i0, u.b, fb);
              tcg::tma_load_3d_2sm(sa + C::OPA, ml, x, (int)u.i0, u.b, fb);
            }
            tcg::tma_load_3d_2sm(sb, mh, x, (int)u.j0 + 128 * rank, u.b, fb);
            tcg::tma_load_3d_2sm(sb + C::OPB, ml, x, (int)u.j0 + 128 * rank, u.b, fb);
          } else {
            tcg::mbar_arrive_expect_tx(&full[st], (shared_a ? 0 : 2 * C::OPA) + 2 * C::OPB);
            if (!shared_a) {
              tcg::tma_load_3d(sa, mh, x, (int)u.i0, u.b, &full[st]);
              tcg::tma_load_3d(sa + C::OPA, ml, x, (int)u.i0, u.b, &full[st]);
            }
#pragma unroll
            for (int hb = 0; hb < C::BROWS / 128; hb++) {
              tcg::tma_load_3d(sb + hb * C::OPA, mh, x, (int)u.j0 + 128 * hb, u.b, &full[st]);
              tcg::tma_load_3d(sb + C::OPB + hb * C::OPA, ml, x, (int)u.j0 + 128 * hb, u.b, &full[st]);
            }
          }
          ++issued;
          if (++st == NS) {
            st = 0;
            ph ^= 1;
          }
        }
      }
      *issued_s = issued;
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {   // MMA issuer (paired: the even CTA, for both)
      const uint32_t idesc = F16 ? tcg::idesc_f16(PAIR ? 256 : 128, TN) : tcg::idesc_tf32(PAIR ? 256 : 128, TN);
      uint32_t st = 0, ph = 0, acc = 0, aph = 0;
      for (int64_t tt = t_first; tt < ntiles && !*abort_flag; tt += t_step) {
        const UTile u = decode_tile<TN, PAIR>(fronts, pre, nfront, total, kb, mode, group, dp, slot_of, tt, rank);
        const int ab = a_in_b(u);
        const int nch = (u.K + KCH - 1) / KCH;
        if (!tcg::mbar_wait(&tempty[acc], aph ^ 1, lim)) {
          fail();
          break;
        }
        tcg::tc_fence_after();
        const uint32_t d = tmem + acc * TN;
        bool ok = true;
        for (int c = 0; c < nch; c++) {
          if (!tcg::mbar_wait(&full[st], ph, lim)) {
            ok = false;
            break;
          }
          tcg::tc_fence_after();
          const uint32_t bH = sbase + st * C::STAGE + 2 * C::OPA, bL = bH + C::OPB;
          const uint32_t aH = ab >= 0 ? bH + ab * C::OPA : bH - 2 * C::OPA;
          const uint32_t aL = ab >= 0 ? bL + ab * C::OPA : bH - C::OPA;
#pragma unroll
          for (int kk = 0; kk < 4; kk++) {
            const uint32_t o = kk * 32;
            const uint64_t ah = tcg::smem_desc_sw128(aH + o), al = tcg::smem_desc_sw128(aL + o);
            const uint64_t bh = tcg::smem_desc_sw128(bH + o), bl = tcg::smem_desc_sw128(bL + o);
            if (PAIR) {
              tcg::mma_2sm<F16>(d, al, bh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
              tcg::mma_2sm<F16>(d, ah, bl, idesc, 1u);
              tcg::mma_2sm<F16>(d, ah, bh, idesc, 1u);
            } else {
              tcg::mma_1sm<F16>(d, al, bh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
              tcg::mma_1sm<F16>(d, ah, bl, idesc, 1u);
              tcg::mma_1sm<F16>(d, ah, bh, idesc, 1u);
            }
          }
          if (PAIR) tcg::mma_commit2_mc(&empty[st], 3);
          else tcg::mma_commit(&empty[st]);
          if (++st == NS) {
            st = 0;
            ph ^= 1;
          }
        }
        if (!ok) {
          fail();
          break;
        }
        if (PAIR) tcg::mma_commit2_mc(&tfull[acc], 3);
        else tcg::mma_commit(&tfull[acc]);
        if (++acc == 2) {
          acc = 0;
          aph ^= 1;
        }
      }
    }
  } else {   // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns [h TN / 2, (h + 1) TN / 2)
    constexpr int NSL = TN / 64;   // 32-column slabs per warp
    const int q = warp & 3, h = (warp - 2) >> 2;
    float* slab = epi + (warp - 2) * 1024;
    uint32_t acc = 0, aph = 0;
    for (int64_t tt = t_first; tt < ntiles && !*abort_flag; tt += t_step) {
      const UTile u = decode_tile<TN, PAIR>(fronts, pre, nfront, total, kb, mode, group, dp, slot_of, tt, rank);
      float* P = p32 + (int64_t)u.b * P32E + dp.loff32[u.s];
      float* U = u32 + (int64_t)u.b * UE + dp.uoff[u.s];
      double* D = dg + (int64_t)u.b * DE + dp.doff[u.s];
      // FP16 pairs: the accumulator holds 2^2k L_I L_J^T; 2^-k twice scales it back exactly
      const float isc = F16 ? pow2f(-f16_scale_exp(dmax, u.b)) : 1.f;
      const int64_t ib = u.i0 + q * 32;
      const int64_t jc = u.j0 + h * (TN / 2);
      // while the tile's MMAs run: pull this warp's target rows (NSL x 128 bytes each) into L2
      {
        const int64_t i = ib + lane;
        if (i < u.m) {
#pragma unroll
          for (int sl = 0; sl < NSL; sl++) {
            const int64_t j = jc + sl * 32;
            if (j <= i && j < u.jlim) {
              const float* pa = j < u.w ? P + i * u.ldw + j : U + (i - u.w) * u.r + (j - u.w);
              asm volatile("prefetch.global.L2 [%0];" ::"l"(pa));
            }
          }
        }
      }
      if (!tcg::mbar_wait(&tfull[acc], aph, lim)) {
        fail();
        break;
      }
      tcg::tc_fence_after();
      const uint32_t ta = tmem + acc * TN + ((uint32_t)(q * 32) << 16) + h * (TN / 2);
      for (int sl = 0; sl < NSL; sl++) {
        {
          float v[32];
          tcg::tmem_ld32(ta + sl * 32, v);
          if (sl == NSL - 1) {   // this warp's part of the accumulator has been read
            tcg::tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if (PAIR) tcg::mbar_arrive_cluster(tcg::mapa_shared(tcg::smem_u32(&tempty[acc]), 0));
              else tcg::mbar_arrive(&tempty[acc]);
            }
          }
          __syncwarp();
          if (F16) {
#pragma unroll
            for (int e = 0; e < 32; e++) v[e] = (v[e] * isc) * isc;
          }
#pragma unroll
          for (int e = 0; e < 32; e++) slab[lane * 32 + (e ^ lane)] = v[e];
        }
        __syncwarp();
        const int64_t j = jc + sl * 32 + lane;
        const bool colok = j < u.jlim;
        float* cb;
        int64_t cs;
        if (j < u.w) {
          cb = P + j;
          cs = u.ldw;
        } else {
          cb = U + (j - u.w) - (int64_t)u.w * u.r;
          cs = u.r;
        }
        // rows of this lane's column in the warp's 32: [lo, hi) = lower triangle inside the front (and inside
        // the update's column range), minus [dlo, dhi) = rows whose entry lives in an FP64 diagonal tile;
        // all 32 loads in flight before the first store
        int lo = 32, hi = 0, dlo = 0, dhi = 0;
        if (colok) {
          lo = (int)imin64(32, j > ib ? j - ib : 0);
          hi = (int)imin64(32, u.m > ib ? u.m - ib : 0);
          if (j < u.w) {
            const int64_t b0 = j & ~(int64_t)63, b1 = imin64(b0 + 64, u.w);
            dlo = (int)imin64(32, b0 > ib ? b0 - ib : 0);
            dhi = (int)imin64(32, b1 > ib ? b1 - ib : 0);
          }
        }
        const uint32_t okm = lo < hi ? (below32(hi) & ~below32(lo)) & ~(below32(dhi) & ~below32(dlo)) : 0u;
        float* base = cb + ib * cs;   // dereferenced only at valid rows
        const int csi = (int)cs;
        float old[32];
#pragma unroll
        for (int rr = 0; rr < 32; rr++) old[rr] = (okm >> rr & 1) ? base[rr * csi] : 0.f;
#pragma unroll
        for (int rr = 0; rr < 32; rr++)
          if (okm >> rr & 1) base[rr * csi] = old[rr] - slab[rr * 32 + (lane ^ rr)];
        const int d0 = max(dlo, lo), d1 = min(dhi, hi);
        for (int rr = d0; rr < d1; rr++) {   // entries of the FP64 diagonal tiles
          const int64_t i = ib + rr;
          D[(i >> 6) * (T * T) + (i & 63) * T + (j & 63)] -= (double)slab[rr * 32 + (lane ^ rr)];
        }
        __syncwarp();
      }
      if (++acc == 2) {
        acc = 0;
        aph ^= 1;
      }
    }
  }
  // Winding down (waits that return at once after a normal run): every role has left its loop and no producer
  // issues any more. Before tensor memory is freed and the CTAs exit, wait for every operand copy issued into
  // either CTA's shared memory and for every MMA issued, so that nothing still targets them. A CTA pair's copies
  // all complete on the even CTA's barriers; chunks one producer issued and the other did not (an aborted run) are
  // balanced there first: the odd CTA's bytes expected but never sent are completed without a copy, bytes sent
  // but never expected are expected now.
  tcg::tc_fence_before();
  if (PAIR) tcg::cluster_sync();
  else __syncthreads();
  if (warp == 0 && lane == 0 && rank == 0) {
    uint32_t n_hi = *issued_s;
    if (PAIR) {
      const uint32_t n_e = *issued_s;
      const uint32_t n_o = tcg::ld_shared_cluster_u32(tcg::mapa_shared(tcg::smem_u32(issued_s), 1));
      const uint32_t n_lo = min(n_e, n_o);
      n_hi = max(n_e, n_o);
      uint32_t c = 0;
      for (int64_t tt = t_first; tt < ntiles && c < n_hi && n_lo < n_hi; tt += t_step) {
        const UTile u = decode_tile<TN, PAIR>(fronts, pre, nfront, total, kb, mode, group, dp, slot_of, tt, 1);
        const uint32_t ob = (u.i0 == u.j0 + 128 ? 0 : 2 * C::OPA) + 2 * C::OPB;   // the odd CTA's bytes
        const int nch = (u.K + KCH - 1) / KCH;
        for (int q = 0; q < nch && c < n_hi; q++, c++) {
          if (c < n_lo) continue;
          if (n_e > n_o) tcg::mbar_complete_tx(&full[c % NS], ob);
          else tcg::mbar_arrive_expect_tx(&full[c % NS], ob);
        }
      }
    }
    for (uint32_t c = n_hi > (uint32_t)NS ? n_hi - NS : 0; c < n_hi; c++)
      if (!tcg::mbar_wait(&full[c % NS], (c / NS) & 1)) fail();
  }
  if (warp == 1 && lane == 0 && rank == 0) {   // the MMAs issued so far have completed once this commit arrives
    if (PAIR) tcg::mma_commit2_mc(drain, 1);
    else tcg::mma_commit(drain);
    if (!tcg::mbar_wait(drain, 0)) fail();
  }
  tcg::tc_fence_before();
  if (PAIR) tcg::cluster_sync();   // no copy, multicast or remote arrive may still target either CTA
  else __syncthreads();
  if (warp == 1) {
    tcg::tc_fence_after();
    if (PAIR) tcg::tmem_dealloc2(tmem, C::TMEM_COLS);
    else tcg::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

std::once_flag g_attrs_once;
template <bool F16>
void set_update_attrs() {
  GP_CUDA(cudaFuncSetAttribute(k_update_ws<GP_TN_LEFT, false, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               UW<GP_TN_LEFT>::SMEM));
  GP_CUDA(cudaFuncSetAttribute(k_update_ws<128, false, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               UW<128>::SMEM));
  GP_CUDA(cudaFuncSetAttribute(k_update_ws<256, true, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               UW<256, true>::SMEM));
}
void set_attrs() {   // once per process (contexts may run on several host threads)
  std::call_once(g_attrs_once, [] {
    GP_CUDA(cudaFuncSetAttribute(k_small_front32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 GP_SMALL_M * GP_SMALL_M * (int)sizeof(double)));
    set_update_attrs<false>();
    set_update_attrs<true>();
  });
}

// max_i C_ii of each proposal (grid: columns x proposals), for the FP16 pairs' scale: the diagonal entries sit in
// the FP64 diagonal tiles once the values are in; the maximum of non-negative doubles is that of their bit
// patterns as unsigned integers (atomicMax after a warp maximum). Non-positive or NaN entries count as 0 (the
// factorization reports them).
__global__ void __launch_bounds__(256) k_diag_max(DevPlan dp, int64_t n, const double* __restrict__ dg, int64_t DE,
                                                  unsigned long long* __restrict__ dmax) {
  const int b = blockIdx.y;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (j < n) {
    const int32_t s = dp.sn_of_col[j];
    const int64_t i = j - dp.sn_first[s];
    const double d = dg[(int64_t)b * DE + dp.doff[s] + (i >> 6) * (T * T) + (i & 63) * (T + 1)];
    v = d > 0.0 ? (unsigned long long)__double_as_longlong(d) : 0ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(dmax + b, v);
}

__global__ void k_fill_i32(int32_t* p, int n, int32_t v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// dest32[e]: FP32 panel offset (row-major) or DIAG_FLAG | diagonal-tile offset for lower entries, else -1.
__global__ void k_dest32(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n,
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
    int64_t lr;
    if (pi < f + w) {
      lr = pi - f;
    } else {
      const int32_t* R = dp.frows + dp.frow_off[s] + w;
      int lo = 0, hi = r;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (R[mid] < pi) lo = mid + 1;
        else hi = mid;
      }
      if (lo == r || R[lo] != pi) {
        dest[e] = -1;
        continue;
      }
      lr = w + lo;
    }
    int64_t lc = pj - f;
    if (lr < w && (lr >> 6) == (lc >> 6))
      dest[e] = DIAG_FLAG | (dp.doff[s] + (lr >> 6) * (T * T) + (lr & 63) * T + (lc & 63));
    else
      dest[e] = dp.loff32[s] + lr * dp.ldw[s] + lc;
  }
}

}  // namespace

void set_attrs_mixed() { set_attrs(); }

void compute_dest_map_mixed(gp_ctx* ctx, gp_pointset* ps) {
  ps->dest32 = dalloc<int64_t>(ctx, ps->bufs, ps->nnz);
  k_dest32<<<grid_for(ps->n * 32, 256), 256, 0, ctx->stream>>>(ps->rowptr, ps->col, ps->n, ps->pinv, ps->dp,
                                                               ps->dest32);
  GP_CHECK_LAUNCH(ctx);
}

namespace {
// One update launch over `total` tiles per proposal of the fronts of a list: mode 3 on 128 x 64 tiles, mode 2
// with 256-column tiles on clusters of two CTAs, mode 2 with 128-column tiles and mode 4 on 128 x 128 tiles.
template <bool F16>
void launch_update_t(gp_ctx* ctx, gp_factor_t* f, int64_t total, const int32_t* fronts, const int64_t* pre,
                     int32_t nfront, int32_t kb, int mode_part, cudaStream_t st, int reserve) {
  const SymPlan& sp = f->ps->sp;
  const int mode = mode_part & 7;
  const int64_t ntiles = total * f->B;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, std::max(1, ctx->nsm - reserve));
  if (mode == 3) {
    k_update_ws<GP_TN_LEFT, false, F16><<<grid, UW_THREADS, UW<GP_TN_LEFT>::SMEM, st>>>(
        fronts, pre, nfront, total, ntiles, kb, mode_part, sp.group, f->ps->dp, f->op_maps, f->op_slot, f->panels32,
        f->diag, f->upd32, sp.panel32_entries, sp.diag_entries, sp.update_entries, f->tiles_err, f->wait_lim,
        f->op_dmax);
  } else if (mode == 2 && sp.tn_group == 256) {   // clusters of two CTAs, one tile pair each
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * std::min<int64_t>(ntiles, std::max(1, (ctx->nsm - reserve) / 2))));
    cfg.blockDim = dim3(UW_THREADS);
    cfg.dynamicSmemBytes = UW<256, true>::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GP_CUDA(cudaLaunchKernelEx(&cfg, k_update_ws<256, true, F16>, fronts, pre, nfront, total, ntiles, kb, mode_part,
                               sp.group, f->ps->dp, (const uint8_t*)f->op_maps, (const int32_t*)f->op_slot,
                               f->panels32, f->diag, f->upd32, sp.panel32_entries, sp.diag_entries,
                               sp.update_entries, f->tiles_err, f->wait_lim,
                               (const unsigned long long*)f->op_dmax));
  } else {
    k_update_ws<128, false, F16><<<grid, UW_THREADS, UW<128>::SMEM, st>>>(
        fronts, pre, nfront, total, ntiles, kb, mode_part, sp.group, f->ps->dp, f->op_maps, f->op_slot, f->panels32,
        f->diag, f->upd32, sp.panel32_entries, sp.diag_entries, sp.update_entries, f->tiles_err, f->wait_lim,
        f->op_dmax);
  }
  GP_CHECK_LAUNCH(ctx);
}
// mode_part: the mode, plus 8 x the part of the strip for modes 3 and 4 (decode_tile); st: the stream; reserve:
// SMs the launch leaves free (for a concurrent launch on another stream).
void launch_update(gp_ctx* ctx, gp_factor_t* f, int64_t total, const int32_t* fronts, const int64_t* pre,
                   int32_t nfront, int32_t kb, int mode_part, cudaStream_t st = nullptr, int reserve = 0) {
  if (!st) st = ctx->stream;
  if (f->op_f16) launch_update_t<true>(ctx, f, total, fronts, pre, nfront, kb, mode_part, st, reserve);
  else launch_update_t<false>(ctx, f, total, fronts, pre, nfront, kb, mode_part, st, reserve);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    GP_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    GP_REQUIRE(q == cudaDriverEntryPointSuccess && p, "cuTensorMapEncodeTiled is not available from the driver");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
}  // namespace

// The operand split stores only the low half of each TF32 pair and lets the MMA read the high half from the FP32
// panel, which is exact only if kind::tf32 truncates an FP32 operand (ignores its low 13 mantissa bits). One CTA
// checks that once per device: a 128 x 32 x 8 MMA of A rows that each repeat one value (so the tile's 128-byte
// swizzle does not matter) by B = 1 gives 8 x the value as the tensor core reads it. Row 0 holds 1 + 0.75 ulp
// (rounding would give 1 + 1 ulp), row 1 its negative, row 2 1 + 1.5 ulp (a tie), the rest 1. The wait is
// bounded; *out = 1 when every row matches the truncated value, 0 when one does not, -1 when the wait ran out.
__global__ void __launch_bounds__(128) k_tf32_trunc_check(int32_t* __restrict__ out) {
  extern __shared__ __align__(1024) uint8_t cs_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)cs_raw + 1023) & ~(uintptr_t)1023);
  float* A = reinterpret_cast<float*>(sm);            // 128 rows x 32 FP32
  float* Bt = reinterpret_cast<float*>(sm + 16384);   // 32 rows x 32 FP32
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int bad;
  const int t = threadIdx.x;
  const float a = t == 0 ? __uint_as_float(0x3F801800u) : t == 1 ? __uint_as_float(0xBF801800u)
                : t == 2 ? __uint_as_float(0x3F803000u) : 1.f;
  for (int k = 0; k < 32; k++) A[t * 32 + k] = a;
  if (t < 32)
    for (int k = 0; k < 32; k++) Bt[t * 32 + k] = 1.f;
  if (t == 0) {
    tcg::mbar_init(&bar, 1);
    bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (t < 32) tcg::tmem_alloc(&tslot, 32);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // the tiles are visible to the tensor core
  tcg::tc_fence_before();
  __syncthreads();
  tcg::tc_fence_after();
  const uint32_t tm = tslot;
  if (t == 0) {
    tcg::mma_tf32(tm, tcg::smem_desc_sw128(tcg::smem_u32(A)), tcg::smem_desc_sw128(tcg::smem_u32(Bt)),
                  tcg::idesc_tf32(128, 32), 0);
    tcg::mma_commit(&bar);
  }
  __syncwarp();
  const bool ok = __syncthreads_and(tcg::mbar_wait(&bar, 0)) != 0;   // the same answer in every thread
  if (ok) {
    tcg::tc_fence_after();
    float v[32];
    tcg::tmem_ld32(tm + ((uint32_t)((t >> 5) * 32) << 16), v);
    const float want = 8.f * __uint_as_float(__float_as_uint(a) & 0xFFFFE000u);
    if (v[0] != want || v[31] != want) atomicExch(&bad, 1);
  }
  tcg::tc_fence_before();
  __syncthreads();
  if (t < 32) {
    if (ok) tcg::tmem_dealloc(tm, 32);
    else {   // the MMA may still be in flight: wait once more before freeing its accumulator
      const bool ok2 = tcg::mbar_wait(&bar, 0);
      tcg::tmem_dealloc(tm, 32);
      (void)ok2;
    }
  }
  if (t == 0) *out = !ok ? -1 : (bad ? 0 : 1);
}

// Runs k_tf32_trunc_check once per device (the first mixed factor on it; synchronises ctx's stream then) and
// refuses the mixed path on a GPU whose TF32 MMAs do not truncate.
void require_tf32_truncation(gp_ctx* ctx) {
  static std::mutex mu;
  static int state[64] = {};   // per device: 0 unknown, 1 truncates
  std::lock_guard<std::mutex> lock(mu);
  GP_REQUIRE(ctx->device >= 0 && ctx->device < 64, "device index out of range");
  if (state[ctx->device] == 1) return;
  constexpr int smem = 16384 + 4096 + 1024;
  GP_CUDA(cudaFuncSetAttribute(k_tf32_trunc_check, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int32_t* d_out = nullptr;
  GP_CUDA(cudaMallocAsync((void**)&d_out, sizeof(int32_t), ctx->stream));
  int32_t h = 0;
  cudaError_t e = cudaSuccess;
  k_tf32_trunc_check<<<1, 128, smem, ctx->stream>>>(d_out);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_out, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFreeAsync(d_out, ctx->stream);
  GP_CUDA(e);
  if (h == -1) throw GpError{GP_ERR_TIMEOUT, "the TF32 truncation check's MMA did not complete"};
  if (h != 1)
    throw GpError{GP_ERR_STATE, "this GPU's TF32 MMAs do not truncate FP32 operands, which the mixed path's "
                                "operand split relies on"};
  state[ctx->device] = 1;
}

// Tensor maps of the operand pair of every large front (those with tensor-core updates under any blocking of
// plan_mixed_updates): per front two 3-D maps (columns x rows x proposals) with 128-byte boxes of 128 rows and the
// 128-byte swizzle; rows past the front and columns past the row length read as zeros. TF32 pairs: the high
// part over the FP32 panel and the low part over the front's region of op_lo (rows of ldw FP32, boxes of 32
// columns). FP16 pairs: both over the front's region (rows of ldh halves, high parts first, boxes of 64
// columns). op_slot[s] gives the front's map pair (-1 for none).
void build_update_maps(gp_ctx* ctx, gp_factor_t* f) {
  if (!f->op_f16) require_tf32_truncation(ctx);
  const SymPlan& sp = f->ps->sp;
  const int64_t ns = (int64_t)sp.sn_w.size();
  std::vector<int32_t> slot(ns, -1);
  std::vector<int32_t> order;
  for (int32_t s : sp.large_fronts)
    if (slot[s] < 0) {
      slot[s] = (int32_t)order.size();
      order.push_back(s);
    }
  const size_t nmaps = std::max<size_t>(order.size(), 1);
  std::vector<CUtensorMap> maps(2 * nmaps);
  std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
  auto enc = tensor_map_encoder();
  GP_REQUIRE(sp.panel32_entries % 4 == 0, "FP32 panel stride must be a multiple of 16 bytes");
  for (size_t k = 0; k < order.size(); k++) {
    const int32_t s = order[k];
    const int64_t ldw = sp.sn_ldw[s], m = (int64_t)sp.sn_w[s] + sp.sn_r[s];
    GP_REQUIRE(ldw % 4 == 0 && sp.sn_loff32[s] % 4 == 0, "FP32 panel rows must start on 16-byte boundaries");
    GP_REQUIRE(sp.sn_lo_off[s] % 4 == 0 && sp.lo_entries % 4 == 0, "low-part rows must start on 16-byte boundaries");
    const int64_t ldh = (ldw + 7) / 8 * 8;
    GP_REQUIRE(sp.sn_lo_off[s] % 8 == 0, "operand regions must start on 32-byte boundaries");
    for (int part = 0; part < 2; part++) {
      CUresult r;
      cuuint32_t es[3] = {1, 1, 1};
      if (f->op_f16) {   // halves: high parts at the region's start, low parts m x ldh halves further
        void* base = reinterpret_cast<uint16_t*>(f->op_lo + sp.sn_lo_off[s]) + part * m * ldh;
        cuuint64_t dims[3] = {(cuuint64_t)ldh, (cuuint64_t)m, (cuuint64_t)f->B};
        cuuint64_t strides[2] = {(cuuint64_t)ldh * 2, (cuuint64_t)sp.lo_entries * 4};
        cuuint32_t box[3] = {64, 128, 1};
        r = enc(&maps[2 * k + part], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      } else {
        float* base = part == 0 ? f->panels32 + sp.sn_loff32[s] : f->op_lo + sp.sn_lo_off[s];
        const int64_t pstride = part == 0 ? sp.panel32_entries : sp.lo_entries;
        cuuint64_t dims[3] = {(cuuint64_t)ldw, (cuuint64_t)m, (cuuint64_t)f->B};
        cuuint64_t strides[2] = {(cuuint64_t)ldw * 4, (cuuint64_t)pstride * 4};
        cuuint32_t box[3] = {32, 128, 1};
        r = enc(&maps[2 * k + part], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      }
      GP_REQUIRE(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled rejected an operand map");
    }
  }
  f->op_maps = dalloc<uint8_t>(ctx, f->bufs, maps.size() * sizeof(CUtensorMap));
  f->op_slot = dalloc<int32_t>(ctx, f->bufs, (size_t)ns + 1);
  GP_CUDA(cudaMemcpyAsync(f->op_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                          ctx->stream));
  GP_CUDA(cudaMemcpyAsync(f->op_slot, slot.data(), (size_t)ns * sizeof(int32_t), cudaMemcpyHostToDevice,
                          ctx->stream));
  GP_CUDA(cudaStreamSynchronize(ctx->stream));   // the host vectors go out of scope
}

void factor_run_mixed(gp_ctx* ctx, gp_factor_t* f) {
  gp_pointset* ps = f->ps;
  const SymPlan& sp = ps->sp;
  const DevPlan& dp = ps->dp;
  cudaStream_t st = ctx->stream;
  set_attrs();
  const int B = f->B;
  const int64_t P32E = sp.panel32_entries, DE = sp.diag_entries, UE = sp.update_entries, LOE = sp.lo_entries;
  values_run_mixed(ctx, f);   // A3, A4 into the FP32 panels and FP64 tiles (zeroed first)
  k_fill_i32<<<grid_for(B, 128), 128, 0, st>>>(f->notpd, B, INT_MAX);
  GP_CHECK_LAUNCH(ctx);
  const unsigned long long* dmax = f->op_f16 ? f->op_dmax : nullptr;   // FP16 pairs: their scale, from max C_ii
  if (dmax) {
    GP_CUDA(cudaMemsetAsync(f->op_dmax, 0, sizeof(unsigned long long) * B, st));
    ProfScope ps_(ctx, KC_VALUES);
    k_diag_max<<<dim3(grid_for(ps->n, 256), B), 256, 0, st>>>(dp, ps->n, f->diag, DE, f->op_dmax);
    GP_CHECK_LAUNCH(ctx);
  }
  GP_CUDA(cudaMemsetAsync(f->tiles_err, 0, sizeof(int32_t), st));
  ProfLevelScope pls_(ctx);
  // Work off the level chain goes to the context's side stream (not while profiling, which times every launch on
  // the main stream): zeroing level L + 1's update matrices once level L's extend-add has read the matrices they
  // may reuse, and the FP64 L_11 of level L's diagonal tiles once its block steps are done (nothing later touches
  // them). The main stream waits for a level's zeroing before its extend-add, and for everything at the end.
  const bool overlap = ctx->side != nullptr && !ctx->prof;
  const bool tiles64 = !f->diag_fp32 && !sp.large_fronts.empty();
  auto zero_level = [&](int32_t L, cudaStream_t s) {
    const SymPlan::Level& lz = sp.levels[L];
    if (lz.zero_n == 0) return;
    ProfScope ps_(ctx, KC_EXTEND_ADD);   // the update matrices this level's fronts will fill
    k_zero_updates32<<<dim3((unsigned)lz.zero_n, B), EA_THREADS, 0, s>>>(dp.zero_tab + lz.zero_off, dp, f->upd32, UE);
    GP_CHECK_LAUNCH(ctx);
  };
  auto fork = [&]() {
    GP_CUDA(cudaEventRecord(ctx->ev_fork, st));
    GP_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  };
  if (overlap && sp.nlevels > 0) {
    fork();
    zero_level(0, ctx->side);
    GP_CUDA(cudaEventRecord(ctx->ev_join, ctx->side));
  }
  // The left-looking update of a step (mode 3, or 4 for a pair of block columns). With a third stream (explicit
  // streams, not while profiling) and at most half the SMs taken by the step's fronts, the strip's first 128-row
  // tile of each front -- the rows of the step's diagonal tiles, which the POTRF factors -- runs on the main
  // stream, and the other tiles on side2 beside the POTRF, on all SMs but those the POTRF's CTAs take; the caller
  // joins side2 back before the TRSM (returns true). Otherwise one launch on the main stream. Each tile computes
  // the same sums either way.
  auto left_update = [&](const SymPlan::StepLaunch& sl, double flops, int mode) -> bool {
    const int32_t* lf = dp.upd_fronts + sl.left_off;
    const int reserve = sl.nfront * B;
    if (!overlap || !ctx->side2 || sl.lrest_total == 0 || reserve > ctx->nsm / 2) {
      ProfScope ps_(ctx, KC_UPDATE_LEFT, B * flops);
      launch_update(ctx, f, sl.left_total, lf, dp.upd_pre + sl.left_pre_off, sl.n_left, sl.kb, mode);
      return false;
    }
    GP_CUDA(cudaEventRecord(ctx->ev_fork2, st));
    GP_CUDA(cudaStreamWaitEvent(ctx->side2, ctx->ev_fork2, 0));
    launch_update(ctx, f, sl.lrest_total, lf, dp.upd_pre + sl.lrest_pre_off, sl.n_left, sl.kb, mode + 16, ctx->side2,
                  reserve);
    GP_CUDA(cudaEventRecord(ctx->ev_join2, ctx->side2));
    launch_update(ctx, f, sl.n_left, lf, dp.upd_pre + sl.left_pre_off, sl.n_left, sl.kb, mode + 8);
    return true;
  };
  for (int32_t L = 0; L < sp.nlevels; L++) {
    const SymPlan::Level& lv = sp.levels[L];
    ctx->prof_level = L;
    if (overlap) GP_CUDA(cudaStreamWaitEvent(st, ctx->ev_join, 0));   // this level's zeroing
    else zero_level(L, st);
    for (const auto& ea : lv.ea32) {
      ProfScope ps_(ctx, KC_EXTEND_ADD);
      k_extend_add32<<<dim3((unsigned)ea.ncta, B), EA_THREADS, 0, st>>>(dp.ea32_tab + ea.tab_off, dp, f->panels32,
                                                                        f->diag, f->upd32, P32E, DE, UE);
      GP_CHECK_LAUNCH(ctx);
    }
    if (overlap && L + 1 < sp.nlevels) {   // the next level's zeroing, beside this level's steps
      fork();
      zero_level(L + 1, ctx->side);
      GP_CUDA(cudaEventRecord(ctx->ev_join, ctx->side));
    }
    if (lv.nsmall > 0) {
      int32_t mmax = 1;
      for (int32_t q = 0; q < lv.nsmall; q++) {
        int32_t s = sp.small_list[lv.small_off + q];
        mmax = std::max(mmax, sp.sn_w[s] + sp.sn_r[s]);
      }
      ProfScope ps_(ctx, KC_FRONT_SMALL);
      k_small_front32<<<dim3(lv.nsmall, B), 256, (size_t)mmax * mmax * sizeof(double), st>>>(
          dp.small_list + lv.small_off, dp, f->panels32, f->diag, f->upd32, P32E, DE, UE, f->notpd);
      GP_CHECK_LAUNCH(ctx);
    }
    for (size_t q = 0; q < lv.steps.size();) {
      const auto& stp = lv.steps[q];
      const int32_t* fronts = dp.large_fronts + stp.fr_off;
      if (sp.group % 2 == 0 && q + 1 < lv.steps.size()) {   // block columns kb and kb + 1 (never across a group)
        const auto& st2 = lv.steps[q + 1];
        const bool joined = stp.left_total > 0 && left_update(stp, stp.left2_flops, 4);
        {
          ProfScope ps_(ctx, KC_POTRF, B * (stp.potrf_flops + st2.potrf_flops));
          auto kp = f->diag_fp32 ? k_potrf_pair<true> : k_potrf_pair<false>;
          kp<<<dim3(stp.nfront, B), POTRF_THREADS, 0, st>>>(fronts, st2.nfront, stp.kb, dp, f->panels32, f->op_lo,
                                                            LOE, f->diag, f->dinv32, P32E, DE, f->notpd, dmax);
          GP_CHECK_LAUNCH(ctx);
        }
        if (joined) GP_CUDA(cudaStreamWaitEvent(st, ctx->ev_join2, 0));   // the rows below, for the TRSM
        if (stp.pair_total > 0) {
          ProfScope ps_(ctx, KC_TRSM, B * (stp.trsm_flops + st2.trsm_flops));
          k_trsm32_pair<<<dim3((unsigned)stp.pair_total, B), 256, 0, st>>>(
              fronts, dp.pair_pre + stp.pair_pre_off, stp.nfront, st2.nfront, stp.kb, dp, f->panels32, f->op_lo,
              LOE, f->dinv32, P32E, DE, dmax);
          GP_CHECK_LAUNCH(ctx);
        }
        for (const auto* sg : {&stp, &st2})
          if (sg->group_total > 0) {   // fronts whose group ends at kb (their last block) or at kb + 1
            ProfScope ps_(ctx, KC_UPDATE, B * sg->group_flops);
            launch_update(ctx, f, sg->group_total, dp.upd_fronts + sg->group_off, dp.upd_pre + sg->group_pre_off,
                          sg->n_group, sg->kb, 2);
          }
        q += 2;
        continue;
      }
      q += 1;
      const int64_t* pre_tr = dp.step_pre + stp.pre_off;
      // this block column from the earlier blocks of its group
      const bool joined = stp.left_total > 0 && left_update(stp, stp.left_flops, 3);
      {
        ProfScope ps_(ctx, KC_POTRF, B * stp.potrf_flops);
        auto kd = f->diag_fp32 ? k_potrf_diag<true> : k_potrf_diag<false>;
        kd<<<dim3(stp.nfront, B), POTRF_THREADS, 0, st>>>(fronts, stp.kb, dp, f->diag, DE, f->notpd, f->dinv32);
        GP_CHECK_LAUNCH(ctx);
      }
      if (joined) GP_CUDA(cudaStreamWaitEvent(st, ctx->ev_join2, 0));
      if (stp.trsm_total > 0) {
        ProfScope ps_(ctx, KC_TRSM, B * stp.trsm_flops);
        k_trsm32<<<dim3((unsigned)stp.trsm_total, B), 256, 0, st>>>(fronts, pre_tr, stp.nfront, stp.kb, dp,
                                                                    f->panels32, f->op_lo, LOE, f->dinv32, P32E,
                                                                    DE, dmax);
        GP_CHECK_LAUNCH(ctx);
      }
      if (stp.group_total > 0) {   // fronts whose group ends here: the deferred update with K = group width
        ProfScope ps_(ctx, KC_UPDATE, B * stp.group_flops);
        launch_update(ctx, f, stp.group_total, dp.upd_fronts + stp.group_off, dp.upd_pre + stp.group_pre_off,
                      stp.n_group, stp.kb, 2);
      }
    }
    const auto& ll = sp.level_large[L];
    if (overlap && tiles64 && ll.count > 0) {   // this level's diagonal tiles are final: their FP64 L_11 beside
      fork();                                   // the next levels
      k_potrf_tiles64<<<dim3((unsigned)ll.count, B), POTRF_THREADS, 0, ctx->side>>>(
          dp.large_fronts + ll.off, dp.large_kb + ll.off, dp, f->diag, DE, f->notpd);
      GP_CHECK_LAUNCH(ctx);
    }
  }
  ctx->prof_level = -1;   // one launch over all levels
  if (overlap) {
    GP_CUDA(cudaEventRecord(ctx->ev_join, ctx->side));
    GP_CUDA(cudaStreamWaitEvent(st, ctx->ev_join, 0));
  } else if (tiles64) {   // L_11 of every diagonal tile in FP64
    ProfScope ps_(ctx, KC_POTRF);
    k_potrf_tiles64<<<dim3((unsigned)sp.large_fronts.size(), B), POTRF_THREADS, 0, st>>>(
        dp.large_fronts, dp.large_kb, dp, f->diag, DE, f->notpd);
    GP_CHECK_LAUNCH(ctx);
  }
}
