// assemble.cu -- steps A1 (cell list), A2 (support pattern of C_z as CSR) and A5 (nested dissection).
//
// A1: u = x / core_radius per coordinate (IEEE division), cell coordinates c_k = floor(u_k) - floor(min u_k),
//     cell key c_0 + nc_0 (c_1 + nc_1 c_2), points sorted stably by (key, index), dense cell ranges.
// A2: for each point, the 3^d neighbouring cells are scanned and a pair enters the pattern iff
//     q^2 = sum_k (u_ik - u_jk)^2 < 1, evaluated left to right with separately rounded products and sums
//     (no FMA contraction), so the pattern is exactly symmetric and reproducible. This is the support of the
//     compact core C_core (Sec. 2, C_y = C_core x C_sparse): outside it C_z is zero for every theta.
//     Rows are sorted ascending by original index (warp-per-row rank counting).
// A5: the separator rule of the build (the paper does no factorization at scale): recursively, a set of more
//     than 64 points is sorted along the coordinate of largest extent (ties: lowest coordinate) by (u_k, index),
//     split at floor(|V|/2); points of the lower half with a pattern neighbour in the upper half form the
//     separator S; the order is [order(L \ S), order(R), S in sort order]; sets of at most 64 points are
//     ordered by (cell key, index). Every level of the recursion runs as one set of device passes.
#include <algorithm>
#include <cmath>

#include "gp_internal.cuh"

namespace {

__device__ __forceinline__ uint64_t ord_key(double x) {
  if (x == 0.0) x = 0.0;   // one key for +0 and -0
  uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_key_inv(uint64_t k) {
  uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

__global__ void k_scale(const double* __restrict__ X, int64_t n, int d, double r0, double r1, double r2,
                        double* __restrict__ U, unsigned long long* __restrict__ mnmx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double rr[3] = {r0, r1, r2};
  uint64_t lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0, 0, 0};
  if (i < n) {
    for (int k = 0; k < d; k++) {
      double u = X[i * d + k] / rr[k];
      U[i * d + k] = u;
      uint64_t kk = ord_key(u);
      lo[k] = kk;
      hi[k] = kk;
    }
  }
  for (int k = 0; k < d; k++) {
    for (int o = 16; o > 0; o >>= 1) {
      uint64_t a = __shfl_xor_sync(0xffffffffu, lo[k], o);
      uint64_t b = __shfl_xor_sync(0xffffffffu, hi[k], o);
      lo[k] = a < lo[k] ? a : lo[k];
      hi[k] = b > hi[k] ? b : hi[k];
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&mnmx[2 * k], (unsigned long long)lo[k]);
      atomicMax(&mnmx[2 * k + 1], (unsigned long long)hi[k]);
    }
  }
}

__global__ void k_decode_minmax(const unsigned long long* __restrict__ mnmx, int d, double* __restrict__ out) {
  int k = threadIdx.x;
  if (k < 2 * d) out[k] = ord_key_inv(mnmx[k]);
}

struct Grid {
  int d;
  long long c0[3], nc[3];
};

__device__ __forceinline__ long long cell_coord(double u, long long c0) { return (long long)floor(u) - c0; }

__global__ void k_cell_keys(const double* __restrict__ U, int64_t n, Grid g, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long kk = 0;
  for (int k = g.d - 1; k >= 0; k--) kk = kk * g.nc[k] + cell_coord(U[i * g.d + k], g.c0[k]);
  keys[i] = (uint64_t)kk;
  vals[i] = (uint32_t)i;
}

__global__ void k_cell_start(const uint64_t* __restrict__ skeys, int64_t n, int64_t ncells,
                             int64_t* __restrict__ cell_start) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > n) return;
  int64_t prev = (p == 0) ? -1 : (int64_t)skeys[p - 1];
  int64_t cur = (p == n) ? ncells : (int64_t)skeys[p];
  for (int64_t c = prev + 1; c <= cur; c++) cell_start[c] = p;
}

__global__ void k_gather_sorted(const double* __restrict__ U, const uint32_t* __restrict__ perm, int64_t n, int d,
                                double* __restrict__ Us, int32_t* __restrict__ cell_perm,
                                const uint64_t* __restrict__ skeys, int64_t* __restrict__ key_of) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint32_t i = perm[p];
  cell_perm[p] = (int32_t)i;
  for (int k = 0; k < d; k++) Us[p * d + k] = U[(int64_t)i * d + k];
  key_of[i] = (int64_t)skeys[p];
}

// q^2 < 1 with separately rounded operations in coordinate order (matches the oracle's predicate).
__device__ __forceinline__ bool in_support(const double* ui, const double* uj, int d) {
  double s = 0.0;
  for (int k = 0; k < d; k++) {
    double dk = __dsub_rn(ui[k], uj[k]);
    s = __dadd_rn(s, __dmul_rn(dk, dk));
  }
  return s < 1.0;
}

// Count (FILL=false) or write (FILL=true) each point's pattern row by scanning its 3^d neighbouring cells.
template <bool FILL>
__global__ void k_pattern(const double* __restrict__ Us, const int32_t* __restrict__ cell_perm,
                          const int64_t* __restrict__ cell_start, int64_t n, Grid g,
                          int64_t* __restrict__ rowcnt, const int64_t* __restrict__ rowptr,
                          int32_t* __restrict__ col) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int d = g.d;
  double ui[3] = {0, 0, 0};
  long long ci[3] = {0, 0, 0};
  for (int k = 0; k < d; k++) {
    ui[k] = Us[p * d + k];
    ci[k] = cell_coord(ui[k], g.c0[k]);
  }
  int32_t i = cell_perm[p];
  int64_t out = FILL ? rowptr[i] : 0;
  int64_t cnt = 0;
  int nb = 1;
  for (int k = 0; k < d; k++) nb *= 3;
  for (int t = 0; t < nb; t++) {
    long long cc[3] = {0, 0, 0};
    int tt = t;
    bool ok = true;
    for (int k = 0; k < d; k++) {
      cc[k] = ci[k] + (tt % 3) - 1;
      tt /= 3;
      if (cc[k] < 0 || cc[k] >= g.nc[k]) ok = false;
    }
    if (!ok) continue;
    long long cell = 0;
    for (int k = d - 1; k >= 0; k--) cell = cell * g.nc[k] + cc[k];
    for (int64_t q = cell_start[cell]; q < cell_start[cell + 1]; q++) {
      double uj[3] = {0, 0, 0};
      for (int k = 0; k < d; k++) uj[k] = Us[q * d + k];
      if (in_support(ui, uj, d)) {
        if (FILL) col[out + cnt] = cell_perm[q];
        cnt++;
      }
    }
  }
  if (!FILL) rowcnt[i] = cnt;
}

// The support of C_sparse (the pattern with a non-compact core). Bit i of fam[k]: point k lies inside the support of
// bump family i, sum over the leading bd coordinates of (x_c - h_c)^2 < r^2 for one of the family's bumps (Eq.
// bumpFcn), each operation rounded separately in coordinate order.
__global__ void k_family_mask(const double* __restrict__ X, int64_t n, int d, const double* __restrict__ h,
                              const double* __restrict__ r, int n1, int n2, int bd, uint32_t* __restrict__ fam) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  uint32_t m = 0;
  for (int i = 0; i < n1; i++)
    for (int j = 0; j < n2; j++) {
      const int ij = i * n2 + j;
      double s = 0.0;
      for (int c = 0; c < bd; c++) {
        const double dc = __dsub_rn(X[k * d + c], h[(int64_t)ij * bd + c]);
        s = __dadd_rn(s, __dmul_rn(dc, dc));
      }
      if (s < __dmul_rn(r[ij], r[ij])) m |= 1u << i;
    }
  fam[k] = m;
}

// Row i of the support of C_sparse: j with q0^2 < 1 (u = x / r0) or sharing a bump family with i. A warp per row,
// lanes over 32 consecutive j at a time, so the row comes out ascending (ballot prefix for the fill).
template <bool FILL>
__global__ void k_pattern_support(const double* __restrict__ U, const uint32_t* __restrict__ fam, int64_t n, int d,
                                  int64_t* __restrict__ rowcnt, const int64_t* __restrict__ rowptr,
                                  int32_t* __restrict__ col) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double ui[3] = {0, 0, 0};
  for (int k = 0; k < d; k++) ui[k] = U[i * d + k];
  const uint32_t mi = fam[i];
  const int64_t out = FILL ? rowptr[i] : 0;
  int64_t cnt = 0;
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    const int64_t j = j0 + lane;
    bool p = false;
    if (j < n) p = (mi & fam[j]) != 0 || in_support(ui, U + j * d, d);
    const uint32_t bal = __ballot_sync(0xffffffffu, p);
    if (FILL && p) col[out + cnt + __popc(bal & ((1u << lane) - 1u))] = (int32_t)j;
    cnt += __popc(bal);
  }
  if (!FILL && lane == 0) rowcnt[i] = cnt;
}

// Sort each CSR row ascending: warp per row, every element's destination is the count of smaller entries.
__global__ void k_sort_rows(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ in, int64_t n,
                            int32_t* __restrict__ out) {
  int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  int64_t a = rowptr[row], b = rowptr[row + 1];
  for (int64_t e = a + lane; e < b; e += 32) {
    int32_t v = in[e];
    int64_t rank = 0;
    for (int64_t f = a; f < b; f++) rank += in[f] < v;
    out[a + rank] = v;
  }
}

// ---------------------------------------------------------------------------------------- nested dissection
__global__ void k_axis_keys(const double* __restrict__ U, int64_t n, int d, int k, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = ord_key(U[i * d + k]);
  vals[i] = (uint32_t)i;
}

__global__ void k_rank_of(const uint32_t* __restrict__ vals, int64_t n, int32_t* __restrict__ rank) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) rank[vals[p]] = (int32_t)p;
}

__global__ void k_seg_extent(const int32_t* __restrict__ act, const int32_t* __restrict__ act_seg, int64_t tot,
                             const double* __restrict__ U, int d, unsigned long long* __restrict__ smm) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = p < tot;
  int32_t v = valid ? act[p] : 0, s = valid ? act_seg[p] : -1;
  // lanes of one segment reduce in registers first (the top levels hold one huge segment)
  int32_t s0 = __shfl_sync(0xffffffffu, s, 0);
  bool uniform = __all_sync(0xffffffffu, s == s0 || !valid) && s0 >= 0;
  for (int k = 0; k < d; k++) {
    unsigned long long lo = ~0ull, hi = 0ull;
    if (valid) lo = hi = ord_key(U[(int64_t)v * d + k]);
    if (uniform) {
      for (int o = 16; o > 0; o >>= 1) {
        unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
        unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
      }
      if ((threadIdx.x & 31) == 0) {
        atomicMin(&smm[(int64_t)s0 * 6 + 2 * k], lo);
        atomicMax(&smm[(int64_t)s0 * 6 + 2 * k + 1], hi);
      }
    } else if (valid) {
      atomicMin(&smm[(int64_t)s * 6 + 2 * k], lo);
      atomicMax(&smm[(int64_t)s * 6 + 2 * k + 1], hi);
    }
  }
}

__global__ void k_seg_axis(const unsigned long long* __restrict__ smm, int64_t nseg, int d,
                           int32_t* __restrict__ axis) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  int best = 0;
  double bext = -1.0;
  for (int k = 0; k < d; k++) {
    double ext = ord_key_inv(smm[s * 6 + 2 * k + 1]) - ord_key_inv(smm[s * 6 + 2 * k]);
    if (ext > bext) {
      bext = ext;
      best = k;
    }
  }
  axis[s] = best;
}

__global__ void k_seg_sortkeys(const int32_t* __restrict__ act, const int32_t* __restrict__ act_seg, int64_t tot,
                               const int32_t* __restrict__ axis, const int32_t* __restrict__ rank, int64_t n,
                               uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= tot) return;
  int32_t v = act[p], s = act_seg[p];
  keys[p] = (uint64_t)s * (uint64_t)n + (uint64_t)rank[(int64_t)axis[s] * n + v];
  vals[p] = (uint32_t)v;
}

__global__ void k_mark_sides(const uint32_t* __restrict__ sorted, const int32_t* __restrict__ act_seg, int64_t tot,
                             const int64_t* __restrict__ seg_start, const int64_t* __restrict__ seg_size,
                             const int64_t* __restrict__ seg_gid, int32_t* __restrict__ act,
                             int64_t* __restrict__ vgid, int8_t* __restrict__ vside) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= tot) return;
  int32_t v = (int32_t)sorted[p];
  int32_t s = act_seg[p];
  act[p] = v;
  int64_t local = p - seg_start[s];
  vgid[v] = seg_gid[s];
  vside[v] = local < seg_size[s] / 2 ? 0 : 1;
}

__global__ void k_sep_flags(const int32_t* __restrict__ act, const int32_t* __restrict__ act_seg, int64_t tot,
                            const int64_t* __restrict__ seg_start, const int64_t* __restrict__ seg_size,
                            const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const int64_t* __restrict__ vgid, const int8_t* __restrict__ vside,
                            int64_t* __restrict__ sflag, int64_t* __restrict__ lflag) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > tot) return;
  if (p == tot) {   // trailing zero so that the exclusive scans end with the totals
    sflag[p] = 0;
    lflag[p] = 0;
    return;
  }
  int32_t v = act[p], s = act_seg[p];
  int64_t local = p - seg_start[s];
  int64_t fs = 0, fl = 0;
  if (local < seg_size[s] / 2) {
    int64_t g = vgid[v];
    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
      int32_t w = col[e];
      if (vgid[w] == g && vside[w] == 1) {
        fs = 1;
        break;
      }
    }
    fl = 1 - fs;
  }
  sflag[p] = fs;
  lflag[p] = fl;
}

// Per segment: separator size and size of L \ S from the scanned flags.
__global__ void k_seg_counts(const int64_t* __restrict__ sidx, const int64_t* __restrict__ lidx, int64_t nseg,
                             const int64_t* __restrict__ seg_start, const int64_t* __restrict__ seg_size,
                             int64_t* __restrict__ cnt) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  int64_t a = seg_start[s], b = a + seg_size[s];
  cnt[2 * s] = sidx[b] - sidx[a];
  cnt[2 * s + 1] = lidx[b] - lidx[a];
}

// Route every active point: separator points to their final slots; L \ S and R points to the next level's
// active list (child larger than a leaf) or to the leaf list.
__global__ void k_route(const int32_t* __restrict__ act, const int32_t* __restrict__ act_seg, int64_t tot,
                        const int64_t* __restrict__ seg_start, const int64_t* __restrict__ seg_size,
                        const int64_t* __restrict__ seg_out, const int64_t* __restrict__ sidx,
                        const int64_t* __restrict__ lidx, const int64_t* __restrict__ cnt,
                        const int64_t* __restrict__ dstA, const int64_t* __restrict__ dstB,
                        const int32_t* __restrict__ segA, const int32_t* __restrict__ segB,
                        int32_t* __restrict__ perm, int32_t* __restrict__ nact, int32_t* __restrict__ nact_seg,
                        int32_t* __restrict__ leafv) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= tot) return;
  int32_t v = act[p], s = act_seg[p];
  int64_t st = seg_start[s], m = seg_size[s], local = p - st, half = m / 2;
  int64_t nS = cnt[2 * s];
  if (local < half) {
    if (sidx[p + 1] != sidx[p]) {   // separator point
      perm[seg_out[s] + m - nS + (sidx[p] - sidx[st])] = v;
      return;
    }
    int64_t idx = lidx[p] - lidx[st];
    if (segA[s] >= 0) {
      nact[dstA[s] + idx] = v;
      nact_seg[dstA[s] + idx] = segA[s];
    } else {
      leafv[dstA[s] + idx] = v;
    }
  } else {
    int64_t idx = local - half;
    if (segB[s] >= 0) {
      nact[dstB[s] + idx] = v;
      nact_seg[dstB[s] + idx] = segB[s];
    } else {
      leafv[dstB[s] + idx] = v;
    }
  }
}

// Leaves (<= 64 points): order by (cell key, index), warp per leaf, rank by counting.
__global__ void k_leaf_order(const int32_t* __restrict__ leafv, const int64_t* __restrict__ leaf_start,
                             const int64_t* __restrict__ leaf_out, int64_t nleaf, const int64_t* __restrict__ key_of,
                             int32_t* __restrict__ perm) {
  int64_t L = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (L >= nleaf) return;
  int64_t a = leaf_start[L], b = leaf_start[L + 1];
  for (int64_t e = a + lane; e < b; e += 32) {
    int32_t v = leafv[e];
    int64_t kv = key_of[v];
    int64_t rank = 0;
    for (int64_t f = a; f < b; f++) {
      int32_t w = leafv[f];
      int64_t kw = key_of[w];
      rank += (kw < kv) || (kw == kv && w < v);
    }
    perm[leaf_out[L] + rank] = v;
  }
}

__global__ void k_inverse(const int32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ pinv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pinv[perm[i]] = (int32_t)i;
}

int bits_for(uint64_t maxval) {
  int b = 0;
  while (b < 64 && (maxval >> b) != 0) b++;
  return (b + 7) / 8 * 8;
}

}  // namespace

void assemble_pointset(gp_ctx* ctx, gp_pointset* ps, const double* d_X) {
  const int64_t n = ps->n;
  const int d = ps->d;
  cudaStream_t st = ctx->stream;
  std::vector<DevBuf> tmp;   // temporaries freed at the end
  ps->X = dalloc<double>(ctx, ps->bufs, (size_t)n * d);
  GP_CUDA(cudaMemcpyAsync(ps->X, d_X, sizeof(double) * n * d, cudaMemcpyDeviceToDevice, st));
  ps->U = dalloc<double>(ctx, ps->bufs, (size_t)n * d);
  ps->Us = dalloc<double>(ctx, ps->bufs, (size_t)n * d);
  ps->cell_perm = dalloc<int32_t>(ctx, ps->bufs, n);

  // ---- A1: scale, grid extent
  unsigned long long* mnmx = dalloc<unsigned long long>(ctx, tmp, 6);
  double* mm_dev = dalloc<double>(ctx, tmp, 6);
  unsigned long long init[6] = {~0ull, 0ull, ~0ull, 0ull, ~0ull, 0ull};
  h2d(ctx, mnmx, init, 6);
  k_scale<<<grid_for(n, 256), 256, 0, st>>>(ps->X, n, d, ps->rho[0], ps->rho[1], ps->rho[2], ps->U, mnmx);
  GP_CHECK_LAUNCH(ctx);
  k_decode_minmax<<<1, 32, 0, st>>>(mnmx, d, mm_dev);
  GP_CHECK_LAUNCH(ctx);
  double mm[6];
  d2h(ctx, mm, mm_dev, 2 * d);
  GP_CUDA(cudaStreamSynchronize(st));
  Grid g{};
  g.d = d;
  double cells = 1.0;
  for (int k = 0; k < d; k++) {
    GP_REQUIRE(std::isfinite(mm[2 * k]) && std::isfinite(mm[2 * k + 1]), "non-finite coordinate in X");
    g.c0[k] = (long long)std::floor(mm[2 * k]);
    g.nc[k] = (long long)std::floor(mm[2 * k + 1]) - g.c0[k] + 1;
    cells *= (double)g.nc[k];
    ps->c0[k] = g.c0[k];
    ps->nc[k] = g.nc[k];
  }
  for (int k = d; k < 3; k++) { g.c0[k] = 0; g.nc[k] = 1; }
  const double cell_cap = std::max(16777216.0, 8.0 * (double)n);
  GP_REQUIRE(cells <= cell_cap, "cell grid too large: the point extent over the core radius exceeds max(2^24, 8n) cells");
  const int64_t ncells = (int64_t)cells;
  ps->ncells = ncells;

  // ---- A1: sort by (cell key, index)
  size_t sort_tmp = radix_sort_temp_bytes(n);
  void* stmp = dev_alloc(ctx, tmp, sort_tmp);
  uint64_t* keys = dalloc<uint64_t>(ctx, tmp, n + 1);
  uint32_t* vals = dalloc<uint32_t>(ctx, tmp, n + 1);
  int64_t* key_of = dalloc<int64_t>(ctx, tmp, n);
  k_cell_keys<<<grid_for(n, 256), 256, 0, st>>>(ps->U, n, g, keys, vals);
  GP_CHECK_LAUNCH(ctx);
  radix_sort_pairs(ctx, keys, vals, n, 0, bits_for((uint64_t)ncells), stmp);
  ps->cell_start = dalloc<int64_t>(ctx, ps->bufs, ncells + 1);
  k_cell_start<<<grid_for(n + 1, 256), 256, 0, st>>>(keys, n, ncells, ps->cell_start);
  GP_CHECK_LAUNCH(ctx);
  k_gather_sorted<<<grid_for(n, 256), 256, 0, st>>>(ps->U, vals, n, d, ps->Us, ps->cell_perm, keys, key_of);
  GP_CHECK_LAUNCH(ctx);

  // ---- A2: pattern (count, scan, fill, sort rows)
  int64_t* rowcnt = dalloc<int64_t>(ctx, tmp, n + 1);
  GP_CUDA(cudaMemsetAsync(rowcnt, 0, sizeof(int64_t) * (n + 1), st));
  if (ps->support == 1) {   // the support of C_sparse (non-compact core): bump-family masks, then all pairs
    const int64_t nb = (int64_t)ps->sup_n1 * ps->sup_n2;
    double* hd = dalloc<double>(ctx, tmp, std::max<int64_t>(1, nb * ps->sup_bd));
    double* rd = dalloc<double>(ctx, tmp, std::max<int64_t>(1, nb));
    if (nb > 0) {
      h2d(ctx, hd, ps->sup_h.data(), (size_t)(nb * ps->sup_bd));
      h2d(ctx, rd, ps->sup_r.data(), (size_t)nb);
    }
    ps->fam = dalloc<uint32_t>(ctx, ps->bufs, n);
    k_family_mask<<<grid_for(n, 256), 256, 0, st>>>(ps->X, n, d, hd, rd, ps->sup_n1, ps->sup_n2, ps->sup_bd, ps->fam);
    GP_CHECK_LAUNCH(ctx);
    k_pattern_support<false><<<grid_for(n * 32, 256), 256, 0, st>>>(ps->U, ps->fam, n, d, rowcnt, nullptr, nullptr);
  } else {
    k_pattern<false><<<grid_for(n, 128), 128, 0, st>>>(ps->Us, ps->cell_perm, ps->cell_start, n, g, rowcnt, nullptr,
                                                       nullptr);
  }
  GP_CHECK_LAUNCH(ctx);
  ps->rowptr = dalloc<int64_t>(ctx, ps->bufs, n + 1);
  void* scan_tmp = dev_alloc(ctx, tmp, scan_temp_bytes(std::max<int64_t>(n + 1, 2 * n + 2)));
  exclusive_scan_i64(ctx, rowcnt, ps->rowptr, n + 1, scan_tmp);
  int64_t nnz = 0;
  d2h(ctx, &nnz, ps->rowptr + n, 1);
  GP_CUDA(cudaStreamSynchronize(st));
  ps->nnz = nnz;
  GP_REQUIRE(nnz < (int64_t)1 << 40, "pattern too large");
  ps->col = dalloc<int32_t>(ctx, ps->bufs, nnz);
  if (ps->support == 1) {   // rows come out ascending
    k_pattern_support<true><<<grid_for(n * 32, 256), 256, 0, st>>>(ps->U, ps->fam, n, d, nullptr, ps->rowptr, ps->col);
    GP_CHECK_LAUNCH(ctx);
  } else {
    int32_t* col_unsorted = dalloc<int32_t>(ctx, tmp, nnz);
    k_pattern<true><<<grid_for(n, 128), 128, 0, st>>>(ps->Us, ps->cell_perm, ps->cell_start, n, g, nullptr,
                                                      ps->rowptr, col_unsorted);
    GP_CHECK_LAUNCH(ctx);
    k_sort_rows<<<grid_for(n * 32, 256), 256, 0, st>>>(ps->rowptr, col_unsorted, n, ps->col);
    GP_CHECK_LAUNCH(ctx);
  }

  // ---- A5: nested dissection
  ps->perm = dalloc<int32_t>(ctx, ps->bufs, n);
  ps->pinv = dalloc<int32_t>(ctx, ps->bufs, n);
  int32_t* rank = dalloc<int32_t>(ctx, tmp, (size_t)n * d);
  for (int k = 0; k < d; k++) {
    k_axis_keys<<<grid_for(n, 256), 256, 0, st>>>(ps->U, n, d, k, keys, vals);
    GP_CHECK_LAUNCH(ctx);
    radix_sort_pairs(ctx, keys, vals, n, 0, 64, stmp);
    k_rank_of<<<grid_for(n, 256), 256, 0, st>>>(vals, n, rank + (int64_t)k * n);
    GP_CHECK_LAUNCH(ctx);
  }
  int32_t* act = dalloc<int32_t>(ctx, tmp, n);
  int32_t* act_seg = dalloc<int32_t>(ctx, tmp, n);
  int32_t* nact = dalloc<int32_t>(ctx, tmp, n);
  int32_t* nact_seg = dalloc<int32_t>(ctx, tmp, n);
  int32_t* leafv = dalloc<int32_t>(ctx, tmp, n);
  int64_t* vgid = dalloc<int64_t>(ctx, tmp, n);
  int8_t* vside = dalloc<int8_t>(ctx, tmp, n);
  int64_t* sflag = dalloc<int64_t>(ctx, tmp, n + 1);
  int64_t* lflag = dalloc<int64_t>(ctx, tmp, n + 1);
  int64_t* sidx = dalloc<int64_t>(ctx, tmp, n + 1);
  int64_t* lidx = dalloc<int64_t>(ctx, tmp, n + 1);
  GP_CUDA(cudaMemsetAsync(vgid, 0xff, sizeof(int64_t) * n, st));
  const int64_t maxseg = n / (GP_ND_LEAF + 1) + 2;
  int64_t* seg_i64 = dalloc<int64_t>(ctx, tmp, (size_t)maxseg * 8);   // start, size, out, gid, cnt(2), dstA, dstB
  int32_t* seg_i32 = dalloc<int32_t>(ctx, tmp, (size_t)maxseg * 3);   // axis, segA, segB
  unsigned long long* smm = dalloc<unsigned long long>(ctx, tmp, (size_t)maxseg * 6);
  int64_t* leaf_i64 = dalloc<int64_t>(ctx, tmp, (size_t)2 * (n + 2));
  std::vector<int64_t> leaf_start_h, leaf_out_h;   // leaves of the current level
  int64_t leafpos = 0;

  // host-side segment tables
  std::vector<int64_t> s_start, s_size, s_out, s_gid;
  int64_t gid_next = 0;
  int64_t tot = 0;
  if (n > GP_ND_LEAF) {
    std::vector<int32_t> iota(n), zero(n, 0);
    for (int64_t i = 0; i < n; i++) iota[i] = (int32_t)i;
    h2d(ctx, act, iota.data(), n);
    h2d(ctx, act_seg, zero.data(), n);
    s_start = {0};
    s_size = {n};
    s_out = {0};
    s_gid = {gid_next++};
    tot = n;
    GP_CUDA(cudaStreamSynchronize(st));   // host vectors above go out of scope
  } else {
    leaf_start_h = {0, n};
    leaf_out_h = {0};
    std::vector<int32_t> iota(n);
    for (int64_t i = 0; i < n; i++) iota[i] = (int32_t)i;
    h2d(ctx, leafv, iota.data(), n);
    GP_CUDA(cudaStreamSynchronize(st));
    leafpos = n;
  }
  auto flush_leaves = [&]() {
    int64_t nleaf = (int64_t)leaf_out_h.size();
    if (nleaf == 0) return;
    h2d(ctx, leaf_i64, leaf_start_h.data(), nleaf + 1);
    h2d(ctx, leaf_i64 + nleaf + 1, leaf_out_h.data(), nleaf);
    k_leaf_order<<<grid_for(nleaf * 32, 256), 256, 0, st>>>(leafv, leaf_i64, leaf_i64 + nleaf + 1, nleaf, key_of,
                                                            ps->perm);
    GP_CHECK_LAUNCH(ctx);
    GP_CUDA(cudaStreamSynchronize(st));
    leaf_start_h.clear();
    leaf_out_h.clear();
    leafpos = 0;
  };
  if (n <= GP_ND_LEAF) flush_leaves();

  while (tot > 0) {
    const int64_t nseg = (int64_t)s_start.size();
    int64_t* d_start = seg_i64;
    int64_t* d_size = seg_i64 + maxseg;
    int64_t* d_out = seg_i64 + 2 * maxseg;
    int64_t* d_gid = seg_i64 + 3 * maxseg;
    int64_t* d_cnt = seg_i64 + 4 * maxseg;   // 2 per segment
    int64_t* d_dstA = seg_i64 + 6 * maxseg;
    int64_t* d_dstB = seg_i64 + 7 * maxseg;
    int32_t* d_axis = seg_i32;
    int32_t* d_segA = seg_i32 + maxseg;
    int32_t* d_segB = seg_i32 + 2 * maxseg;
    h2d(ctx, d_start, s_start.data(), nseg);
    h2d(ctx, d_size, s_size.data(), nseg);
    h2d(ctx, d_out, s_out.data(), nseg);
    h2d(ctx, d_gid, s_gid.data(), nseg);
    // extents and split axis
    std::vector<unsigned long long> sinit((size_t)nseg * 6);
    for (int64_t s = 0; s < nseg; s++)
      for (int k = 0; k < 3; k++) {
        sinit[s * 6 + 2 * k] = ~0ull;
        sinit[s * 6 + 2 * k + 1] = 0ull;
      }
    h2d(ctx, smm, sinit.data(), (size_t)nseg * 6);
    k_seg_extent<<<grid_for(tot, 256), 256, 0, st>>>(act, act_seg, tot, ps->U, d, smm);
    GP_CHECK_LAUNCH(ctx);
    k_seg_axis<<<grid_for(nseg, 128), 128, 0, st>>>(smm, nseg, d, d_axis);
    GP_CHECK_LAUNCH(ctx);
    // sort each segment by (u_axis, index) == rank along that axis
    k_seg_sortkeys<<<grid_for(tot, 256), 256, 0, st>>>(act, act_seg, tot, d_axis, rank, n, keys, vals);
    GP_CHECK_LAUNCH(ctx);
    radix_sort_pairs(ctx, keys, vals, tot, 0, bits_for((uint64_t)nseg * (uint64_t)n), stmp);
    k_mark_sides<<<grid_for(tot, 256), 256, 0, st>>>(vals, act_seg, tot, d_start, d_size, d_gid, act, vgid, vside);
    GP_CHECK_LAUNCH(ctx);
    k_sep_flags<<<grid_for(tot + 1, 256), 256, 0, st>>>(act, act_seg, tot, d_start, d_size, ps->rowptr, ps->col,
                                                        vgid, vside, sflag, lflag);
    GP_CHECK_LAUNCH(ctx);
    exclusive_scan_i64(ctx, sflag, sidx, tot + 1, scan_tmp);
    exclusive_scan_i64(ctx, lflag, lidx, tot + 1, scan_tmp);
    k_seg_counts<<<grid_for(nseg, 128), 128, 0, st>>>(sidx, lidx, nseg, d_start, d_size, d_cnt);
    GP_CHECK_LAUNCH(ctx);
    std::vector<int64_t> cnt((size_t)2 * nseg);
    d2h(ctx, cnt.data(), d_cnt, 2 * nseg);
    GP_CUDA(cudaStreamSynchronize(st));
    // children tables
    std::vector<int64_t> n_start, n_size, n_out, n_gid, dstA(nseg), dstB(nseg);
    std::vector<int32_t> segA(nseg, -1), segB(nseg, -1);
    int64_t ntot = 0;
    for (int64_t s = 0; s < nseg; s++) {
      int64_t m = s_size[s], half = m / 2, nS = cnt[2 * s], nLr = cnt[2 * s + 1];
      int64_t sizes[2] = {nLr, m - half};
      int64_t outs[2] = {s_out[s], s_out[s] + nLr};
      for (int c = 0; c < 2; c++) {
        int64_t sz = sizes[c];
        int64_t* dst = c == 0 ? &dstA[s] : &dstB[s];
        int32_t* sg = c == 0 ? &segA[s] : &segB[s];
        if (sz > GP_ND_LEAF) {
          *sg = (int32_t)n_start.size();
          *dst = ntot;
          n_start.push_back(ntot);
          n_size.push_back(sz);
          n_out.push_back(outs[c]);
          n_gid.push_back(gid_next++);
          ntot += sz;
        } else {
          *dst = leafpos;
          if (sz > 0) {
            if (leaf_start_h.empty()) leaf_start_h.push_back(leafpos);
            leaf_out_h.push_back(outs[c]);
            leafpos += sz;
            leaf_start_h.push_back(leafpos);
          }
        }
      }
      (void)nS;
    }
    h2d(ctx, d_dstA, dstA.data(), nseg);
    h2d(ctx, d_dstB, dstB.data(), nseg);
    h2d(ctx, d_segA, segA.data(), nseg);
    h2d(ctx, d_segB, segB.data(), nseg);
    k_route<<<grid_for(tot, 256), 256, 0, st>>>(act, act_seg, tot, d_start, d_size, d_out, sidx, lidx, d_cnt, d_dstA,
                                                d_dstB, d_segA, d_segB, ps->perm, nact, nact_seg, leafv);
    GP_CHECK_LAUNCH(ctx);
    GP_CUDA(cudaStreamSynchronize(st));   // host tables are reused next level
    flush_leaves();
    std::swap(act, nact);
    std::swap(act_seg, nact_seg);
    s_start.swap(n_start);
    s_size.swap(n_size);
    s_out.swap(n_out);
    s_gid.swap(n_gid);
    tot = ntot;
  }
  k_inverse<<<grid_for(n, 256), 256, 0, st>>>(ps->perm, n, ps->pinv);
  GP_CHECK_LAUNCH(ctx);
  GP_CUDA(cudaStreamSynchronize(st));
  dev_free_all(ctx, tmp);
}

// ------------------------------------------------------------------------------------------ no-allocation counts
// gp_pattern_counts_noalloc: the count pass of the support pattern (cell list plus per-point neighbour count)
// for callers that cannot allocate device memory. All of its scratch lives in this one file-scope device array,
// which every GPU that loads the library holds until the process exits. Every call shares it and it keeps the
// last call's contents; the call writes every scratch entry it later reads (the min/max words are reset from
// the host), so no state leaks from one call to the next, but two calls that overlap on the GPU (different
// streams or contexts on one device) race on it.
#define GP_NOALLOC_MAX_N 65536
#define GP_NOALLOC_MAX_CELLS (1 << 20)
#define GP_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[GP_NOALLOC_SCRATCH_BYTES];

namespace {
// Device address of g_noalloc_scratch per device, looked up once per device (contexts on several host threads
// may make their first call at the same time).
std::atomic<void*> g_noalloc_base[64] = {};
std::mutex g_noalloc_lookup;

struct Carver {
  char* base;
  size_t used, cap;
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (used + bytes > cap) throw GpError{GP_ERR_ARG, "gp_pattern_counts_noalloc: scratch array too small"};
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};
}  // namespace

extern "C" gp_status gp_pattern_counts_noalloc(gp_ctx* ctx, const double* d_X, int64_t n, int d,
                                               const double* core_radius, int64_t* d_counts) {
  if (!ctx) return GP_ERR_ARG;
  try {
    GP_CUDA(cudaSetDevice(ctx->device));
    GP_REQUIRE(d_X && core_radius && d_counts, "d_X, core_radius and d_counts are required");
    GP_REQUIRE(n >= 1 && n <= GP_NOALLOC_MAX_N, "gp_pattern_counts_noalloc: n must be in 1..65536");
    GP_REQUIRE(d >= 1 && d <= GP_MAX_D, "d must be 1, 2 or 3");
    for (int k = 0; k < d; k++)
      GP_REQUIRE(core_radius[k] > 0.0 && std::isfinite(core_radius[k]), "core_radius must be positive");
    GP_REQUIRE(ctx->device >= 0 && ctx->device < 64, "device index out of range");
    // host code sees only a stand-in for the array: fetch its device address with the device current
    void* base = g_noalloc_base[ctx->device].load(std::memory_order_acquire);
    if (!base) {
      std::lock_guard<std::mutex> lk(g_noalloc_lookup);
      base = g_noalloc_base[ctx->device].load(std::memory_order_acquire);
      if (!base) {
        GP_CUDA(cudaGetSymbolAddress(&base, g_noalloc_scratch));
        g_noalloc_base[ctx->device].store(base, std::memory_order_release);
      }
    }
    cudaStream_t st = ctx->stream;
    Carver cv{static_cast<char*>(base), 0, GP_NOALLOC_SCRATCH_BYTES};
    double* U = cv.take<double>((size_t)n * d);
    double* Us = cv.take<double>((size_t)n * d);
    uint64_t* keys = cv.take<uint64_t>(n + 1);
    uint32_t* vals = cv.take<uint32_t>(n + 1);
    int32_t* cell_perm = cv.take<int32_t>(n);
    int64_t* key_of = cv.take<int64_t>(n);
    unsigned long long* mnmx = cv.take<unsigned long long>(6);
    double* mm_dev = cv.take<double>(6);
    void* sort_tmp = cv.take<char>(radix_sort_temp_bytes(n));
    const unsigned long long init[6] = {~0ull, 0ull, ~0ull, 0ull, ~0ull, 0ull};
    GP_CUDA(cudaMemcpyAsync(mnmx, init, sizeof(init), cudaMemcpyHostToDevice, st));
    double rho[3] = {1.0, 1.0, 1.0};
    for (int k = 0; k < d; k++) rho[k] = core_radius[k];
    k_scale<<<grid_for(n, 256), 256, 0, st>>>(d_X, n, d, rho[0], rho[1], rho[2], U, mnmx);
    GP_CHECK_LAUNCH(ctx);
    k_decode_minmax<<<1, 32, 0, st>>>(mnmx, d, mm_dev);
    GP_CHECK_LAUNCH(ctx);
    double mm[6];
    GP_CUDA(cudaMemcpyAsync(mm, mm_dev, sizeof(double) * 2 * d, cudaMemcpyDeviceToHost, st));
    GP_CUDA(cudaStreamSynchronize(st));
    Grid g{};
    g.d = d;
    double cells = 1.0;
    for (int k = 0; k < d; k++) {
      GP_REQUIRE(std::isfinite(mm[2 * k]) && std::isfinite(mm[2 * k + 1]), "non-finite coordinate in X");
      g.c0[k] = (long long)std::floor(mm[2 * k]);
      g.nc[k] = (long long)std::floor(mm[2 * k + 1]) - g.c0[k] + 1;
      cells *= (double)g.nc[k];
    }
    for (int k = d; k < 3; k++) {
      g.c0[k] = 0;
      g.nc[k] = 1;
    }
    GP_REQUIRE(cells <= (double)GP_NOALLOC_MAX_CELLS,
               "gp_pattern_counts_noalloc: more than 2^20 cells (point extent over core radius too large)");
    const int64_t ncells = (int64_t)cells;
    int64_t* cell_start = cv.take<int64_t>(ncells + 1);
    k_cell_keys<<<grid_for(n, 256), 256, 0, st>>>(U, n, g, keys, vals);
    GP_CHECK_LAUNCH(ctx);
    radix_sort_pairs(ctx, keys, vals, n, 0, bits_for((uint64_t)ncells), sort_tmp);
    k_cell_start<<<grid_for(n + 1, 256), 256, 0, st>>>(keys, n, ncells, cell_start);
    GP_CHECK_LAUNCH(ctx);
    k_gather_sorted<<<grid_for(n, 256), 256, 0, st>>>(U, vals, n, d, Us, cell_perm, keys, key_of);
    GP_CHECK_LAUNCH(ctx);
    k_pattern<false><<<grid_for(n, 128), 128, 0, st>>>(Us, cell_perm, cell_start, n, g, d_counts, nullptr, nullptr);
    GP_CHECK_LAUNCH(ctx);
    ctx->err.clear();
    return GP_OK;
  } catch (const GpError& e) {
    ctx->err = e.msg;
    return e.st;
  }
}
