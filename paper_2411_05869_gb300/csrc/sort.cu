// sort.cu -- device-wide primitives used by the cached steps A1, A2 and A5:
//   * a stable least-significant-digit radix sort of (uint64 key, uint32 value) pairs, 8-bit digits, with
//     per-tile histograms, one exclusive scan and a stable per-tile scatter (ranks from warp match masks);
//   * an exclusive prefix sum over int64 (block scans, recursive scan of block totals, add-back).
#include "gp_internal.cuh"

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ROUNDS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ROUNDS;   // 2048 keys per tile
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void k_digit_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int64_t ntiles,
                             int64_t* __restrict__ hist) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * SORT_TILE;
  for (int r = 0; r < SORT_ROUNDS; r++) {
    int64_t i = base + r * SORT_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: item i of the tile goes to offset[digit] + (number of earlier tile items with that digit).
__global__ void k_digit_scatter(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
                                int shift, int64_t ntiles, const int64_t* __restrict__ offs,
                                uint64_t* __restrict__ okeys, uint32_t* __restrict__ ovals) {
  __shared__ int64_t running[256];
  __shared__ int wcnt[SORT_THREADS / 32][256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  running[t] = offs[(int64_t)t * ntiles + blockIdx.x];
  for (int w = 0; w < SORT_THREADS / 32; w++) wcnt[w][t] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * SORT_TILE;
  for (int r = 0; r < SORT_ROUNDS; r++) {
    int64_t i = base + r * SORT_THREADS + t;
    bool valid = i < n;
    uint64_t k = valid ? keys[i] : 0;
    unsigned dig = valid ? (unsigned)((k >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, dig);
    int leader = __ffs(peers) - 1;
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == leader) wcnt[warp][dig] = __popc(peers);
    __syncthreads();
    if (valid) {
      int64_t pos = running[dig] + rank;
      for (int w = 0; w < warp; w++) pos += wcnt[w][dig];
      okeys[pos] = k;
      ovals[pos] = vals[i];
    }
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < SORT_THREADS / 32; w++) {
      tot += wcnt[w][t];
      wcnt[w][t] = 0;
    }
    running[t] += tot;
    __syncthreads();
  }
}

// Block-level exclusive scan of SCAN_TILE int64 values; writes the tile total to sums[blockIdx.x].
__global__ void k_scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             int64_t* __restrict__ sums) {
  __shared__ int64_t wsum[SCAN_THREADS / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)t * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; k++) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int64_t incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < SCAN_THREADS / 32) wsum[lane] = w;   // inclusive warp prefix
  }
  __syncthreads();
  int64_t excl = incl - s + (warp > 0 ? wsum[warp - 1] : 0);
  for (int k = 0; k < SCAN_ITEMS; k++) {
    if (base + k < n) out[base + k] = excl;
    excl += v[k];
  }
  if (t == SCAN_THREADS - 1) sums[blockIdx.x] = wsum[SCAN_THREADS / 32 - 1];
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ sums) {
  int64_t i = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
  int64_t add = sums[blockIdx.x];
  for (int k = 0; k < SCAN_ITEMS; k++, i += SCAN_THREADS)
    if (i < n) out[i] += add;
}

}  // namespace

size_t scan_temp_bytes(int64_t n) {
  size_t b = 0;
  while (n > SCAN_TILE) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    b += (size_t)(nb + 1) * sizeof(int64_t);
    n = nb;
  }
  return b + 2 * sizeof(int64_t);
}

void exclusive_scan_i64(gp_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, void* temp) {
  if (n <= 0) return;
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  int64_t* sums = static_cast<int64_t*>(temp);
  k_scan_tiles<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, out, n, sums);
  GP_CHECK_LAUNCH(ctx);
  if (nb > 1) {
    exclusive_scan_i64(ctx, sums, sums, nb, sums + nb + 1);
    k_scan_add<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(out, n, sums);
    GP_CHECK_LAUNCH(ctx);
  }
}

size_t radix_sort_temp_bytes(int64_t n) {
  int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
  size_t b = (size_t)n * (sizeof(uint64_t) + sizeof(uint32_t));
  b = (b + 255) & ~size_t(255);
  b += (size_t)256 * ntiles * sizeof(int64_t) * 2;
  b += scan_temp_bytes(256 * ntiles) + 256;
  return b;
}

void radix_sort_pairs(gp_ctx* ctx, uint64_t* keys, uint32_t* vals, int64_t n, int begin_bit, int end_bit,
                      void* temp) {
  if (n <= 1 || end_bit <= begin_bit) return;
  int64_t ntiles = (n + SORT_TILE - 1) / SORT_TILE;
  char* t = static_cast<char*>(temp);
  uint64_t* k2 = reinterpret_cast<uint64_t*>(t);
  uint32_t* v2 = reinterpret_cast<uint32_t*>(t + (size_t)n * sizeof(uint64_t));
  size_t off = ((size_t)n * (sizeof(uint64_t) + sizeof(uint32_t)) + 255) & ~size_t(255);
  int64_t* hist = reinterpret_cast<int64_t*>(t + off);
  int64_t* offs = hist + 256 * ntiles;
  void* scratch = offs + 256 * ntiles;
  uint64_t *ka = keys, *kb = k2;
  uint32_t *va = vals, *vb = v2;
  int passes = 0;
  for (int shift = begin_bit; shift < end_bit; shift += 8, passes++) {
    k_digit_hist<<<(unsigned)ntiles, SORT_THREADS, 0, ctx->stream>>>(ka, n, shift, ntiles, hist);
    GP_CHECK_LAUNCH(ctx);
    exclusive_scan_i64(ctx, hist, offs, 256 * ntiles, scratch);
    k_digit_scatter<<<(unsigned)ntiles, SORT_THREADS, 0, ctx->stream>>>(ka, va, n, shift, ntiles, offs, kb, vb);
    GP_CHECK_LAUNCH(ctx);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (passes & 1) {
    GP_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream));
    GP_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream));
  }
}
