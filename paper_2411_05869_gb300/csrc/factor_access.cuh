// factor_access.cuh -- read access to a numeric factor for the solve-type kernels (the forward/backward sweeps,
// the log-determinant and the predictive variance): FP64 column-major panels (GP_FP64) or FP32 row-major panels
// with FP64 64 x 64 diagonal tiles (GP_MIXED), with the inverses of the diagonal blocks in the working precision.
#pragma once
#include "gp_internal.cuh"

namespace fa {

constexpr int T = GP_TILE;

// ---------------------------------------------------------------------------------------- factor access
// L(i, j) in the solve's working precision; Ld(i, j) in FP64 (the log-determinant).
struct AccF64 {
  const double* P;
  int64_t m;
  __device__ __forceinline__ double L(int64_t i, int64_t j) const { return P[j * m + i]; }
  __device__ __forceinline__ double Ld(int64_t i, int64_t j) const { return P[j * m + i]; }
};
struct AccMix {
  const float* P;
  const double* D;
  int w, ldw;
  __device__ __forceinline__ double Ld(int64_t i, int64_t j) const {
    if (i < w && (i >> 6) == (j >> 6)) return D[(i >> 6) * (T * T) + (i & 63) * T + (j & 63)];
    return (double)P[i * ldw + j];
  }
  __device__ __forceinline__ float L(int64_t i, int64_t j) const {
    if (i < w && (i >> 6) == (j >> 6)) return (float)D[(i >> 6) * (T * T) + (i & 63) * T + (j & 63)];
    return P[i * ldw + j];
  }
};
// The solve's working precision V: FP64 with the FP64 factor; FP32 with the mixed factor, whose solves only
// precondition the FP64 refinement (the FP64 residual fixes the accuracy of alpha).
struct StoreF64 {
  using V = double;
  static constexpr bool kRowMajor = false;
  const double* P;
  int64_t PE;
  const double* DI;   // inverses of the 64 x 64 diagonal blocks
  int64_t DE;
  __device__ __forceinline__ const double* inv(const DevPlan& dp, int32_t s, int b) const {
    return DI + (int64_t)b * DE + dp.doff[s];
  }
  using Acc = AccF64;
  __device__ __forceinline__ AccF64 acc(const DevPlan& dp, int32_t s, int b) const {
    return AccF64{P + (int64_t)b * PE + dp.loff[s], (int64_t)dp.w[s] + dp.r[s]};
  }
};
struct StoreMix {
  using V = float;
  static constexpr bool kRowMajor = true;
  const float* P;
  const double* D;
  int64_t P32E, DE;
  const float* DI;   // FP32 inverses of the 64 x 64 diagonal blocks
  __device__ __forceinline__ const float* inv(const DevPlan& dp, int32_t s, int b) const {
    return DI + (int64_t)b * DE + dp.doff[s];
  }
  using Acc = AccMix;
  __device__ __forceinline__ AccMix acc(const DevPlan& dp, int32_t s, int b) const {
    return AccMix{P + (int64_t)b * P32E + dp.loff32[s], D + (int64_t)b * DE + dp.doff[s], dp.w[s], dp.ldw[s]};
  }
};


// Index of the front whose tile prefix pre[0..nfront) covers task t.
__device__ __forceinline__ int find_front(const int64_t* pre, int nfront, int64_t t) {
  int lo = 0, hi = nfront - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace fa
