// common.cuh - device helpers and launch declarations shared by libtdb's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tdb.h"

namespace tdb {

constexpr int kMaxModes = TDB_MAX_MODES;
constexpr int kMaxRank = TDB_MAX_RANK;

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread gets the result.  `sh` must hold >= 32 values.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) r = warp_sum(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Per-mode descriptors passed by value to small-matrix kernels
// ---------------------------------------------------------------------------

struct ModeDesc {
  int p;
  int64_t N[kMaxModes];   // sizes
  int r[kMaxModes];       // ranks
};

// The core / projection views: for mode n a tensor with sizes
// (prod_{m<n} r_m) x X_n x (prod_{m>n} r_m) where X_n is r_n (core) or N_n (Y_n).
__host__ __device__ inline int64_t prod_r_below(const ModeDesc& d, int n) {
  int64_t v = 1;
  for (int m = 0; m < n; ++m) v *= d.r[m];
  return v;
}
__host__ __device__ inline int64_t prod_r_above(const ModeDesc& d, int n) {
  int64_t v = 1;
  for (int m = n + 1; m < d.p; ++m) v *= d.r[m];
  return v;
}
__host__ __device__ inline int64_t prod_r(const ModeDesc& d) {
  int64_t v = 1;
  for (int m = 0; m < d.p; ++m) v *= d.r[m];
  return v;
}

// Device status word bits (sticky, read back by the host).
enum : unsigned {
  kFlagNonFinite = 1u,
  kFlagCholGram = 2u,     // T_(n) T_(n)^T not positive definite
  kFlagCholQR = 4u,       // U^T W U not positive definite
  kFlagTimeout = 8u,
  kFlagEigNoConv = 16u,
};

}  // namespace tdb
