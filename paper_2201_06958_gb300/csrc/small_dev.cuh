// small_dev.cuh - shared-memory dense kernels used inside single CTAs:
// cyclic Jacobi, Cholesky and triangular inverse.
#pragma once
#include "common.cuh"
#include "fastrcp.cuh"

namespace tdb {

// ---------------------------------------------------------------------------
// Jacobi eigensolver for a symmetric matrix held in shared memory (one CTA).
// Brent-Luk round-robin ordering: in round k of a sweep the index pairs are
// (k, n'-1) and ((k+j) mod (n'-1), (k-j) mod (n'-1)) for j = 1..n'/2-1, with n'
// the size rounded up to even.  Each 2x2 block of A is rotated by its two pair
// rotations; V accumulates the rotations.  Returns the number of sweeps used.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ int jacobi_smem(T* A, T* V, int lda, int n, int max_sweeps, T tol, T* cs /* 2 * 64 */,
                           int* pq /* 2 * 64 */, T* red /* 32 */) {
  const int nn = (n + 1) & ~1;
  const int half = nn / 2;
  // pad
  for (int e = threadIdx.x; e < nn * nn; e += blockDim.x) {
    int i = e % nn, j = e / nn;
    if (i >= n || j >= n) A[i + lda * j] = (i == j) ? T(0) : T(0);
    V[i + lda * j] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // convergence test: off-diagonal vs diagonal mass
    T off = 0, dia = 0;
    for (int e = threadIdx.x; e < nn * nn; e += blockDim.x) {
      int i = e % nn, j = e / nn;
      T v = A[i + lda * j];
      if (i == j) dia += v * v; else off += v * v;
    }
    off = block_sum(off, red);
    dia = block_sum(dia, red);
    if (off <= tol * tol * dia || dia == T(0)) break;
    for (int rd = 0; rd < nn - 1; ++rd) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int p, q;
        if (k == 0) { p = rd; q = nn - 1; }
        else { p = (rd + k) % (nn - 1); q = (rd - k + (nn - 1)) % (nn - 1); }
        T app = A[p + lda * p], aqq = A[q + lda * q], apq = A[p + lda * q];
        T c = 1, s = 0;
        const T thr = tol * T(1e-3);   // skip rotations of negligible pairs (no square root, compute type)
        if (apq != T(0) && apq * apq > thr * thr * fabs(app * aqq)) {
          if constexpr (sizeof(T) == 8) {
            // the same formulas with the Newton-refined reciprocal and reciprocal square root
            // (FP64 division and square root are long sequences here; this runs per pair per round)
            const double theta = (aqq - app) * drcp(2.0 * apq);
            const double at = fabs(theta);
            const double x = fma(at, at, 1.0);
            const double root = at < 1e150 ? x * drsqrt(x) : at;      // sqrt(theta^2 + 1)
            const double t = (theta >= 0 ? 1.0 : -1.0) * drcp(at + root);
            c = drsqrt(fma(t, t, 1.0));
            s = t * c;
          } else {
            T theta = (aqq - app) / (T(2) * apq);
            T t = (theta >= 0 ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
            c = T(1) / sqrt(t * t + T(1));
            s = t * c;
          }
        }
        cs[2 * k] = c; cs[2 * k + 1] = s;
        pq[2 * k] = p; pq[2 * k + 1] = q;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < half * half; e += blockDim.x) {
        int I = e % half, J = e / half;
        int pI = pq[2 * I], qI = pq[2 * I + 1], pJ = pq[2 * J], qJ = pq[2 * J + 1];
        T cI = cs[2 * I], sI = cs[2 * I + 1], cJ = cs[2 * J], sJ = cs[2 * J + 1];
        T b00 = A[pI + lda * pJ], b01 = A[pI + lda * qJ], b10 = A[qI + lda * pJ], b11 = A[qI + lda * qJ];
        // columns (right multiply by the J rotation)
        T c00 = cJ * b00 - sJ * b01, c01 = sJ * b00 + cJ * b01;
        T c10 = cJ * b10 - sJ * b11, c11 = sJ * b10 + cJ * b11;
        // rows (left multiply by the transposed I rotation)
        A[pI + lda * pJ] = cI * c00 - sI * c10;
        A[pI + lda * qJ] = cI * c01 - sI * c11;
        A[qI + lda * pJ] = sI * c00 + cI * c10;
        A[qI + lda * qJ] = sI * c01 + cI * c11;
      }
      for (int e = threadIdx.x; e < nn * half; e += blockDim.x) {
        int i = e % nn, J = e / nn;
        int pJ = pq[2 * J], qJ = pq[2 * J + 1];
        T cJ = cs[2 * J], sJ = cs[2 * J + 1];
        T vp = V[i + lda * pJ], vq = V[i + lda * qJ];
        V[i + lda * pJ] = cJ * vp - sJ * vq;
        V[i + lda * qJ] = sJ * vp + cJ * vq;
      }
      __syncthreads();
    }
  }
  return sweep;
}

// Cholesky of the SPD matrix S (r x r, shared, leading dim lda) in place: lower
// factor L with S = L L^T.  Returns false if a pivot is not positive.
template <typename T>
__device__ __forceinline__ bool chol_smem_t(T* S, int lda, int r, bool* ok_sh) {
  if (threadIdx.x == 0) *ok_sh = true;
  __syncthreads();
  __shared__ T inv_dk;
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      T d = S[k + lda * k];
      if (!(d > T(0))) { *ok_sh = false; d = T(1); }
      if constexpr (sizeof(T) == 8) {
        const double y = drsqrt(d);     // one reciprocal square root per pivot (Newton-refined)
        S[k + lda * k] = d * y;
        inv_dk = y;
      } else {
        const T sd = sqrt(d);
        S[k + lda * k] = sd;
        inv_dk = T(1) / sd;
      }
    }
    __syncthreads();
    const T ik = inv_dk;
    for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) S[i + lda * k] *= ik;
    __syncthreads();
    for (int e = threadIdx.x; e < (r - k - 1) * (r - k - 1); e += blockDim.x) {
      int i = k + 1 + e % (r - k - 1), j = k + 1 + e / (r - k - 1);
      if (j <= i) S[i + lda * j] -= S[i + lda * k] * S[j + lda * k];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int i = e % r, j = e / r;
    if (j > i) S[i + lda * j] = T(0);
  }
  __syncthreads();
  return *ok_sh;
}
__device__ __forceinline__ bool chol_smem(double* S, int lda, int r, bool* ok_sh) { return chol_smem_t<double>(S, lda, r, ok_sh); }

// Inverse of the lower-triangular L (shared) into Li (shared): column j solves L x = e_j.
template <typename T>
__device__ __forceinline__ void trinv_lower_smem_t(const T* L, T* Li, int lda, int r) {
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    for (int i = 0; i < r; ++i) {
      if (i < j) { Li[i + lda * j] = T(0); continue; }
      T s = (i == j) ? T(1) : T(0);
      for (int k = j; k < i; ++k) s -= L[i + lda * k] * Li[k + lda * j];
      Li[i + lda * j] = s / L[i + lda * i];
    }
  }
  __syncthreads();
}
__device__ __forceinline__ void trinv_lower_smem(const double* L, double* Li, int lda, int r) {
  trinv_lower_smem_t<double>(L, Li, lda, r);
}

}  // namespace tdb
