// k_small.cu - rank-sized algebra outside the per-step update (FP64): the weighted
// Cholesky-QR of freshly computed bases at (re)initialisation,
//   C_n = U^T W U = R^T R,  U <- U R^{-1},  A = W U
// (the paper does not say how it keeps Eq. 2.6; this is the reading used), and a
// single-CTA Jacobi eigensolver for small symmetric matrices.
//
// Small r x r matrices are stored column-major with leading dimension 32
// (TDB_MAX_RANK): A[a + 32 b].  N x r matrices are column-major with leading
// dimension N.  Rank-sized reductions over N_n rows are split across CTAs into
// partial r x r blocks, then summed in a fixed order (deterministic).
#include "common.cuh"
#include "kernels.h"
#include "small_dev.cuh"

namespace tdb {

constexpr int LD = kMaxRank;  // leading dimension of r x r matrices

// sum_{k < n} p[k * stride] with four independent accumulators (fixed order, loads in flight)
__device__ __forceinline__ double sum_strided(const double* __restrict__ p, int n, int64_t stride) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int k = 0;
  for (; k + 4 <= n; k += 4) {
    s0 += p[(int64_t)k * stride];
    s1 += p[(int64_t)(k + 1) * stride];
    s2 += p[(int64_t)(k + 2) * stride];
    s3 += p[(int64_t)(k + 3) * stride];
  }
  for (; k < n; ++k) s0 += p[(int64_t)k * stride];
  return (s0 + s1) + (s2 + s3);
}

// ---------------------------------------------------------------------------
// Row kernels.  Grid (row tiles of 32, p); block 1024 = 32 rows x 32 rank slots.
// ---------------------------------------------------------------------------

// C = sum partials; C = L L^T; R = L^T; Rinv = L^{-T}; also R itself.
__global__ void k_cholqr_small(ModeDesc d, const double* __restrict__ part, int ntile, double* __restrict__ R,
                               double* __restrict__ Rinv, unsigned* flags) {
  __shared__ double C[LD * LD];
  __shared__ double Li[LD * LD];
  __shared__ bool ok;
  const int n = blockIdx.x;
  const int r = d.r[n];
  const int nt = (int)((d.N[n] + 31) / 32);
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
    int a = e % LD, b = e / LD;
    double s = 0.0;
    if (a < r && b < r) s = sum_strided(part + (int64_t)n * ntile * LD * LD + e, nt, LD * LD);
    C[e] = s;
  }
  __syncthreads();
  bool good = chol_smem(C, LD, r, &ok);
  if (!good && threadIdx.x == 0) atomicOr(flags, kFlagCholQR);
  trinv_lower_smem(C, Li, LD, r);
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
    int a = e % LD, b = e / LD;
    // R = L^T (upper), Rinv = (L^{-1})^T
    R[(int64_t)n * LD * LD + e] = (a < r && b < r) ? C[b + LD * a] : 0.0;
    Rinv[(int64_t)n * LD * LD + e] = (a < r && b < r) ? Li[b + LD * a] : 0.0;
  }
}

// U'' = U' R^{-1}; A = W U'' in the compute type.
template <typename Ta>
__global__ void k_rows_u2(RowArgs a) {
  const int n = blockIdx.y;
  const int r = a.d.r[n];
  const int64_t N = a.d.N[n];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  if (i0 >= N) return;
  const int li = threadIdx.x & 31, ca = threadIdx.x >> 5;
  const int64_t i = i0 + li;
  __shared__ double Ush[32][LD + 1];
  __shared__ double Rsh[LD * LD];
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) Rsh[e] = a.Rinv[(int64_t)n * LD * LD + e];
  if (ca < r) Ush[li][ca] = (i < N) ? a.Up[n][i + N * ca] : 0.0;
  __syncthreads();
  if (ca < r && i < N) {
    double s = 0.0;
    for (int b = 0; b <= ca; ++b) s += Ush[li][b] * Rsh[b + LD * ca];
    a.Uout[n][i + N * ca] = s;
    ((Ta*)a.A[n])[i + N * ca] = (Ta)(a.w[n][i] * s);
  }
}

// ---------------------------------------------------------------------------
// Weighted Cholesky-QR of freshly computed bases (no core compensation; used at
// (re)initialisation): C = U^T W U, U <- U R^{-1}, A = W U.
// ---------------------------------------------------------------------------
__global__ void k_rows_cpart(RowArgs a) {
  const int n = blockIdx.y;
  const int r = a.d.r[n];
  const int64_t N = a.d.N[n];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  if (i0 >= N) return;
  const int li = threadIdx.x & 31, ca = threadIdx.x >> 5;
  const int64_t i = i0 + li;
  __shared__ double Ush[32][LD + 1];
  if (ca < r) Ush[li][ca] = (i < N) ? a.Up[n][i + N * ca] : 0.0;
  __syncthreads();
  if (threadIdx.x < r * r) {
    int ra = threadIdx.x % r, rb = threadIdx.x / r;
    double s = 0.0;
    for (int t = 0; t < 32; ++t) {
      int64_t ii = i0 + t;
      if (ii < N) s += Ush[t][ra] * a.w[n][ii] * Ush[t][rb];
    }
    a.part[(((int64_t)n * a.ntile) + blockIdx.x) * LD * LD + ra + LD * rb] = s;
  }
}

template <typename Tc>
void launch_orthonormalize(RowArgs& a, double* R, double* Rinv, unsigned* flags, cudaStream_t s) {
  int64_t Nmax = 0;
  for (int n = 0; n < a.d.p; ++n) Nmax = std::max<int64_t>(Nmax, a.d.N[n]);
  dim3 grid((unsigned)((Nmax + 31) / 32), a.d.p);
  k_rows_cpart<<<grid, 1024, 0, s>>>(a); count_launch();
  k_cholqr_small<<<a.d.p, 256, 0, s>>>(a.d, a.part, a.ntile, R, Rinv, flags); count_launch();
  a.Rinv = Rinv;
  k_rows_u2<Tc><<<grid, 1024, 0, s>>>(a); count_launch();
}
template void launch_orthonormalize<float>(RowArgs&, double*, double*, unsigned*, cudaStream_t);
template void launch_orthonormalize<double>(RowArgs&, double*, double*, unsigned*, cudaStream_t);

// ---------------------------------------------------------------------------
// Standalone Jacobi on an n x n symmetric matrix (n <= 96), one CTA; eigenvalues
// descending into ev, eigenvectors (columns, ld n) into Vout with the largest-
// magnitude entry of each column made positive.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_jacobi_eig(const T* __restrict__ Ain, int n, double* __restrict__ ev, T* __restrict__ Vout,
                             int max_sweeps, T tol, unsigned* flags) {
  extern __shared__ unsigned char smraw[];
  const int lda = 97;
  T* A = (T*)smraw;
  T* V = A + lda * 96;
  T* cs = V + lda * 96;
  T* red = cs + 128;
  int* pq = (int*)(red + 32);
  __shared__ int order[96];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e % n, j = e / n;
    A[i + lda * j] = Ain[i + (int64_t)n * j];
  }
  __syncthreads();
  int sw = jacobi_smem<T>(A, V, lda, n, max_sweeps, tol, cs, pq, red);
  if (sw >= max_sweeps && threadIdx.x == 0 && flags) atomicOr(flags, kFlagEigNoConv);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < n; ++j) order[j] = j;
    for (int i = 0; i < n; ++i) {
      int best = i;
      for (int j = i + 1; j < n; ++j)
        if (A[order[j] + lda * order[j]] > A[order[best] + lda * order[best]]) best = j;
      int t = order[i]; order[i] = order[best]; order[best] = t;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int o = order[j];
    ev[j] = (double)A[o + lda * o];
    int im = 0;
    T best = 0;
    for (int i = 0; i < n; ++i) {
      T v = fabs(V[i + lda * o]);
      if (v > best) { best = v; im = i; }
    }
    T sgn = V[im + lda * o] < T(0) ? T(-1) : T(1);
    for (int i = 0; i < n; ++i) Vout[i + (int64_t)n * j] = sgn * V[i + lda * o];
  }
}

template <typename T>
void launch_jacobi_eig(const T* A, int n, double* ev, T* V, unsigned* flags, cudaStream_t s) {
  size_t sm = (2 * 97 * 96 + 128 + 32) * sizeof(T) + 128 * sizeof(int);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_jacobi_eig<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  T tol = sizeof(T) == 8 ? T(1e-15) : T(1e-6);
  k_jacobi_eig<T><<<1, 512, sm, s>>>(A, n, ev, V, 40, tol, flags); count_launch();
}
template void launch_jacobi_eig<float>(const float*, int, double*, float*, unsigned*, cudaStream_t);
template void launch_jacobi_eig<double>(const double*, int, double*, double*, unsigned*, cudaStream_t);

}  // namespace tdb
