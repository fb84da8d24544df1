// k_small.cu - the rank-sized algebra of one step, in FP64 unless noted.
//
//   G_n   = T_(n) T_(n)^T, its Cholesky factor and inverse   (pseudo-inverse, Sec. 2.2)
//   M_n   = Y_(n) T_(n)^T,  X_n = M_n G_n^{-1}                 (Eq. 2.16 times dt)
//   P_n   = U_n^T W_n X_n,  U'_n = U_n + X_n - U_n P_n         (complement projector, Sec. 2.2;
//                                                               Euler update, Sec. 2.3)
//   C_n   = U'^T W U' = R^T R,  U''_n = U'_n R^{-1}            (weighted Cholesky-QR; the
//                                                               paper does not say how it keeps
//                                                               Eq. 2.6, this is the reading used)
//   sigma^(n): eigenvalues of G_n                              (Eq. 2.18)
//
// Small r x r matrices are stored column-major with leading dimension 32
// (TDB_MAX_RANK): A[a + 32 b].  N x r matrices are column-major with leading
// dimension N.  Y_n and T use the tensor views (L_n, X_n, Q_n) of common.cuh.
// Rank-sized reductions over N_n rows are split across CTAs into partial r x r
// blocks, then summed in a fixed order (deterministic).
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
// G_n = T_(n) T_(n)^T : partial sums over slices of the column range (p modes at once)
// ---------------------------------------------------------------------------
__global__ void k_gram_partial(ModeDesc d, const double* __restrict__ T, double* __restrict__ Gpart, int nsplit) {
  const int n = blockIdx.y;
  const int r = d.r[n];
  const int64_t L = prod_r_below(d, n), Q = prod_r_above(d, n);
  const int64_t ncol = L * Q;
  const int64_t c0 = ncol * blockIdx.x / nsplit, c1 = ncol * (blockIdx.x + 1) / nsplit;
  double* out = Gpart + ((int64_t)n * nsplit + blockIdx.x) * LD * LD;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int a = e % r, b = e / r;
    double s = 0.0;
    if (a <= b) {
      for (int64_t c = c0; c < c1; ++c) {
        int64_t l = c % L, q = c / L;
        const double* base = T + l + L * r * q;
        s += base[L * a] * base[L * b];
      }
    }
    out[a + LD * b] = s;
  }
}

// Sum the G partials, Cholesky, inverse and eigenvalues (sigma^2) of G_n.
// The eigenvalues: float Jacobi (warm-started from the previous eigenvectors in
// Vprev, r x r, ld 32), then Rayleigh quotients v^T G v / v^T v in double.
__global__ void k_gram_finish(ModeDesc d, const double* __restrict__ Gpart, int nsplit, double* __restrict__ Gout,
                              double* __restrict__ Ginv, double* __restrict__ sig2, float* __restrict__ Vprev,
                              int warm, unsigned* flags) {
  extern __shared__ double smem[];
  const int n = blockIdx.x;
  const int r = d.r[n];
  double* G = smem;                     // LD*LD
  double* Lc = G + LD * LD;             // LD*LD
  double* Li = Lc + LD * LD;            // LD*LD
  float* Af = (float*)(Li + LD * LD);   // LD*LD (float)
  float* Vf = Af + LD * LD;             // LD*LD
  float* csf = Vf + LD * LD;            // 64
  float* redf = csf + 64;               // 32
  int* pq = (int*)(redf + 32);          // 64
  __shared__ bool ok;
  __shared__ double lam[LD];

  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
    int a = e % LD, b = e / LD;
    double s = 0.0;
    if (a < r && b < r) {
      int aa = a <= b ? a : b, bb = a <= b ? b : a;
      s = sum_strided(Gpart + (int64_t)n * nsplit * LD * LD + aa + LD * bb, nsplit, LD * LD);
    }
    G[e] = s;
    Lc[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) Gout[(int64_t)n * LD * LD + e] = G[e];
  bool good = chol_smem(Lc, LD, r, &ok);
  if (!good && threadIdx.x == 0) atomicOr(flags, kFlagCholGram);
  trinv_lower_smem(Lc, Li, LD, r);
  // G^{-1} = L^{-T} L^{-1}
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int a = e % r, b = e / r;
    double s = 0.0;
    int k0 = a > b ? a : b;
    for (int k = k0; k < r; ++k) s += Li[k + LD * a] * Li[k + LD * b];
    Ginv[(int64_t)n * LD * LD + a + LD * b] = s;
  }
  // eigenvalues of G (sigma^2)
  double scale = 0.0;
  for (int a = 0; a < r; ++a) scale = fmax(scale, G[a + LD * a]);
  if (scale <= 0.0) scale = 1.0;
  float* Vp = Vprev + (int64_t)n * LD * LD;
  // A = Vp^T (G / scale) Vp in float when warm (two r^3 products through Vf as scratch), else G / scale
  if (warm) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      int i = e % r, b = e / r;
      float s = 0.f;
      for (int j = 0; j < r; ++j) s += (float)(G[i + LD * j] / scale) * Vp[j + LD * b];
      Vf[i + LD * b] = s;                        // G Vp
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      int a = e % r, b = e / r;
      float s = 0.f;
      for (int i = 0; i < r; ++i) s += Vp[i + LD * a] * Vf[i + LD * b];
      Af[a + LD * b] = s;
    }
  } else {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      int a = e % r, b = e / r;
      Af[a + LD * b] = (float)(G[a + LD * b] / scale);
    }
  }
  __syncthreads();
  jacobi_smem<float>(Af, Vf, LD, r, 30, 1e-6f, csf, pq, redf);
  // eigenvectors in the original basis: W = Vp * Vf (or Vf)
  // store W (float) as next warm start; Rayleigh quotients in double
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int a = e % r, b = e / r;
    float s = 0.f;
    if (warm) {
      for (int k = 0; k < r; ++k) s += Vp[a + LD * k] * Vf[k + LD * b];
    } else {
      s = Vf[a + LD * b];
    }
    Af[a + LD * b] = s;   // reuse Af as the eigenvector matrix
  }
  __syncthreads();
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double num = 0.0, den = 0.0;
    for (int i = 0; i < r; ++i) {
      double gi = 0.0;
      for (int k = 0; k < r; ++k) gi += G[i + LD * k] * (double)Af[k + LD * j];
      num += (double)Af[i + LD * j] * gi;
      den += (double)Af[i + LD * j] * (double)Af[i + LD * j];
    }
    lam[j] = den > 0 ? num / den : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // selection sort descending, carrying eigenvector columns' order
    int idx[LD];
    for (int j = 0; j < r; ++j) idx[j] = j;
    for (int i = 0; i < r; ++i) {
      int best = i;
      for (int j = i + 1; j < r; ++j)
        if (lam[idx[j]] > lam[idx[best]]) best = j;
      int t = idx[i]; idx[i] = idx[best]; idx[best] = t;
    }
    for (int j = 0; j < r; ++j) sig2[(int64_t)n * LD + j] = lam[idx[j]];
    for (int j = r; j < LD; ++j) sig2[(int64_t)n * LD + j] = 0.0;
    for (int j = 0; j < r; ++j)
      for (int i = 0; i < r; ++i) Vp[i + LD * j] = Af[i + LD * idx[j]];
  }
}

void launch_gram(const ModeDesc& d, const double* T, double* Gpart, int nsplit, double* G, double* Ginv,
                 double* sig2, float* Vprev, int warm, unsigned* flags, cudaStream_t s) {
  dim3 g1(nsplit, d.p);
  k_gram_partial<<<g1, 256, 0, s>>>(d, T, Gpart, nsplit); count_launch();
  size_t sm = 3 * LD * LD * sizeof(double) + 2 * LD * LD * sizeof(float) + (64 + 32) * sizeof(float) + 64 * sizeof(int);
  k_gram_finish<<<d.p, 256, sm, s>>>(d, Gpart, nsplit, G, Ginv, sig2, Vprev, warm, flags); count_launch();
}

// ---------------------------------------------------------------------------
// Row kernels.  Grid (row tiles of 32, p); block 1024 = 32 rows x 32 rank slots.
// ---------------------------------------------------------------------------

// M = Y_(n) T_(n)^T (compute type), X = M G^{-1} (double), P partial = U^T W X over the tile.
template <typename Tc>
__global__ void k_rows_mx(RowArgs a) {
  const int n = blockIdx.y;
  const int r = a.d.r[n];
  const int64_t N = a.d.N[n];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  if (i0 >= N) return;
  const int li = threadIdx.x & 31, ca = threadIdx.x >> 5;
  const int64_t i = i0 + li;
  __shared__ double Msh[32][LD + 1];
  __shared__ double Xsh[32][LD + 1];
  __shared__ double Gi[LD * LD];
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) Gi[e] = a.Ginv[(int64_t)n * LD * LD + e];
  const int64_t L = prod_r_below(a.d, n), Q = prod_r_above(a.d, n);
  const Tc* Y = (const Tc*)a.Y[n];
  const Tc* T = (const Tc*)a.Tc;
  // M[i, ca] = sum_c Y_(n)[i, c] T_(n)[ca, c] over column chunks of 32 staged in shared memory;
  // column c = l + L q addresses Y[l + L (i + N q)] and T[l + L (ca + r q)]
  __shared__ Tc Ysh[32][33];
  __shared__ Tc Tsh[LD][33];
  const int64_t ncol = L * Q;
  Tc s = Tc(0);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t c0 = 0; c0 < ncol; c0 += 32) {
    {
      const int64_t c = c0 + tx;
      const int64_t ii = i0 + ty;
      Tc vy = Tc(0), vt = Tc(0);
      if (c < ncol) {
        const int64_t l = c % L, q = c / L;
        if (ii < N) vy = Y[l + L * (ii + N * q)];
        if (ty < r) vt = T[l + L * (ty + (int64_t)r * q)];
      }
      Ysh[ty][tx] = vy;
      Tsh[ty][tx] = vt;
    }
    __syncthreads();
    if (ca < r) {
#pragma unroll 8
      for (int x = 0; x < 32; ++x) s += Ysh[li][x] * Tsh[ca][x];
    }
    __syncthreads();
  }
  if (ca < r) Msh[li][ca] = (double)s;
  __syncthreads();
  if (ca < r) {
    double x = 0.0;
    for (int b = 0; b < r; ++b) x += Msh[li][b] * Gi[b + LD * ca];
    Xsh[li][ca] = (i < N) ? x : 0.0;
    if (i < N) a.X[n][i + N * ca] = x;
  }
  __syncthreads();
  // P partial: sum_{rows in tile} U[i,ra] w[i] X[i,rb]
  if (threadIdx.x < r * r) {
    int ra = threadIdx.x % r, rb = threadIdx.x / r;
    double s = 0.0;
    for (int t = 0; t < 32; ++t) {
      int64_t ii = i0 + t;
      if (ii < N) s += a.U[n][ii + N * ra] * a.w[n][ii] * Xsh[t][rb];
    }
    a.part[(((int64_t)n * a.ntile) + blockIdx.x) * LD * LD + ra + LD * rb] = s;
  }
}

// Sum per-tile partials of each mode into out (p x LD x LD); tiles beyond a mode's N are zero-skipped.
__global__ void k_sum_tiles(ModeDesc d, const double* __restrict__ part, int ntile, double* __restrict__ out) {
  const int n = blockIdx.x;
  const int r = d.r[n];
  const int nt = (int)((d.N[n] + 31) / 32);
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
    int a = e % LD, b = e / LD;
    double s = 0.0;
    if (a < r && b < r) s = sum_strided(part + (int64_t)n * ntile * LD * LD + e, nt, LD * LD);
    out[(int64_t)n * LD * LD + e] = s;
  }
}

// U' = U + X - U P ; C partial = U'^T W U' over the tile.
__global__ void k_rows_u1(RowArgs a) {
  const int n = blockIdx.y;
  const int r = a.d.r[n];
  const int64_t N = a.d.N[n];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  if (i0 >= N) return;
  const int li = threadIdx.x & 31, ca = threadIdx.x >> 5;
  const int64_t i = i0 + li;
  __shared__ double Ush[32][LD + 1];
  __shared__ double Psh[LD * LD];
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) Psh[e] = a.P[(int64_t)n * LD * LD + e];
  if (ca < r) Ush[li][ca] = (i < N) ? a.U[n][i + N * ca] : 0.0;
  __syncthreads();
  double up = 0.0;
  if (ca < r && i < N) {
    double s = 0.0;
    for (int b = 0; b < r; ++b) s += Ush[li][b] * Psh[b + LD * ca];
    up = Ush[li][ca] + a.X[n][i + N * ca] - s;
    a.Up[n][i + N * ca] = up;
  }
  __syncthreads();
  if (ca < r) Ush[li][ca] = up;
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

// R = Rinv = I (re-orthonormalisation switched off)
__global__ void k_set_identity(int p, double* __restrict__ R, double* __restrict__ Rinv) {
  for (int e = threadIdx.x; e < p * LD * LD; e += blockDim.x) {
    int i = e % LD, j = (e / LD) % LD;
    R[e] = Rinv[e] = (i == j) ? 1.0 : 0.0;
  }
}

template <typename Tc>
void launch_update_rows(RowArgs& a, double* P, double* R, double* Rinv, unsigned* flags, bool reorth, cudaStream_t s) {
  int64_t Nmax = 0;
  for (int n = 0; n < a.d.p; ++n) Nmax = std::max<int64_t>(Nmax, a.d.N[n]);
  dim3 grid((unsigned)((Nmax + 31) / 32), a.d.p);
  k_rows_mx<Tc><<<grid, 1024, 0, s>>>(a); count_launch();
  k_sum_tiles<<<a.d.p, 256, 0, s>>>(a.d, a.part, a.ntile, P); count_launch();
  a.P = P;
  k_rows_u1<<<grid, 1024, 0, s>>>(a); count_launch();
  if (reorth)
    { k_cholqr_small<<<a.d.p, 256, 0, s>>>(a.d, a.part, a.ntile, R, Rinv, flags); count_launch(); }
  else
    { k_set_identity<<<1, 256, 0, s>>>(a.d.p, R, Rinv); count_launch(); }
  a.Rinv = Rinv;
  k_rows_u2<Tc><<<grid, 1024, 0, s>>>(a); count_launch();
}
template void launch_update_rows<float>(RowArgs&, double*, double*, double*, unsigned*, bool, cudaStream_t);
template void launch_update_rows<double>(RowArgs&, double*, double*, double*, unsigned*, bool, cudaStream_t);

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
