// k_hosvd.cu - truncated HOSVD used to initialise and re-initialise the bases
// (Sec. 2.3 last paragraph, Sec. 2.5), on the weighted mode-n Gram matrices
//     C_n = W_n^{1/2} V_(n) W_{-n} V_(n)^T W_n^{1/2}          (Sec. 2.6 names this matrix)
// whose eigenvalues are the squared mode-n singular values of the weighted data.
//
// Eigen-decomposition: cyclic Jacobi with the Brent-Luk round-robin order.
//   n <= 96 : one CTA, matrix in shared memory (k_small.cu).
//   n  > 96 : cooperative multi-CTA kernel, matrix in global memory (L2 resident),
//             one bounded grid barrier per round.  The three values each rotation
//             of the next round needs are written by the updating threads into a
//             parity-double-buffered array, so no second barrier is needed.
//   In reduced-precision modes the eigenvectors come from a float Jacobi and the
//   eigenvalues are refined as Rayleigh quotients v^T C v in double.
#include "common.cuh"
#include "kernels.h"
#include "small_dev.cuh"

namespace tdb {

// ---------------------------------------------------------------------------
// Weighted mode-n Gram: partial 32x32 tiles over column slices, then finish.
// Column c of V_(n) is (l, q): V[l + L (i + N q)].
// ---------------------------------------------------------------------------

__device__ __forceinline__ double column_weight(const GramView& g, int64_t c) {
  int64_t l = c % g.L, q = c / g.L;
  double wc = 1.0;
  for (int m = 0; m < g.n; ++m) { wc *= g.w[m][l % g.N[m]]; l /= g.N[m]; }
  for (int m = g.n + 1; m < g.p; ++m) { wc *= g.w[m][q % g.N[m]]; q /= g.N[m]; }
  return wc;
}

template <typename Tv>
__global__ void k_wgram_partial(const Tv* __restrict__ V, GramView g, int ntile, int ksplit, double* __restrict__ part) {
  // blockIdx.x: upper tile pair (ti <= tj), blockIdx.y: column slice
  int t = blockIdx.x, ti = 0;
  while (t >= ntile - ti) { t -= ntile - ti; ++ti; }
  const int tj = ti + t;
  const int64_t i0 = (int64_t)ti * 32, j0 = (int64_t)tj * 32;
  const int64_t ncol = g.L * g.Q;
  const int64_t c0 = ncol * blockIdx.y / ksplit, c1 = ncol * (blockIdx.y + 1) / ksplit;
  __shared__ Tv As[32][33];
  __shared__ Tv Bs[32][33];
  __shared__ double wcol[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc = 0.0;
  const bool ifast = (g.L == 1);
  for (int64_t cb = c0; cb < c1; cb += 32) {
    if (threadIdx.x < 32) {
      int64_t c = cb + threadIdx.x;
      wcol[threadIdx.x] = (c < c1) ? column_weight(g, c) : 0.0;
    }
    __syncthreads();
    // load tiles: element (i, c) with (row, col) = ifast ? (tx, ty) : (ty, tx)
    {
      int ri = ifast ? tx : ty, cc = ifast ? ty : tx;
      int64_t c = cb + cc;
      Tv va = 0, vb = 0;
      if (c < c1) {
        int64_t l = c % g.L, q = c / g.L;
        int64_t ia = i0 + ri, ib = j0 + ri;
        if (ia < g.Nn) va = V[l + g.L * (ia + g.Nn * q)];
        if (ib < g.Nn) vb = V[l + g.L * (ib + g.Nn * q)];
      }
      As[ri][cc] = (Tv)((double)va * wcol[cc]);
      Bs[ri][cc] = vb;
    }
    __syncthreads();
    Tv s = 0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) s += As[tx][k] * Bs[ty][k];
    acc += (double)s;
    __syncthreads();
  }
  part[((int64_t)blockIdx.x * ksplit + blockIdx.y) * 1024 + tx + 32 * ty] = acc;
}

template <typename Tc>
__global__ void k_wgram_finish(GramView g, int ntile, int ksplit, const double* __restrict__ part,
                               double* __restrict__ C64, Tc* __restrict__ Cc) {
  const int64_t Nn = g.Nn;
  const double* wn = g.w[g.n];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Nn * Nn; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % Nn, j = e / Nn;
    int64_t a = i <= j ? i : j, b = i <= j ? j : i;
    int ti = (int)(a / 32), tj = (int)(b / 32);
    int pair = ti * ntile - ti * (ti - 1) / 2 + (tj - ti);
    int tx = (int)(a % 32), ty = (int)(b % 32);
    double s = 0.0;
    for (int k = 0; k < ksplit; ++k) s += part[((int64_t)pair * ksplit + k) * 1024 + tx + 32 * ty];
    s *= sqrt(wn[i] * wn[j]);
    C64[e] = s;
    if (Cc) Cc[e] = (Tc)s;
  }
}

template <typename Tv>
void launch_wgram(const Tv* V, const GramView& g, double* part, size_t part_cap, double* C64, void* Cc, int cc_float,
                  cudaStream_t s) {
  int ntile = (int)((g.Nn + 31) / 32);
  int npair = ntile * (ntile + 1) / 2;
  int64_t ncol = g.L * g.Q;
  int ksplit = (int)std::max<int64_t>(1, std::min<int64_t>((152 * 4 + npair - 1) / npair, (ncol + 255) / 256));
  while ((size_t)npair * ksplit * 1024 > part_cap && ksplit > 1) --ksplit;
  k_wgram_partial<Tv><<<dim3(npair, ksplit), 1024, 0, s>>>(V, g, ntile, ksplit, part); count_launch();
  int blocks = (int)std::min<int64_t>((g.Nn * g.Nn + 255) / 256, 1024);
  if (cc_float)
    { k_wgram_finish<float><<<blocks, 256, 0, s>>>(g, ntile, ksplit, part, C64, (float*)Cc); count_launch(); }
  else
    { k_wgram_finish<double><<<blocks, 256, 0, s>>>(g, ntile, ksplit, part, C64, (double*)Cc); count_launch(); }
}
template void launch_wgram<float>(const float*, const GramView&, double*, size_t, double*, void*, int, cudaStream_t);
template void launch_wgram<double>(const double*, const GramView&, double*, size_t, double*, void*, int, cudaStream_t);

// Selection of the leading eigenpairs from candidate vectors: the m candidates are
// the columns of V (n rows, leading dim ldv) with approximate eigenvalues on the
// diagonal of A (leading dim lda).  Rough order by diag(A), Rayleigh quotients
// v^T C v / v^T v in double against C64 for the top kk = k + 2, final order by them,
// sign fix (largest-magnitude entry positive) and the trace of C64.
template <typename T>
__global__ void k_eig_order(const T* __restrict__ A, int lda, int m, int kk, int* __restrict__ order_out) {
  __shared__ int order[1024];
  __shared__ float dg[1024];
  for (int j = threadIdx.x; j < m; j += blockDim.x) { order[j] = j; dg[j] = (float)A[j + (int64_t)lda * j]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < kk; ++i) {
      int best = i;
      for (int j = i + 1; j < m; ++j)
        if (dg[order[j]] > dg[order[best]]) best = j;
      int t = order[i]; order[i] = order[best]; order[best] = t;
      order_out[i] = order[i];
    }
  }
}

template <typename T>
__global__ void k_eig_cv(const double* __restrict__ C64, int n, const T* __restrict__ V, int ldv,
                         const int* __restrict__ order, int kk, double* __restrict__ CV) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * kk; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % n;
    int j = (int)(e / n);
    const T* v = V + (int64_t)ldv * order[j];
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += C64[i + (int64_t)n * l] * (double)v[l];
    CV[e] = s;
  }
}

template <typename T>
__global__ void k_eig_final(const T* __restrict__ V, int ldv, int n, const double* __restrict__ C64,
                            const int* __restrict__ order_in, int kk, const double* __restrict__ CV, int k,
                            double* __restrict__ ev_out, double* __restrict__ Q_out, double* __restrict__ trace_out) {
  __shared__ double red[32];
  __shared__ double rq[64];
  __shared__ int ord[64];
  __shared__ int imax;
  for (int j = 0; j < kk; ++j) {
    const T* v = V + (int64_t)ldv * order_in[j];
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double vi = (double)v[i];
      num += vi * CV[i + (int64_t)n * j];
      den += vi * vi;
    }
    num = block_sum(num, red);
    den = block_sum(den, red);
    if (threadIdx.x == 0) { rq[j] = den > 0 ? num / den : 0.0; ord[j] = order_in[j]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < kk; ++i) {
      int best = i;
      for (int j = i + 1; j < kk; ++j)
        if (rq[j] > rq[best]) best = j;
      double tv = rq[i]; rq[i] = rq[best]; rq[best] = tv;
      int to = ord[i]; ord[i] = ord[best]; ord[best] = to;
    }
  }
  __syncthreads();
  double tr = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tr += C64[i + (int64_t)n * i];
  tr = block_sum(tr, red);
  if (threadIdx.x == 0) *trace_out = tr;
  __shared__ double bv[32];
  __shared__ int bi[32];
  for (int j = 0; j < k; ++j) {
    const T* v = V + (int64_t)ldv * ord[j];
    double nrm = 0.0;
    double best = -1.0;
    int ib = 0x7fffffff;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double a = (double)v[i];
      nrm += a * a;
      a = fabs(a);
      if (a > best || (a == best && i < ib)) { best = a; ib = i; }
    }
    nrm = block_sum(nrm, red);
    // block argmax of |v_i| (first index on ties)
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, ib, o);
      if (ob > best || (ob == best && oi < ib)) { best = ob; ib = oi; }
    }
    if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = ib; }
    __syncthreads();
    if (threadIdx.x == 0) {
      int nw = (blockDim.x + 31) >> 5;
      double b0 = bv[0];
      int i0 = bi[0];
      for (int w = 1; w < nw; ++w)
        if (bv[w] > b0 || (bv[w] == b0 && bi[w] < i0)) { b0 = bv[w]; i0 = bi[w]; }
      imax = i0;
      ev_out[j] = rq[j];
    }
    __syncthreads();
    double sc = (v[imax] < T(0) ? -1.0 : 1.0) / sqrt(nrm > 0 ? nrm : 1.0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) Q_out[i + (int64_t)n * j] = sc * (double)v[i];
    __syncthreads();
  }
}

template <typename T>
static void eig_select(const T* A, int lda, int m, const T* V, int ldv, int n, const double* C64, int k, double* ev,
                       double* Q, double* trace, double* scratch, cudaStream_t s) {
  int kk = k + 2 < m ? k + 2 : m;
  if (k > kk) k = kk;
  int* order = (int*)scratch;                 // 64 ints
  double* CV = scratch + 64;                  // n x kk
  k_eig_order<T><<<1, 256, 0, s>>>(A, lda, m, kk, order); count_launch();
  int blocks = (int)std::min<int64_t>(((int64_t)n * kk + 127) / 128, 1024);
  k_eig_cv<T><<<blocks, 128, 0, s>>>(C64, n, V, ldv, order, kk, CV); count_launch();
  k_eig_final<T><<<1, 256, 0, s>>>(V, ldv, n, C64, order, kk, CV, k, ev, Q, trace); count_launch();
}

// ---------------------------------------------------------------------------
// Block subspace iteration for the leading eigenpairs of an n x n PSD Gram
// (n > 96): Z = C Q, Q = orth(Z) by Cholesky-QR on the column-normalised Gram
// (a small diagonal shift is added if the factorisation fails), repeated `iters`
// times, then Rayleigh-Ritz: H = Q^T C Q, Jacobi on H, Ritz vectors Q S, and
// the selection above (Rayleigh quotients against C in double).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float hash_unit(uint32_t i, uint32_t j) {
  uint32_t h = i * 0x9E3779B1u ^ (j + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return (float)(h & 0xFFFFFF) / 8388608.0f - 1.0f;   // [-1, 1)
}

template <typename T>
__global__ void k_si_start(T* __restrict__ Q, int n, int m) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * m; e += (int64_t)gridDim.x * blockDim.x)
    Q[e] = (T)hash_unit((uint32_t)(e % n), (uint32_t)(e / n));
}

// Warm start: the first k0 columns from Q0 (n x k0, a previous solve), the rest hash columns.
template <typename T>
__global__ void k_si_warm(T* __restrict__ Q, int n, int m, const double* __restrict__ Q0, int k0) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / n;
    Q[e] = col < k0 ? (T)Q0[e] : (T)hash_unit((uint32_t)(e % n), (uint32_t)col);
  }
}

// Z = C Q   (C: n x n, Q and Z: n x m, all leading dim n).  Block = 32 rows x 8 cols.
template <typename T>
__global__ void k_si_gemm(const T* __restrict__ C, const T* __restrict__ Q, T* __restrict__ Z, int n, int m) {
  __shared__ T Cs[32][33];
  __shared__ T Qs[32][9];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  T acc = 0;
  for (int l0 = 0; l0 < n; l0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int l = l0 + ty + 8 * q;
      Cs[tx][ty + 8 * q] = (i0 + tx < n && l < n) ? C[(i0 + tx) + (int64_t)n * l] : T(0);
    }
    Qs[tx][ty] = (l0 + tx < n && j0 + ty < m) ? Q[(l0 + tx) + (int64_t)n * (j0 + ty)] : T(0);
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) acc += Cs[tx][kk] * Qs[kk][ty];
    __syncthreads();
  }
  if (i0 + tx < n && j0 + ty < m) Z[(i0 + tx) + (int64_t)n * (j0 + ty)] = acc;
}

// G = X^T Y (m x m); X, Y: n x m, leading dim n.  One warp per entry, lanes over
// rows (coalesced), partial sums in T, the warp total in double.
template <typename T>
__global__ void k_si_inner(const T* __restrict__ X, const T* __restrict__ Y, int n, int m, double* __restrict__ G) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int e = warp; e < m * m; e += nw) {
    const int a = e % m, b = e / m;
    const T* x = X + (int64_t)n * a;
    const T* y = Y + (int64_t)n * b;
    T s = 0;
    for (int i = lane; i < n; i += 32) s += x[i] * y[i];
    double d = warp_sum((double)s);
    if (lane == 0) G[a + (int64_t)m * b] = d;
  }
}

// Cholesky-QR factor of the Gram G = Z^T Z, in the working precision T: with
// D = diag(G)^{1/2}, D^{-1} G D^{-1} + shift0 I = L L^T (a shift of 1e-5 or 1e-2 on the
// unit diagonal instead if that fails), and Rinv = D^{-1} L^{-T} so that Q = Z Rinv
// has (near) orthonormal columns.
template <typename T>
__global__ void k_si_cholinv(const double* __restrict__ G, int m, double shift0, double* __restrict__ Rinv,
                             unsigned* flags) {
  extern __shared__ unsigned char smraw_ci[];
  T* S = (T*)smraw_ci;         // m x m (ld 64)
  T* Li = S + 64 * 64;         // m x m (ld 64)
  __shared__ double d[64];
  __shared__ bool ok;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double g = G[j + (int64_t)m * j];
    d[j] = g > 0 ? sqrt(g) : 1.0;
  }
  __syncthreads();
  for (int attempt = 0; attempt < 3; ++attempt) {
    double shift = attempt == 0 ? shift0 : (attempt == 1 ? 1e-5 : 1e-2);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int i = e % m, j = e / m;
      S[i + 64 * j] = (T)(G[i + (int64_t)m * j] / (d[i] * d[j]) + (i == j ? shift : 0.0));
    }
    __syncthreads();
    bool good = chol_smem_t<T>(S, 64, m, &ok);
    if (good) break;
    if (attempt == 2 && threadIdx.x == 0) atomicOr(flags, kFlagEigNoConv);
  }
  // Li = L^{-1} by forward substitution on all columns at once: after step k row k of Li is
  // final (scaled by 1/L_kk) and is taken out of the rows below it (one FMA per entry,
  // spread over the block, instead of one thread per column)
  __shared__ T dinv[64];
  for (int i = threadIdx.x; i < m; i += blockDim.x) dinv[i] = T(1) / S[i + 64 * i];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e % m, j = e / m;
    Li[i + 64 * j] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    for (int j = threadIdx.x; j <= k; j += blockDim.x) Li[k + 64 * j] *= dinv[k];
    __syncthreads();
    const int rows = m - k - 1, cols = k + 1;
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int i = k + 1 + e / cols, j = e % cols;
      Li[i + 64 * j] -= S[i + 64 * k] * Li[k + 64 * j];
    }
    __syncthreads();
  }
  __shared__ double dinvd[64];
  for (int i = threadIdx.x; i < m; i += blockDim.x) dinvd[i] = 1.0 / d[i];
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e % m, j = e / m;
    // Rinv = D^{-1} L^{-T}:  Rinv[i][j] = Li[j][i] / d[i]
    Rinv[i + (int64_t)m * j] = (j >= i) ? (double)Li[j + 64 * i] * dinvd[i] : 0.0;
  }
}

// Y = X M (X: n x m ld n, M: m x mc double ld m, Y: n x mc ld n); upper = M upper triangular.
template <typename T>
__global__ void k_si_apply(const T* __restrict__ X, const double* __restrict__ M, int n, int m, int mc, int upper,
                           T* __restrict__ Y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * mc; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % n;
    int j = (int)(e / n);
    int lmax = upper ? (j < m - 1 ? j : m - 1) : m - 1;
    double s = 0.0;
    for (int l = 0; l <= lmax; ++l) s += (double)X[i + (int64_t)n * l] * M[l + (int64_t)m * j];
    Y[e] = (T)s;
  }
}

// X = Q S: Q n x m (ld n), S mm x mm (ld mm; rows >= m are the padding), X n x mm (ld n)
template <typename T>
__global__ void k_si_ritz(const T* __restrict__ Q, const T* __restrict__ S, int n, int m, int mm, T* __restrict__ X) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * mm; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % n;
    int j = (int)(e / n);
    double acc = 0.0;
    for (int l = 0; l < m; ++l) acc += (double)Q[i + (int64_t)n * l] * (double)S[l + (int64_t)mm * j];
    X[e] = (T)acc;
  }
}

template <typename T>
__global__ void k_to_T(const double* __restrict__ a, T* __restrict__ b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (T)a[i];
}

template <typename T>
__global__ void k_to_double_sym(const double* __restrict__ H, int m, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    int i = e % m, j = e / m;
    out[e] = 0.5 * (H[i + m * j] + H[j + m * i]);
  }
}

// Small n: single-CTA Jacobi then the same selection.
template <typename T>
__global__ void k_jacobi_small_full(const T* __restrict__ Cin, int n, T* __restrict__ Aout, T* __restrict__ Vout,
                                    int max_sweeps, T tol, unsigned* flags) {
  extern __shared__ unsigned char smraw[];
  const int lda = 97;
  T* A = (T*)smraw;
  T* V = A + lda * 96;
  T* cs = V + lda * 96;
  T* red = cs + 128;
  int* pq = (int*)(red + 32);
  const int nn = (n + 1) & ~1;
  for (int e = threadIdx.x; e < nn * nn; e += blockDim.x) {
    int i = e % nn, j = e / nn;
    A[i + lda * j] = (i < n && j < n) ? Cin[i + (int64_t)n * j] : T(0);
  }
  __syncthreads();
  int sw = jacobi_smem<T>(A, V, lda, n, max_sweeps, tol, cs, pq, red);
  if (sw >= max_sweeps && threadIdx.x == 0) atomicOr(flags, kFlagEigNoConv);
  __syncthreads();
  for (int e = threadIdx.x; e < nn * nn; e += blockDim.x) {
    int i = e % nn, j = e / nn;
    Aout[i + (int64_t)nn * j] = A[i + lda * j];
    Vout[i + (int64_t)nn * j] = V[i + lda * j];
  }
}

template <typename T>
tdb_status eig_leading_small(const T* Cc, const double* C64, int n, int k, T* A_ws, T* V_ws, unsigned* flags,
                             double* ev, double* Q, double* trace, double* scratch, cudaStream_t s) {
  size_t sm = (2 * 97 * 96 + 128 + 32) * sizeof(T) + 128 * sizeof(int);
  cudaFuncSetAttribute(k_jacobi_small_full<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  T tol = sizeof(T) == 8 ? T(1e-15) : T(1e-6);
  k_jacobi_small_full<T><<<1, 512, sm, s>>>(Cc, n, A_ws, V_ws, 40, tol, flags); count_launch();
  int nn = (n + 1) & ~1;
  eig_select<T>(A_ws, nn, nn, V_ws, nn, n, C64, k, ev, Q, trace, scratch, s);
  return TDB_OK;
}
template tdb_status eig_leading_small<float>(const float*, const double*, int, int, float*, float*, unsigned*,
                                             double*, double*, double*, double*, cudaStream_t);
template tdb_status eig_leading_small<double>(const double*, const double*, int, int, double*, double*, unsigned*,
                                              double*, double*, double*, double*, cudaStream_t);

template <typename T>
tdb_status eig_subspace(const T* Cc, const double* C64, int n, int k, int iters, const SubspaceWs<T>& ws,
                        unsigned* flags, double* ev, double* Q, double* trace, double* scratch, cudaStream_t s,
                        const double* Q0) {
  const int m = std::min(n, std::min(64, k + 16));
  const int mm = (m + 1) & ~1;
  int blocks_nm = (int)std::min<int64_t>(((int64_t)n * m + 255) / 256, 1024);
  dim3 ggrid((n + 31) / 32, (m + 7) / 8);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_si_cholinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * (int)sizeof(T));
    attr = true;
  }
  // Each iteration re-orthonormalises Z = C Q by shifted Cholesky-QR followed by two plain
  // passes (shifted CholeskyQR3 of Fukaya, Kannan, Nakatsukasa, Yamamoto and Yanagisawa,
  // SIAM J. Sci. Comput. 2020).  The shift s = 11 (n m + m (m + 1)) u ||Z||_2^2, with
  // ||Z||_2^2 <= m for the unit-diagonal scaled Gram, makes the first factor succeed for
  // kappa(Z) up to about u^{-1}, leaving kappa(Q) near u^{-1/2}; the plain passes then make Q
  // orthonormal to working precision.  A plain Cholesky-QR alone breaks down when C Q is
  // (numerically) rank deficient: a mode longer than the product of the others (a grouped
  // spatial mode), or a fast-decaying spectrum.
  const double u = sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
  const double s0 = 11.0 * ((double)n * m + (double)m * (m + 1)) * u * m;
  const size_t ci_smem = 2 * 64 * 64 * sizeof(T);
  const int inner_blocks = (m * m * 32 + 255) / 256;
  if (Q0) {
    k_si_warm<T><<<blocks_nm, 256, 0, s>>>(ws.Q, n, m, Q0, std::min(k, m)); count_launch();
  } else {
    k_si_start<T><<<blocks_nm, 256, 0, s>>>(ws.Q, n, m); count_launch();
  }
  for (int it = 0; it < iters; ++it) {
    k_si_gemm<T><<<ggrid, 256, 0, s>>>(Cc, ws.Q, ws.Z, n, m); count_launch();
    k_si_inner<T><<<inner_blocks, 256, 0, s>>>(ws.Z, ws.Z, n, m, ws.G); count_launch();
    k_si_cholinv<T><<<1, 256, ci_smem, s>>>(ws.G, m, s0, ws.R, flags); count_launch();
    k_si_apply<T><<<blocks_nm, 256, 0, s>>>(ws.Z, ws.R, n, m, m, 1, ws.Q); count_launch();
    for (int pass = 0; pass < 2; ++pass) {
      T* src = pass == 0 ? ws.Q : ws.Z;
      T* dst = pass == 0 ? ws.Z : ws.Q;
      k_si_inner<T><<<inner_blocks, 256, 0, s>>>(src, src, n, m, ws.G); count_launch();
      k_si_cholinv<T><<<1, 256, ci_smem, s>>>(ws.G, m, 0.0, ws.R, flags); count_launch();
      k_si_apply<T><<<blocks_nm, 256, 0, s>>>(src, ws.R, n, m, m, 1, dst); count_launch();
    }
  }
  // Rayleigh-Ritz
  k_si_gemm<T><<<ggrid, 256, 0, s>>>(Cc, ws.Q, ws.Z, n, m); count_launch();
  k_si_inner<T><<<(m * m * 32 + 255) / 256, 256, 0, s>>>(ws.Q, ws.Z, n, m, ws.G); count_launch();
  k_to_double_sym<T><<<(m * m + 255) / 256, 256, 0, s>>>(ws.G, m, ws.R); count_launch();
  k_to_T<T><<<(m * m + 255) / 256, 256, 0, s>>>(ws.R, ws.H, m * m); count_launch();
  size_t sm = (2 * 97 * 96 + 128 + 32) * sizeof(T) + 128 * sizeof(int);
  static bool attr2 = false;
  if (!attr2) {
    cudaFuncSetAttribute(k_jacobi_small_full<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr2 = true;
  }
  // Rayleigh-Ritz Jacobi: to the rounding floor from a cold start; from a warm start (the
  // refinement of a float solve) off-diagonal mass 1e-26 of the diagonal's suffices (the
  // Ritz values are then refined as Rayleigh quotients against the double Gram)
  T tol = sizeof(T) == 8 ? (Q0 ? T(1e-13) : T(1e-15)) : T(1e-6);
  k_jacobi_small_full<T><<<1, 512, sm, s>>>(ws.H, m, ws.JA, ws.JV, 30, tol, flags); count_launch();
  // Ritz vectors X = Q S  (S = JV, mm x mm with ld mm; use its first m rows)
  k_si_ritz<T><<<(int)std::min<int64_t>(((int64_t)n * mm + 255) / 256, 1024), 256, 0, s>>>(ws.Q, ws.JV, n, m, mm, ws.X); count_launch();
  eig_select<T>(ws.JA, mm, mm, ws.X, n, n, C64, k, ev, Q, trace, scratch, s);
  return TDB_OK;
}
template tdb_status eig_subspace<float>(const float*, const double*, int, int, int, const SubspaceWs<float>&, unsigned*,
                                        double*, double*, double*, double*, cudaStream_t, const double*);
template tdb_status eig_subspace<double>(const double*, const double*, int, int, int, const SubspaceWs<double>&,
                                         unsigned*, double*, double*, double*, double*, cudaStream_t, const double*);

// U = W^{-1/2} Q[:, :r] (before the Cholesky-QR that makes U^T W U = I exact)
__global__ void k_scale_basis(const double* __restrict__ Q, const double* __restrict__ w, int64_t n, int r,
                              double* __restrict__ U) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * r; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % n;
    U[e] = Q[e] / sqrt(w[i]);
  }
}
void launch_scale_basis(const double* Q, const double* w, int64_t n, int r, double* U, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n * r + 255) / 256, 1024);
  if (blocks < 1) blocks = 1;
  k_scale_basis<<<blocks, 256, 0, s>>>(Q, w, n, r, U); count_launch();
}

// ---------------------------------------------------------------------------
// A long first or last mode n (more points than the product M of the other modes) from
// the short side: with B = W_n^{1/2} V_(n) W_{-n}^{1/2} (N_n x M), C_n = B B^T has the
// nonzero eigenvalues of K = B^T B (M x M) and, for K z = lambda z, the unit eigenvector
// B z / sqrt(lambda) - the left singular vectors of B.  So the HOSVD of such a mode needs
// K, its leading eigenpairs and one product with B, never the N_n x N_n matrix.
// Column q of B^T is the merged index of the other modes, whose weight is
// w_q = prod_{m != n} w_m (i_m) with q = i_a + N_a (i_b + ...) over those modes in order.
// ---------------------------------------------------------------------------
__global__ void k_merge_weights(WeightView wv, int skip, int64_t M, double* __restrict__ wq) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < M; c += (int64_t)gridDim.x * blockDim.x) {
    int64_t idx = c;
    double w = 1.0;
    for (int m = 0; m < wv.p; ++m) {
      if (m == skip) continue;
      w *= wv.w[m][idx % wv.N[m]];
      idx /= wv.N[m];
    }
    wq[c] = w;
    wq[M + c] = sqrt(w);
  }
}
void launch_merge_weights(const WeightView& wv, int skip, int64_t M, double* wq, cudaStream_t s) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, 1024));
  k_merge_weights<<<blocks, 256, 0, s>>>(wv, skip, M, wq); count_launch();
}

// Q[:, j] = B Z[:, j] / sqrt(lambda_j) in double.  Element (i, q) of B is
// V[i + N_n q] (first mode) or V[q + M i] (last mode), times sqrt(w_n(i) w_q) when the
// weights are given (sqw_q = sqrt(w_q)), else V is already weighted.
template <typename Tv>
__global__ void k_short_map(const Tv* __restrict__ V, int first, int64_t Nn, int64_t M, const double* __restrict__ wn,
                            const double* __restrict__ sqw, const double* __restrict__ Z, const double* __restrict__ ev,
                            int k, double* __restrict__ Q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nn; i += (int64_t)gridDim.x * blockDim.x) {
    const double si = wn ? sqrt(wn[i]) : 1.0;
    for (int j = 0; j < k; ++j) {
      const double* z = Z + M * j;
      double acc = 0.0;
      for (int64_t q = 0; q < M; ++q) {
        const double v = (double)V[first ? i + Nn * q : q + M * i];
        acc = fma(sqw ? v * sqw[q] : v, z[q], acc);
      }
      const double lam = ev[j];
      Q[i + Nn * j] = lam > 0.0 ? si * acc / sqrt(lam) : 0.0;
    }
  }
}

// Each column scaled to unit length, its entry of largest magnitude made positive (the
// first such entry on ties), as for the eigenvectors of the direct route.
__global__ void k_col_unit_sign(double* __restrict__ Q, int64_t n) {
  __shared__ double red[32];
  __shared__ double bv[32];
  __shared__ long long bi[32];
  __shared__ long long imax;
  double* q = Q + n * blockIdx.x;
  double nrm = 0.0, best = -1.0;
  long long ib = 0x7fffffffffffffffll;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = q[i];
    nrm += a * a;
    if (fabs(a) > best) { best = fabs(a); ib = i; }
  }
  nrm = block_sum(nrm, red);
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, ib, o);
    if (ob > best || (ob == best && oi < ib)) { best = ob; ib = oi; }
  }
  if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = ib; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b0 = bv[0];
    long long i0 = bi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > b0 || (bv[w] == b0 && bi[w] < i0)) { b0 = bv[w]; i0 = bi[w]; }
    imax = i0;
  }
  __syncthreads();
  const double sc = (q[imax] < 0.0 ? -1.0 : 1.0) / sqrt(nrm > 0.0 ? nrm : 1.0);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) q[i] *= sc;
}

template <typename Tv>
void launch_short_map(const Tv* V, int first, int64_t Nn, int64_t M, const double* wn, const double* sqw,
                      const double* Z, const double* ev, int k, double* Q, cudaStream_t s) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((Nn + 127) / 128, 1024));
  k_short_map<Tv><<<blocks, 128, 0, s>>>(V, first, Nn, M, wn, sqw, Z, ev, k, Q); count_launch();
  k_col_unit_sign<<<k, 256, 0, s>>>(Q, Nn); count_launch();
}
template void launch_short_map<float>(const float*, int, int64_t, int64_t, const double*, const double*,
                                      const double*, const double*, int, double*, cudaStream_t);
template void launch_short_map<double>(const double*, int, int64_t, int64_t, const double*, const double*,
                                       const double*, const double*, int, double*, cudaStream_t);

}  // namespace tdb
