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
// Bounded grid barrier (all CTAs co-resident: cooperative launch).  On timeout
// the kernel records kFlagTimeout and every CTA leaves through the flag check.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned* gen, unsigned nblocks, unsigned* flags) {
  __shared__ int timed_out;
  __syncthreads();
  if (threadIdx.x == 0) {
    timed_out = 0;
    volatile unsigned* vgen = gen;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (++spins > (1ll << 24)) {  // ~1 s at the sleep below
          atomicOr(flags, kFlagTimeout);
          timed_out = 1;
          break;
        }
        if (*(volatile unsigned*)flags & kFlagTimeout) { timed_out = 1; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return timed_out == 0;
}

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
  k_wgram_partial<Tv><<<dim3(npair, ksplit), 1024, 0, s>>>(V, g, ntile, ksplit, part);
  int blocks = (int)std::min<int64_t>((g.Nn * g.Nn + 255) / 256, 1024);
  if (cc_float)
    k_wgram_finish<float><<<blocks, 256, 0, s>>>(g, ntile, ksplit, part, C64, (float*)Cc);
  else
    k_wgram_finish<double><<<blocks, 256, 0, s>>>(g, ntile, ksplit, part, C64, (double*)Cc);
}
template void launch_wgram<float>(const float*, const GramView&, double*, size_t, double*, void*, int, cudaStream_t);
template void launch_wgram<double>(const double*, const GramView&, double*, size_t, double*, void*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Multi-CTA Jacobi (cooperative).  A, V: nn x nn (column-major, ld nn), nn even.
// rin: 2 x (nn/2) x 3 rotation inputs (app, aqq, apq) by round parity.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pair_of(int rd, int m /* nn-1 */, int i, int* k, int* role) {
  // round rd pairs: k = 0 -> (rd, m); k >= 1 -> ((rd + k) mod m, (rd - k) mod m)
  if (i == m) { *k = 0; *role = 1; return; }
  if (i == rd) { *k = 0; *role = 0; return; }
  int kk = ((i - rd) % m + m) % m;
  if (kk <= (m - 1) / 2) { *k = kk; *role = 0; return; }
  *k = ((rd - i) % m + m) % m;
  *role = 1;
}

__device__ __forceinline__ void pair_members(int rd, int m, int k, int* p, int* q) {
  if (k == 0) { *p = rd; *q = m; }
  else { *p = (rd + k) % m; *q = ((rd - k) % m + m) % m; }
}

template <typename T>
__global__ void k_jacobi_coop(T* A, T* V, int nn, T* rin, double* redpart, unsigned* bar, unsigned* flags, int max_sweeps, double tol,
                              int* sweeps_out) {
  extern __shared__ unsigned char smraw[];
  T* cs = (T*)smraw;                         // 2 * half
  int* pq = (int*)(cs + nn);                 // 2 * half
  __shared__ double red[32];
  const int half = nn / 2, m = nn - 1;
  const unsigned nb = gridDim.x;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  // V = I; rotation inputs of round 0 from A
  for (int64_t e = gtid; e < (int64_t)nn * nn; e += gstride) {
    int64_t i = e % nn, j = e / nn;
    V[e] = (i == j) ? T(1) : T(0);
  }
  for (int64_t k = gtid; k < half; k += gstride) {
    int p, q;
    pair_members(0, m, (int)k, &p, &q);
    rin[3 * k + 0] = __ldcg(&A[p + (int64_t)nn * p]);
    rin[3 * k + 1] = __ldcg(&A[q + (int64_t)nn * q]);
    rin[3 * k + 2] = __ldcg(&A[p + (int64_t)nn * q]);
  }
  if (!grid_sync(bar, bar + 1, nb, flags)) return;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // convergence: off-diagonal vs diagonal mass (all CTAs reach the same verdict)
    double off = 0.0, dia = 0.0;
    for (int64_t e = gtid; e < (int64_t)nn * nn; e += gstride) {
      int64_t i = e % nn, j = e / nn;
      double v = (double)__ldcg(&A[e]);
      if (i == j) dia += v * v; else off += v * v;
    }
    off = block_sum(off, red);
    dia = block_sum(dia, red);
    if (threadIdx.x == 0) { redpart[2 * blockIdx.x] = off; redpart[2 * blockIdx.x + 1] = dia; }
    if (!grid_sync(bar, bar + 1, nb, flags)) return;
    double to = 0.0, td = 0.0;
    for (unsigned b = 0; b < nb; ++b) { to += __ldcg(&redpart[2 * b]); td += __ldcg(&redpart[2 * b + 1]); }
    if (!grid_sync(bar, bar + 1, nb, flags)) return;
    if (to <= tol * tol * td || td == 0.0) break;
    for (int rd = 0; rd < m; ++rd) {
      const int par = (int)(((int64_t)sweep * m + rd) & 1);   // parity runs on across sweeps
      const T* rcur = rin + (int64_t)par * 3 * half;
      T* rnext = rin + (int64_t)(par ^ 1) * 3 * half;
      const int rdn = (rd + 1) % m;
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int p, q;
        pair_members(rd, m, k, &p, &q);
        T app = __ldcg(&rcur[3 * k]), aqq = __ldcg(&rcur[3 * k + 1]), apq = __ldcg(&rcur[3 * k + 2]);
        T c = 1, s = 0;
        if (apq != T(0) && fabs((double)apq) > tol * 1e-3 * sqrt(fabs((double)app * (double)aqq))) {
          T theta = (aqq - app) / (T(2) * apq);
          T t = (theta >= 0 ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
          c = T(1) / sqrt(t * t + T(1));
          s = t * c;
        }
        cs[2 * k] = c; cs[2 * k + 1] = s;
        pq[2 * k] = p; pq[2 * k + 1] = q;
      }
      __syncthreads();
      for (int64_t e = gtid; e < (int64_t)half * half; e += gstride) {
        int I = (int)(e % half), J = (int)(e / half);
        int pI = pq[2 * I], qI = pq[2 * I + 1], pJ = pq[2 * J], qJ = pq[2 * J + 1];
        T cI = cs[2 * I], sI = cs[2 * I + 1], cJ = cs[2 * J], sJ = cs[2 * J + 1];
        T* a00 = &A[pI + (int64_t)nn * pJ]; T* a01 = &A[pI + (int64_t)nn * qJ];
        T* a10 = &A[qI + (int64_t)nn * pJ]; T* a11 = &A[qI + (int64_t)nn * qJ];
        T b00 = __ldcg(a00), b01 = __ldcg(a01), b10 = __ldcg(a10), b11 = __ldcg(a11);
        T c00 = cJ * b00 - sJ * b01, c01 = sJ * b00 + cJ * b01;
        T c10 = cJ * b10 - sJ * b11, c11 = sJ * b10 + cJ * b11;
        T n00 = cI * c00 - sI * c10, n01 = cI * c01 - sI * c11;
        T n10 = sI * c00 + cI * c10, n11 = sI * c01 + cI * c11;
        *a00 = n00; *a01 = n01; *a10 = n10; *a11 = n11;
        // publish the inputs of next round's rotations that live in this block
        int rows[2] = {pI, qI}, cols[2] = {pJ, qJ};
        T vals[2][2] = {{n00, n01}, {n10, n11}};
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
          for (int y = 0; y < 2; ++y) {
            int i = rows[x], j = cols[y];
            if (i > j) continue;
            int ki, ri, kj, rj;
            pair_of(rdn, m, i, &ki, &ri);
            pair_of(rdn, m, j, &kj, &rj);
            if (i == j) rnext[3 * ki + ri] = vals[x][y];
            else if (ki == kj) rnext[3 * ki + 2] = vals[x][y];
          }
      }
      for (int64_t e = gtid; e < (int64_t)nn * half; e += gstride) {
        int64_t i = e % nn;
        int J = (int)(e / nn);
        int pJ = pq[2 * J], qJ = pq[2 * J + 1];
        T cJ = cs[2 * J], sJ = cs[2 * J + 1];
        T vp = __ldcg(&V[i + (int64_t)nn * pJ]), vq = __ldcg(&V[i + (int64_t)nn * qJ]);
        V[i + (int64_t)nn * pJ] = cJ * vp - sJ * vq;
        V[i + (int64_t)nn * qJ] = sJ * vp + cJ * vq;
      }
      if (!grid_sync(bar, bar + 1, nb, flags)) return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *sweeps_out = sweep;
    if (sweep >= max_sweeps) atomicOr(flags, kFlagEigNoConv);
  }
}

// Selection of the leading eigenpairs of a Jacobi result (A diagonalised, V its
// rotations, both nn x nn): rough order by diag(A), Rayleigh quotients
// v^T C v / v^T v in double against C64 for the top kk = k + 2, final order by
// them, sign fix (largest-magnitude entry positive) and the trace of C64.
template <typename T>
__global__ void k_eig_order(const T* __restrict__ A, int nn, int kk, int* __restrict__ order_out) {
  __shared__ int order[1024];
  __shared__ float dg[1024];
  for (int j = threadIdx.x; j < nn; j += blockDim.x) { order[j] = j; dg[j] = (float)A[j + (int64_t)nn * j]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < kk; ++i) {
      int best = i;
      for (int j = i + 1; j < nn; ++j)
        if (dg[order[j]] > dg[order[best]]) best = j;
      int t = order[i]; order[i] = order[best]; order[best] = t;
      order_out[i] = order[i];
    }
  }
}

template <typename T>
__global__ void k_eig_cv(const double* __restrict__ C64, int n, const T* __restrict__ V, int nn,
                         const int* __restrict__ order, int kk, double* __restrict__ CV) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * kk; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % n;
    int j = (int)(e / n);
    const T* v = V + (int64_t)nn * order[j];
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += C64[i + (int64_t)n * l] * (double)v[l];
    CV[e] = s;
  }
}

template <typename T>
__global__ void k_eig_final(const T* __restrict__ V, int nn, int n, const double* __restrict__ C64,
                            const int* __restrict__ order_in, int kk, const double* __restrict__ CV, int k,
                            double* __restrict__ ev_out, double* __restrict__ Q_out, double* __restrict__ trace_out) {
  __shared__ double red[32];
  __shared__ double rq[64];
  __shared__ int ord[64], pos[64];
  __shared__ int imax;
  for (int j = 0; j < kk; ++j) {
    const T* v = V + (int64_t)nn * order_in[j];
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double vi = (double)v[i];
      num += vi * CV[i + (int64_t)n * j];
      den += vi * vi;
    }
    num = block_sum(num, red);
    den = block_sum(den, red);
    if (threadIdx.x == 0) { rq[j] = den > 0 ? num / den : 0.0; ord[j] = order_in[j]; pos[j] = j; }
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
  for (int j = 0; j < k; ++j) {
    const T* v = V + (int64_t)nn * ord[j];
    if (threadIdx.x == 0) {
      double best = -1.0;
      int ib = 0;
      for (int i = 0; i < n; ++i) {
        double a = fabs((double)v[i]);
        if (a > best) { best = a; ib = i; }
      }
      imax = ib;
      ev_out[j] = rq[j];
    }
    __syncthreads();
    double sgn = v[imax] < T(0) ? -1.0 : 1.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) Q_out[i + (int64_t)n * j] = sgn * (double)v[i];
    __syncthreads();
  }
}

template <typename T>
static void eig_select(const T* A_ws, const T* V_ws, int nn, int n, const double* C64, int k, double* ev, double* Q,
                       double* trace, double* scratch, cudaStream_t s) {
  int kk = k + 2 < n ? k + 2 : n;
  int* order = (int*)scratch;                 // 64 ints
  double* CV = scratch + 64;                  // n x kk
  k_eig_order<T><<<1, 256, 0, s>>>(A_ws, nn, kk, order);
  int blocks = (int)std::min<int64_t>(((int64_t)n * kk + 127) / 128, 1024);
  k_eig_cv<T><<<blocks, 128, 0, s>>>(C64, n, V_ws, nn, order, kk, CV);
  k_eig_final<T><<<1, 256, 0, s>>>(V_ws, nn, n, C64, order, kk, CV, k, ev, Q, trace);
}

template <typename T>
__global__ void k_pad_copy(const T* __restrict__ C, int n, T* __restrict__ A, int nn) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)nn * nn; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % nn, j = e / nn;
    A[e] = (i < n && j < n) ? C[i + (int64_t)n * j] : T(0);
  }
}

// Eigen-decomposition of the n x n Gram (C64 double; Cc in type T) -> leading k
// eigenpairs (descending) into ev, Q (n x k double) and the trace.
template <typename T>
tdb_status eig_leading(const T* Cc, const double* C64, int n, int k, T* A_ws, T* V_ws, T* rin_ws, double* red_ws,
                       unsigned* bar, unsigned* flags, int* sweeps, double* ev, double* Q, double* trace,
                       double* scratch, cudaStream_t s) {
  int nn = (n + 1) & ~1;
  int blocks = (int)std::min<int64_t>(((int64_t)nn * nn + 255) / 256, 1024);
  k_pad_copy<T><<<blocks, 256, 0, s>>>(Cc, n, A_ws, nn);
  double tol = sizeof(T) == 8 ? 1e-15 : 1e-7;
  int max_sweeps = 40;
  int dev = 0;
  cudaGetDevice(&dev);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return TDB_ERR_UNSUPPORTED;
  size_t sm = (size_t)nn * sizeof(T) + (size_t)nn * sizeof(int);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_coop<T>, 256, sm);
  if (per_sm < 1) return TDB_ERR_UNSUPPORTED;
  int64_t work = (int64_t)(nn / 2) * (nn / 2) + (int64_t)nn * (nn / 2);
  int grid = (int)std::min<int64_t>((int64_t)nsm * std::min(per_sm, 2), std::max<int64_t>(1, (work + 255) / 256));
  cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  void* args[] = {(void*)&A_ws, (void*)&V_ws, (void*)&nn, (void*)&rin_ws, (void*)&red_ws, (void*)&bar,
                  (void*)&flags, (void*)&max_sweeps, (void*)&tol, (void*)&sweeps};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_jacobi_coop<T>, grid, 256, args, sm, s);
  if (e != cudaSuccess) return TDB_ERR_CUDA;
  eig_select<T>(A_ws, V_ws, nn, n, C64, k, ev, Q, trace, scratch, s);
  return TDB_OK;
}
template tdb_status eig_leading<float>(const float*, const double*, int, int, float*, float*, float*, double*,
                                       unsigned*, unsigned*, int*, double*, double*, double*, double*, cudaStream_t);
template tdb_status eig_leading<double>(const double*, const double*, int, int, double*, double*, double*, double*,
                                        unsigned*, unsigned*, int*, double*, double*, double*, double*, cudaStream_t);

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
  T tol = sizeof(T) == 8 ? T(1e-15) : T(1e-7);
  k_jacobi_small_full<T><<<1, 512, sm, s>>>(Cc, n, A_ws, V_ws, 40, tol, flags);
  int nn = (n + 1) & ~1;
  eig_select<T>(A_ws, V_ws, nn, n, C64, k, ev, Q, trace, scratch, s);
  return TDB_OK;
}
template tdb_status eig_leading_small<float>(const float*, const double*, int, int, float*, float*, unsigned*,
                                             double*, double*, double*, double*, cudaStream_t);
template tdb_status eig_leading_small<double>(const double*, const double*, int, int, double*, double*, unsigned*,
                                              double*, double*, double*, double*, cudaStream_t);

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
  k_scale_basis<<<blocks, 256, 0, s>>>(Q, w, n, r, U);
}

}  // namespace tdb
