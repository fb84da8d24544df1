// k_eig.cu - truncated-HOSVD spectra for the float compute types (Sec. 2.3 last
// paragraph, Sec. 2.5): the weighted mode-n Gram
//     C_n = W_n^{1/2} V_(n) W_{-n} V_(n)^T W_n^{1/2}
// formed as Vw_(n) Vw_(n)^T with Vw = V scaled by sqrt(w_1 ... w_p) once, and its
// leading eigenpairs by block subspace iteration with Rayleigh-Ritz in one
// cooperative launch.
//
// Precision: products in float, 32-column chunk sums in float, chunks accumulated
// as float-float pairs (TwoSum), so the Gram carries the float rounding of the
// chunk sums and nothing coarser; the subspace iteration and Ritz values are float
// (eigenvalues to ~1e-7 of the largest, which resolves the energy fractions of
// Eq. 2.21 used by the rank rule), the eigenvectors are returned in double.
#include "common.cuh"
#include "kernels.h"

namespace tdb {

namespace {

constexpr int SY_T = 64;          // Gram output tile
constexpr int SY_K = 32;          // columns per chunk
constexpr int EIG_THREADS = 256;
constexpr int RB = 16;            // rows per row block in the eigensolver
constexpr int MMAX = 64;          // block size limit
constexpr int LDM = MMAX + 1;     // leading dimension of m x m float matrices in shared memory

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += err;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded grid barrier (monotonic counter zeroed before the launch; the k-th barrier
// waits for k * gridDim.x arrivals).
__device__ bool eig_grid_sync(unsigned* count, unsigned k, unsigned* flags, volatile int* abort_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_gpu(count, 1u);
    const unsigned target = k * gridDim.x;
    const long long t0 = clock64();
    while (ld_acquire_gpu(count) < target) {
      if (clock64() - t0 > 4000000000ll || (ld_acquire_gpu(flags) & kFlagTimeout)) {
        atomicOr(flags, kFlagTimeout);
        *abort_sh = 1;
        break;
      }
      __nanosleep(20);
    }
  }
  __syncthreads();
  return *abort_sh == 0;
}

__device__ __forceinline__ float hash_unit(uint32_t i, uint32_t j) {
  uint32_t h = i * 0x9E3779B1u ^ (j + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return (float)(h & 0xFFFFFF) / 8388608.0f - 1.0f;   // [-1, 1)
}

}  // namespace

// ---------------------------------------------------------------------------
// Vw = V * sqrt(w_1[i_1] ... w_p[i_p])   (ws[n] = sqrt(w_n) in float)
// ---------------------------------------------------------------------------
struct SqrtWeights {
  int p;
  int N[kMaxModes];
  const float* ws[kMaxModes];
};

__global__ void k_weight_data(const float* __restrict__ V, SqrtWeights sw, int S, float* __restrict__ Vw) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < S; e += gridDim.x * blockDim.x) {
    int rem = e;
    float f = 1.f;
    for (int n = 0; n < sw.p; ++n) {
      const int i = rem % sw.N[n];
      rem /= sw.N[n];
      f *= sw.ws[n][i];
    }
    Vw[e] = V[e] * f;
  }
}

__global__ void k_sqrt_weights(const double* __restrict__ w, int n, float* __restrict__ ws) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) ws[i] = (float)sqrt(w[i]);
}

// ---------------------------------------------------------------------------
// Gram tiles: blockIdx.x = upper tile pair (ti <= tj) of 64 x 64, blockIdx.y =
// column slice.  256 threads, 4 x 4 outputs each.  Column c of Vw_(n) is (l, q):
// Vw[l + L (i + N q)].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_syrk_partial(const float* __restrict__ Vw, int64_t L, int64_t Nn, int64_t Q,
                                                      int ntile, int ksplit, double* __restrict__ part) {
  int t = blockIdx.x, ti = 0;
  while (t >= ntile - ti) { t -= ntile - ti; ++ti; }
  const int tj = ti + t;
  const bool diag = (ti == tj);
  const int64_t i0 = (int64_t)ti * SY_T, j0 = (int64_t)tj * SY_T;
  const int64_t ncol = L * Q;
  const int64_t c0 = ncol * blockIdx.y / ksplit, c1 = ncol * (blockIdx.y + 1) / ksplit;
  __shared__ __align__(16) float As[SY_K][SY_T + 4];
  __shared__ __align__(16) float Bs[SY_K][SY_T + 4];
  const int tid = threadIdx.x;
  const int tr = tid & 15, tc = tid >> 4;       // output rows tr*4.., columns tc*4..
  const bool rows_fast = (L == 1);
  // load mapping: 8 elements per panel per thread.  With L == 1 the lanes run along
  // rows (contiguous) and column c is q = c; otherwise the lanes run along columns
  // (l contiguous) and each thread keeps its column's (l, q), advanced by 32 per chunk.
  const int ccol = tid & 31;
  int64_t lcur = 0, qcur = 0;
  if (!rows_fast) { lcur = (c0 + ccol) % L; qcur = (c0 + ccol) / L; }
  auto load = [&](int64_t cb, float* ra, float* rb) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      int ri;
      int64_t c, l, q;
      if (rows_fast) { ri = tid & 63; c = cb + (tid >> 6) + 4 * u; l = 0; q = c; }
      else { ri = (tid >> 5) + 8 * u; c = cb + ccol; l = lcur; q = qcur; }
      float va = 0.f, vb = 0.f;
      if (c < c1) {
        const int64_t ia = i0 + ri, ib = j0 + ri;
        if (ia < Nn) va = Vw[l + L * (ia + Nn * q)];
        if (!diag && ib < Nn) vb = Vw[l + L * (ib + Nn * q)];
      }
      ra[u] = va;
      rb[u] = vb;
    }
    if (!rows_fast) {
      lcur += SY_K;
      while (lcur >= L) { lcur -= L; ++qcur; }
    }
  };
  auto store = [&](const float* ra, const float* rb) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      int ri, cc;
      if (rows_fast) { ri = tid & 63; cc = (tid >> 6) + 4 * u; }
      else { cc = ccol; ri = (tid >> 5) + 8 * u; }
      As[cc][ri] = ra[u];
      if (!diag) Bs[cc][ri] = rb[u];
    }
  };
  float hi[16], lo[16];
#pragma unroll
  for (int x = 0; x < 16; ++x) { hi[x] = 0.f; lo[x] = 0.f; }
  float ra[8], rb[8];
  load(c0, ra, rb);
  for (int64_t cb = c0; cb < c1; cb += SY_K) {
    __syncthreads();
    store(ra, rb);
    __syncthreads();
    if (cb + SY_K < c1) load(cb + SY_K, ra, rb);
    const float (*Bp)[SY_T + 4] = diag ? As : Bs;
    float acc[16];
#pragma unroll
    for (int x = 0; x < 16; ++x) acc[x] = 0.f;
#pragma unroll 4
    for (int k = 0; k < SY_K; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&As[k][tr * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bp[k][tc * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x * 4 + y] = fmaf(av[x], bv[y], acc[x * 4 + y]);
    }
#pragma unroll
    for (int x = 0; x < 16; ++x) two_sum(hi[x], lo[x], acc[x]);
  }
  double* out = part + ((int64_t)blockIdx.x * ksplit + blockIdx.y) * SY_T * SY_T;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y)
      out[(tr * 4 + x) + SY_T * (tc * 4 + y)] = (double)hi[x * 4 + y] + (double)lo[x * 4 + y];
}

// Sum the slices: C64 (double) and Cc (float), both full n x n; trace of C64.
__global__ void k_syrk_finish(int64_t Nn, int ntile, int ksplit, const double* __restrict__ part,
                              double* __restrict__ C64, float* __restrict__ Cc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Nn * Nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % Nn, j = e / Nn;
    const int64_t a = i <= j ? i : j, b = i <= j ? j : i;
    const int ti = (int)(a / SY_T), tj = (int)(b / SY_T);
    const int pair = ti * ntile - ti * (ti - 1) / 2 + (tj - ti);
    int x = (int)(a % SY_T), y = (int)(b % SY_T);
    if (ti == tj && x > y) { const int t = x; x = y; y = t; }
    double s = 0.0;
    const double* src = part + (int64_t)pair * ksplit * SY_T * SY_T + x + SY_T * y;
#pragma unroll 8
    for (int k = 0; k < ksplit; ++k) s += src[(int64_t)k * SY_T * SY_T];
    C64[e] = s;
    Cc[e] = (float)s;
  }
}

// ---------------------------------------------------------------------------
// Eigensolver.  Every CTA owns row blocks of 16 rows (CTA b: blocks b, b + nb, ...).
// Iteration: Z <- C Q with Q = Z X and X^T (Z^T Z) X = I.  Each CTA sums the
// per-CTA partial Grams of Z itself, factors the m x m Gram, forms W = C Z for its
// rows, then Z' = W X and the partial Gram of Z' for its rows.  Z and the partials
// are double-buffered, so an iteration takes one grid barrier.  X comes from Gaussian elimination of the
// diagonally scaled Gram without pivoting: [G^ | I] -> [U | E], G^ = E^{-1} D_u E^{-T},
// X = D^{-1} E^T D_u^{-1/2} (shifted diagonal retried if a pivot fails).  Every CTA
// runs the same instructions on the same data, so all hold the same X.
// ---------------------------------------------------------------------------
struct EigArgs {
  const float* C;        // n x n (ld n), symmetric
  const double* C64;     // n x n, for the trace
  int n, m, k, iters;
  float* Z[2];           // n x m, row-major (ld ldz, the padding columns zero), ping-pong
  float* W;              // the Ritz vectors at the end, n x k row-major
  int ldz;               // m rounded up to a multiple of 4 (16-byte rows)
  float* Gp[2];          // nb x gstride partial Grams (m x m, column-major), ping-pong
  int gstride;           // m * m rounded up to a multiple of 4
  float* Xg;             // m x k: X S of the Rayleigh-Ritz step
  double* ev;            // k eigenvalues, descending
  double* Qout;          // n x k eigenvectors
  double* trace;
  unsigned* bar;
  unsigned* flags;
  int c_resident;        // one row block per CTA and all of Z staged at once: C rows loaded once
};

__device__ __forceinline__ float frcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float frsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void named_bar(int id, int nthr) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthr) : "memory");
}

// out[e] = sum over CTAs c = 0 .. nb-1 of Gp[c * gstride + e] for the m x m entries,
// stored to Gs[i + LDM j]; float4 loads, eight partials in flight, fixed order.
__device__ void sum_gram(const float* __restrict__ Gp, int nb, int gstride, int m, float* Gs) {
  const int q4 = gstride / 4;
  const float4* p = reinterpret_cast<const float4*>(Gp);
  for (int q = threadIdx.x; q < q4; q += blockDim.x) {
    float4 acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    int c = 0;
    for (; c + 7 < nb; c += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 v = __ldcg(&p[(int64_t)(c + u) * q4 + q]);
        acc[u].x += v.x; acc[u].y += v.y; acc[u].z += v.z; acc[u].w += v.w;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (c + u < nb) {
        const float4 v = __ldcg(&p[(int64_t)(c + u) * q4 + q]);
        acc[u].x += v.x; acc[u].y += v.y; acc[u].z += v.z; acc[u].w += v.w;
      }
#pragma unroll
    for (int u = 1; u < 8; u += 2) {
      acc[u - 1].x += acc[u].x; acc[u - 1].y += acc[u].y; acc[u - 1].z += acc[u].z; acc[u - 1].w += acc[u].w;
    }
    const float r[4] = {(acc[0].x + acc[2].x) + (acc[4].x + acc[6].x), (acc[0].y + acc[2].y) + (acc[4].y + acc[6].y),
                        (acc[0].z + acc[2].z) + (acc[4].z + acc[6].z), (acc[0].w + acc[2].w) + (acc[4].w + acc[6].w)};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = 4 * q + u;
      if (e < m * m) Gs[(e % m) + LDM * (e / m)] = r[u];
    }
  }
}

// X (upper triangular, Xs[i + LDM j]) from the Gram Gs, on all EIG_THREADS threads.
// R is the augmented matrix [G^ | I] (m x 2m, element (i, cc) at R[i + LDM cc], the
// identity block from column m on); Gaussian elimination below the diagonal turns it
// into [U | E] with E = L^{-1}.  Step k updates the contiguous window of columns
// k+1 .. k+m (U right of the pivot, then E up to column k): lane l owns rows l and
// l + 32, warp w the window columns w, w + 8, ...; the pivot row's and the own row's
// entries are loaded into registers before the stores.  (The elimination is a chain of
// m dependent steps; with one warp per SM sub-partition its instruction latency, not
// its arithmetic, sets the time, so it runs on every warp of the CTA.)  A pivot that
// is not positive restarts the elimination with a shifted diagonal (1e-5, then 1e-2:
// the block's tail columns sit below the float resolution of the spectrum); on the
// last attempt such a column is skipped and its column of X is zero.  Every thread
// reads the same pivots after a barrier, so the decisions are uniform.
constexpr int FW = EIG_THREADS / 32;
__device__ void eig_factor(int m, const float* Gs, float* R, float* Xs, float* dsc, unsigned* flags) {
  constexpr int CPT = MMAX / FW;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int i = t; i < m; i += EIG_THREADS) {
    const float g = Gs[i + LDM * i];
    dsc[i] = g > 0.f ? rsqrtf(g) : 1.f;
  }
  bool ok = false;
  for (int attempt = 0; attempt < 3 && !ok; ++attempt) {
    const float shift = attempt == 0 ? 0.f : (attempt == 1 ? 1e-5f : 1e-2f);
    __syncthreads();
    for (int i = lane; i < m; i += 32)
#pragma unroll
      for (int j = 0; j < 2 * CPT; ++j) {
        const int cc = w + FW * j;
        if (cc < 2 * m)
          R[i + LDM * cc] = cc < m ? Gs[i + LDM * cc] * dsc[i] * dsc[cc] + (i == cc ? shift : 0.f)
                                   : (cc - m == i ? 1.f : 0.f);
      }
    __syncthreads();
    ok = true;
    for (int k = 0; k < m; ++k) {
      const float piv = R[k + LDM * k];
      if (!(piv > 1e-30f)) {
        ok = false;
        if (attempt < 2) break;
        continue;
      }
      const float ip = 1.f / piv;
      float prow[CPT];
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int off = w + FW * j;                    // window column k + 1 + off
        prow[j] = off < m ? R[k + LDM * (k + 1 + off)] : 0.f;
      }
      // rows below k: row_i -= (a_ik / a_kk) row_k over the window
      for (int i = k + 1 + lane; i < m; i += 32) {
        const float f = R[i + LDM * k] * ip;
        float rv[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int off = w + FW * j;
          rv[j] = off < m ? R[i + LDM * (k + 1 + off)] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int off = w + FW * j;
          if (off < m) R[i + LDM * (k + 1 + off)] = fmaf(-f, prow[j], rv[j]);
        }
      }
      __syncthreads();
    }
  }
  if (!ok && t == 0) atomicOr(flags, kFlagEigNoConv);
  // X[i][j] = dsc[i] * E[j][i] / sqrt(u_jj) with E[j][i] = R(j, m + i) (upper triangular;
  // zero for a skipped pivot); every load before the first store
  float xv[2][CPT];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
#pragma unroll
    for (int jj = 0; jj < CPT; ++jj) {
      const int j = w + FW * jj;
      float x = 0.f;
      if (i < m && j < m && j >= i) {
        const float u = R[j + LDM * j];
        x = dsc[i] * R[j + LDM * (m + i)] * (u > 0.f ? rsqrtf(u) : 0.f);
      }
      xv[h][jj] = x;
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
#pragma unroll
    for (int jj = 0; jj < CPT; ++jj) {
      const int j = w + FW * jj;
      if (i < m && j < m) Xs[i + LDM * j] = xv[h][jj];
    }
  }
}

// Rows [r0, r0 + RB): Wr = C[rows, :] Zin (RB x m, ld LDM) on threads [t0, t0 + ng).
// Zin is staged in shared memory (chunks of ZCH rows), C rows in [RB][ZCH + 1]
// (kept across calls when load_c is false).  Thread layout: row quad rq (4), column
// quad cq (mq), l-split ls (4 x 4 outputs, 16 FMAs per 5 shared loads); partial sums
// reduced in shared memory.
__device__ void eig_rows_cz(const EigArgs& a, const float* __restrict__ Zin, int r0, float* Wr, float* sm, int ZCH,
                            int t0, int ng, bool load_c) {
  const int n = a.n, m = a.m, lt = threadIdx.x - t0;
  const int mq = (m + 3) / 4, mp = mq * 4;
  float* Zs = sm;                         // ZCH x mp
  float* Cs = Zs + ZCH * mp;              // RB x (ZCH + 1)
  float* Rs = Cs + RB * (ZCH + 1);        // reduction: nls x RB x mp
  const int nthr_rc = 4 * mq;
  const int nls = ng / nthr_rc;
  const int rq = lt % 4, cq = (lt / 4) % mq, ls = lt / nthr_rc;
  float acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
  for (int l0 = 0; l0 < n; l0 += ZCH) {
    const int lc = min(ZCH, n - l0);
    if (l0 > 0) named_bar(1, ng);
    {
      // Z rows l0 .. l0+lc-1 are one contiguous block of lc * ldz floats (ldz == mp)
      const float4* src = (const float4*)(Zin + (int64_t)l0 * a.ldz);
      float4* dst = (float4*)Zs;
      const int nf4 = lc * mp / 4;
#pragma unroll 4
      for (int e = lt; e < nf4; e += ng) dst[e] = __ldcg(&src[e]);
    }
    if (load_c || ZCH < n) {
      if ((n & 3) == 0) {            // rows of C (= columns, C symmetric) as float4 runs
        const int q4 = lc / 4;
#pragma unroll 4
        for (int e = lt; e < RB * q4; e += ng) {
          const int rr = e / q4, l4 = e % q4;
          const int row = r0 + rr;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (row < n) v = __ldcg((const float4*)(a.C + (int64_t)row * n + l0) + l4);
          float* d = Cs + rr * (ZCH + 1) + 4 * l4;
          d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
        }
      } else {
#pragma unroll 4
        for (int e = lt; e < RB * lc; e += ng) {
          const int rr = e / lc, l = e % lc;
          const int row = r0 + rr;
          Cs[rr * (ZCH + 1) + l] = (row < n) ? __ldcg(&a.C[(int64_t)row * n + l0 + l]) : 0.f;
        }
      }
    }
    named_bar(1, ng);
    if (ls < nls) {
      const int lb = lc * ls / nls, le = lc * (ls + 1) / nls;
#pragma unroll 4
      for (int l = lb; l < le; ++l) {
        const float4 z = *reinterpret_cast<const float4*>(&Zs[l * mp + cq * 4]);
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const float cx = Cs[(4 * rq + x) * (ZCH + 1) + l];
          acc[x][0] = fmaf(cx, z.x, acc[x][0]); acc[x][1] = fmaf(cx, z.y, acc[x][1]);
          acc[x][2] = fmaf(cx, z.z, acc[x][2]); acc[x][3] = fmaf(cx, z.w, acc[x][3]);
        }
      }
    }
  }
  if (ls < nls)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) Rs[(ls * RB + 4 * rq + x) * mp + cq * 4 + y] = acc[x][y];
  named_bar(1, ng);
  for (int e = lt; e < RB * m; e += ng) {
    const int rr = e % RB, c = e / RB;
    float s = 0.f;
    for (int q = 0; q < nls; ++q) s += Rs[(q * RB + rr) * mp + c];
    Wr[rr * LDM + c] = s;
  }
}

// Ga (+)= Ar^T Br over the RB staged rows (m x m, column-major, all entries).
__device__ void rows_gram(int m, const float* Ar, const float* Br, float* Ga, bool accumulate) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e % m, j = e / m;
    float s = 0.f;
#pragma unroll 4
    for (int rr = 0; rr < RB; ++rr) s = fmaf(Ar[rr * LDM + i], Br[rr * LDM + j], s);
    Ga[e] = accumulate ? Ga[e] + s : s;
  }
}

__device__ void store_gram(int m, int gstride, const float* Ga, bool any, float* dst) {
  for (int e = threadIdx.x; e < gstride; e += blockDim.x) dst[e] = (any && e < m * m) ? Ga[e] : 0.f;
}

// Convergence of the block (one warp): with Z = C Q and Q orthonormal, the diagonally
// scaled Gram of Z is the identity once the leading columns of Q are eigenvectors
// (C q_i . C q_j = 0), and its off-diagonal entry (i, j) is of the order of the mixing
// of q_i and q_j otherwise.  Converged when every pair among the first k columns is
// below 2e-6 (the rounding of the float Gram) plus 3e-6 sqrt(G_00 / min(G_ii, G_jj)):
// C q_j carries float rounding of ~1e-6 of the largest eigenvalue, so a column of
// eigenvalue lambda_j is resolved to ~1e-6 lambda_1 / lambda_j at best.
constexpr int kMinIters = 4;
__device__ bool gram_converged(int m, int k, const float* Gs) {
  const int lane = threadIdx.x & 31;
  const float g00 = Gs[0];
  const int kk = min(k, m);
  bool ok = g00 > 0.f;
  for (int e = lane; e < kk * kk; e += 32) {
    const int i = e % kk, j = e / kk;
    if (i >= j) continue;
    const float gi = Gs[i + LDM * i], gj = Gs[j + LDM * j];
    const float gmin = fminf(gi, gj);
    if (!(gmin > 0.f)) { ok = false; continue; }
    const float aij = fabsf(Gs[i + LDM * j]) * rsqrtf(gi) * rsqrtf(gj);
    const float tol = 2e-6f + 3e-6f * sqrtf(g00 / gmin);
    if (!(aij <= tol)) ok = false;
  }
  return __all_sync(0xffffffffu, ok);
}

// Shared-memory layout of the kernel (floats): the m x m work area, then the C Z area.
constexpr int EIG_WORK_FLOATS = 5 * MMAX * LDM + 2 * RB * LDM;

__global__ void __launch_bounds__(EIG_THREADS, 1) k_eig_si(EigArgs a, int ZCH) {
  extern __shared__ __align__(16) float smf[];
  __shared__ int abort_sh, conv_sh;
  __shared__ float dsc[MMAX];
  if (threadIdx.x == 0) abort_sh = 0;
  __syncthreads();
  const int n = a.n, m = a.m, tid = threadIdx.x;
  const int nrb = (n + RB - 1) / RB;
  const int nb = gridDim.x, b = blockIdx.x;
  float* Gs = smf;                        // summed Gram (Rayleigh-Ritz: M)
  float* As = Gs + MMAX * LDM;            // elimination [G^ | I]: 2 MMAX columns (H)
  float* Es = As + MMAX * LDM;            // (second half of the above; Jacobi vectors)
  float* Xs = Es + MMAX * LDM;            // X, kept to the Rayleigh-Ritz step
  float* Ga = Xs + MMAX * LDM;            // this CTA's partial Gram (small scratch)
  float* Wr = Ga + MMAX * LDM;            // RB x m rows of C Z
  float* Zr = Wr + RB * LDM;              // RB x m rows of Z
  float* czs = smf + EIG_WORK_FLOATS;     // C Z staging
  unsigned nbar = 0;
  // start: Z = hash columns (a function of the indices only, so the result depends on
  // C alone), partial Grams into Gp[0]
  bool any = false;
  for (int rb = b; rb < nrb; rb += nb) {
    const int r0 = rb * RB;
    for (int e = tid; e < RB * a.ldz; e += blockDim.x) {
      const int rr = e % RB, c = e / RB;
      const int row = r0 + rr;
      const float v = (row < n && c < m) ? hash_unit((uint32_t)row, (uint32_t)c) : 0.f;
      if (c < m) Zr[rr * LDM + c] = v;
      if (row < n) a.Z[0][(int64_t)row * a.ldz + c] = v;
    }
    __syncthreads();
    rows_gram(m, Zr, Zr, Ga, any);
    __syncthreads();
    any = true;
  }
  store_gram(m, a.gstride, Ga, any, a.Gp[0] + (int64_t)b * a.gstride);
  if (!eig_grid_sync(a.bar, ++nbar, a.flags, &abort_sh)) return;
  int it_last = a.iters;                  // the iteration that prepares the Rayleigh-Ritz step
  bool conv_prev = false;
  for (int it = 0; it <= it_last; ++it) {
    const int cur = it & 1;
    const float* Zc = a.Z[cur];
    sum_gram(a.Gp[cur], nb, a.gstride, m, Gs);
    __syncthreads();
    if (it >= kMinIters && it < it_last) {
      // convergence (every CTA holds the same Gram, so all take the same decision)
      if (tid < 32) {
        const bool c = gram_converged(m, a.k, Gs);
        if (tid == 0) conv_sh = c ? 1 : 0;
      }
      __syncthreads();
      const bool conv = conv_sh != 0;
      if (conv && conv_prev) it_last = it;
      conv_prev = conv;
    }
    any = false;
    for (int rb = b; rb < nrb; rb += nb) {
      const int r0 = rb * RB;
      if (!any) {
        eig_factor(m, Gs, As, Xs, dsc, a.flags);
        __syncthreads();
      }
      eig_rows_cz(a, Zc, r0, Wr, czs, ZCH, 0, EIG_THREADS, !(a.c_resident && it > 0));
      __syncthreads();
      if (it < it_last) {
        // Z' = W X for these rows (X upper), and their partial Gram
        float* Zn = a.Z[cur ^ 1];
        for (int e = tid; e < RB * a.ldz; e += blockDim.x) {
          const int rr = e % RB, c = e / RB;
          float s = 0.f;
          if (c < m) {
            for (int l = 0; l <= c; ++l) s = fmaf(Wr[rr * LDM + l], Xs[l + LDM * c], s);
            Zr[rr * LDM + c] = s;
          }
          if (r0 + rr < n) Zn[(int64_t)(r0 + rr) * a.ldz + c] = s;
        }
        __syncthreads();
        rows_gram(m, Zr, Zr, Ga, any);
      } else {
        // Rayleigh-Ritz: partial M = Z^T W = Z^T C Z
        for (int e = tid; e < RB * m; e += blockDim.x) {
          const int rr = e % RB, c = e / RB;
          Zr[rr * LDM + c] = (r0 + rr < n) ? __ldcg(&Zc[(int64_t)(r0 + rr) * a.ldz + c]) : 0.f;
        }
        __syncthreads();
        rows_gram(m, Zr, Wr, Ga, any);
      }
      __syncthreads();
      any = true;
    }
    if (!any) eig_factor(m, Gs, As, Xs, dsc, a.flags);   // (no rows: keeps X defined)
    store_gram(m, a.gstride, Ga, any, a.Gp[cur ^ 1] + (int64_t)b * a.gstride);
    if (!eig_grid_sync(a.bar, ++nbar, a.flags, &abort_sh)) return;
  }
  const int fin = it_last & 1;            // Z[fin] is the final block; Gp[fin ^ 1] holds M
  // trace of C (double), on another CTA while CTA 0 runs the Rayleigh-Ritz step
  if (b == (nb > 1 ? 1 : 0) && tid < 32) {
    double t = 0.0;
#pragma unroll 8
    for (int i = tid; i < n; i += 32) t += __ldcg(&a.C64[i + (int64_t)n * i]);
    t = warp_sum(t);
    if (tid == 0) *a.trace = t;
  }
  // CTA 0: H = X^T M X, Jacobi, ordering; P = X S[:, order] into Xg
  if (b == 0) {
    float* Ms = Gs;
    float* Hs = As;
    float* Vs = Es;
    float* cs = Ga;                       // 2 * MMAX
    int* pq = (int*)(cs + 2 * MMAX);      // 2 * MMAX
    int* ord = pq + 2 * MMAX;             // MMAX
    float* red = (float*)(ord + MMAX);    // 64
    sum_gram(a.Gp[fin ^ 1], nb, a.gstride, m, Ms);
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {          // Vs = M X (temporary)
      const int i = e % m, j = e / m;
      float s = 0.f;
      for (int l = 0; l <= j; ++l) s = fmaf(Ms[i + LDM * l], Xs[l + LDM * j], s);
      Vs[i + LDM * j] = s;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {          // H = X^T (M X), symmetrised below
      const int i = e % m, j = e / m;
      float s = 0.f;
      for (int l = 0; l <= i; ++l) s = fmaf(Xs[l + LDM * i], Vs[l + LDM * j], s);
      Hs[i + LDM * j] = s;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = e % m, j = e / m;
      if (i < j) {
        const float h = 0.5f * (Hs[i + LDM * j] + Hs[j + LDM * i]);
        Hs[i + LDM * j] = h;
        Hs[j + LDM * i] = h;
      }
    }
    __syncthreads();
    // cyclic Jacobi (Brent-Luk ordering) on H, eigenvectors in Vs
    const int nn = (m + 1) & ~1, half = nn / 2;
    for (int e = tid; e < nn * nn; e += blockDim.x) {
      const int i = e % nn, j = e / nn;
      if (i >= m || j >= m) Hs[i + LDM * j] = 0.f;
      Vs[i + LDM * j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    const float tol = 1e-6f, thr = 1e-9f;
    float off_prev = 0.f;
    // the 2 x 2 blocks (I, J) and the V entries (i, J) of this thread, the same in every
    // round (packed I | J << 8; -1 for none): no index arithmetic inside the rounds
    const int nb2 = half * half, nv = nn * half;
    int blk[4], vent[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + EIG_THREADS * u;
      blk[u] = e < nb2 ? ((e % half) | ((e / half) << 8)) : -1;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + EIG_THREADS * u;
      vent[u] = e < nv ? ((e % nn) | ((e / nn) << 8)) : -1;
    }
    for (int sweep = 0; sweep < 40; ++sweep) {
      float off = 0.f, dia = 0.f;
      for (int e = tid; e < nn * nn; e += blockDim.x) {
        const int i = e % nn, j = e / nn;
        const float v = Hs[i + LDM * j];
        if (i == j) { if (i < a.k) dia += v * v; }
        else if (i < a.k || j < a.k) off += v * v;
      }
      off = warp_sum(off);
      dia = warp_sum(dia);
      if ((tid & 31) == 0) { red[tid >> 5] = off; red[8 + (tid >> 5)] = dia; }
      __syncthreads();
      off = 0.f;
      dia = 0.f;
      for (int w = 0; w < EIG_THREADS / 32; ++w) { off += red[w]; dia += red[8 + w]; }
      __syncthreads();
      if (off <= tol * tol * dia || dia == 0.f) break;
      if (sweep >= 3 && off > 0.5f * off_prev) break;
      off_prev = off;
      for (int rd = 0; rd < nn - 1; ++rd) {
        if (tid < half) {
          const int k = tid;
          int p = rd, q = nn - 1;
          if (k > 0) {
            p = rd + k;
            if (p >= nn - 1) p -= nn - 1;
            q = rd - k;
            if (q < 0) q += nn - 1;
          }
          const float app = Hs[p + LDM * p], aqq = Hs[q + LDM * q], apq = Hs[p + LDM * q];
          float c = 1.f, s = 0.f;
          // pairs within the block's tail (columns k.. of Q, below the wanted eigenpairs)
          // are left alone: only the leading k rows and columns must be diagonalised
          if ((p < a.k || q < a.k) && apq != 0.f && apq * apq > thr * thr * fabsf(app * aqq)) {
            // t = sign(theta) / (|theta| + sqrt(theta^2 + 1)) with approximate reciprocals:
            // c = 1 / sqrt(1 + t^2), s = t c keep c^2 + s^2 = 1 whatever t's rounding
            const float theta = (aqq - app) * frcp_approx(2.f * apq);
            const float at = fabsf(theta);
            const float x = fmaf(at, at, 1.f);
            const float root = (at < 1e18f) ? x * frsqrt_approx(x) : at;
            const float tt = copysignf(frcp_approx(at + root), theta);
            c = frsqrt_approx(fmaf(tt, tt, 1.f));
            s = tt * c;
          }
          cs[2 * k] = c;
          cs[2 * k + 1] = s;
          pq[2 * k] = p;
          pq[2 * k + 1] = q;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (blk[u] < 0) continue;
          const int I = blk[u] & 255, J = blk[u] >> 8;
          const int pI = pq[2 * I], qI = pq[2 * I + 1], pJ = pq[2 * J], qJ = pq[2 * J + 1];
          const float cI = cs[2 * I], sI = cs[2 * I + 1], cJ = cs[2 * J], sJ = cs[2 * J + 1];
          const float b00 = Hs[pI + LDM * pJ], b01 = Hs[pI + LDM * qJ], b10 = Hs[qI + LDM * pJ], b11 = Hs[qI + LDM * qJ];
          const float c00 = cJ * b00 - sJ * b01, c01 = sJ * b00 + cJ * b01;
          const float c10 = cJ * b10 - sJ * b11, c11 = sJ * b10 + cJ * b11;
          Hs[pI + LDM * pJ] = cI * c00 - sI * c10;
          Hs[pI + LDM * qJ] = cI * c01 - sI * c11;
          Hs[qI + LDM * pJ] = sI * c00 + cI * c10;
          Hs[qI + LDM * qJ] = sI * c01 + cI * c11;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (vent[u] < 0) continue;
          const int i = vent[u] & 255, J = vent[u] >> 8;
          const int pJ = pq[2 * J], qJ = pq[2 * J + 1];
          const float cJ = cs[2 * J], sJ = cs[2 * J + 1];
          const float vp = Vs[i + LDM * pJ], vq = Vs[i + LDM * qJ];
          Vs[i + LDM * pJ] = cJ * vp - sJ * vq;
          Vs[i + LDM * qJ] = sJ * vp + cJ * vq;
        }
        __syncthreads();
      }
    }
    // descending order of the Ritz values: ranks of order-preserving integer keys of the
    // float bits, ties by index, so the ranks are a permutation whatever the values
    // (a NaN included) and every ord[] entry is written
    auto fkey = [](float v) {
      const int b = __float_as_int(v);
      return b >= 0 ? b : (b ^ 0x7fffffff);
    };
    for (int j = tid; j < m; j += blockDim.x) {
      const int kj = fkey(Hs[j + LDM * j]);
      int rank = 0;
      for (int l = 0; l < m; ++l) {
        const int kl = fkey(Hs[l + LDM * l]);
        rank += (kl > kj) || (kl == kj && l < j);
      }
      ord[rank] = j;
    }
    __syncthreads();
    for (int j = tid; j < a.k; j += blockDim.x) a.ev[j] = (double)Hs[ord[j] + LDM * ord[j]];
    for (int e = tid; e < m * a.k; e += blockDim.x) {        // P = X S[:, ord[:k]] -> Xg (m x k)
      const int i = e % m, j = e / m;
      const int oj = ord[j];
      float s = 0.f;
      for (int l = i; l < m; ++l) s = fmaf(Xs[i + LDM * l], Vs[l + LDM * oj], s);
      a.Xg[i + m * j] = s;
    }
  }
  if (!eig_grid_sync(a.bar, ++nbar, a.flags, &abort_sh)) return;
  // Ritz vectors Y = Z P (n x k) into W; per-CTA column norms^2 and largest |entry|
  float* colnorm = a.Gp[fin];                                 // [cta][k] norms, [cta][MMAX + k] max |y|, index as float bits
  {
    const float* Zf = a.Z[fin];
    float* Ps = Gs;                       // m x k (ld LDM)
    float* Zs = Zr;                       // RB x m
    float* Ys = Wr;                       // RB x k
    float* nrm = Ga;                      // k
    float* mx = nrm + MMAX;               // k
    int* ix = (int*)(mx + MMAX);          // k
    for (int j = tid; j < a.k; j += blockDim.x) { nrm[j] = 0.f; mx[j] = -1.f; ix[j] = 0x7fffffff; }
    for (int e = tid; e < m * a.k; e += blockDim.x) Ps[(e % m) + LDM * (e / m)] = __ldcg(&a.Xg[e]);
    __syncthreads();
    for (int rb = b; rb < nrb; rb += nb) {
      const int r0 = rb * RB;
      for (int e = tid; e < RB * m; e += blockDim.x) {
        const int rr = e % RB, c = e / RB;
        Zs[rr * LDM + c] = (r0 + rr < n) ? __ldcg(&Zf[(int64_t)(r0 + rr) * a.ldz + c]) : 0.f;
      }
      __syncthreads();
      for (int e = tid; e < RB * a.k; e += blockDim.x) {
        const int rr = e % RB, j = e / RB;
        float s = 0.f;
        for (int l = 0; l < m; ++l) s = fmaf(Zs[rr * LDM + l], Ps[l + LDM * j], s);
        Ys[rr * LDM + j] = s;
        if (r0 + rr < n) a.W[(int64_t)(r0 + rr) * a.k + j] = s;
      }
      __syncthreads();
      for (int j = tid; j < a.k; j += blockDim.x) {
        for (int rr = 0; rr < RB && r0 + rr < n; ++rr) {
          const float y = Ys[rr * LDM + j];
          nrm[j] = fmaf(y, y, nrm[j]);
          const float ay = fabsf(y);
          if (ay > mx[j]) { mx[j] = ay; ix[j] = r0 + rr; }
        }
      }
      __syncthreads();
    }
    for (int j = tid; j < a.k; j += blockDim.x) {
      colnorm[(int64_t)b * 3 * MMAX + j] = nrm[j];
      colnorm[(int64_t)b * 3 * MMAX + MMAX + j] = mx[j];
      colnorm[(int64_t)b * 3 * MMAX + 2 * MMAX + j] = __int_as_float(ix[j]);
    }
  }
  if (!eig_grid_sync(a.bar, ++nbar, a.flags, &abort_sh)) return;
  // every CTA: the column scales (1 / norm with the sign making the largest |entry|
  // positive; first index on ties), then its rows of Qout in double
  {
    float* scale = Ga;                    // k
    for (int j = tid; j < a.k; j += blockDim.x) {
      float nr = 0.f, best = -1.f;
      int bi = 0x7fffffff;
      for (int c = 0; c < nb; ++c) {
        nr += __ldcg(&colnorm[(int64_t)c * 3 * MMAX + j]);
        const float v = __ldcg(&colnorm[(int64_t)c * 3 * MMAX + MMAX + j]);
        const int ii = __float_as_int(__ldcg(&colnorm[(int64_t)c * 3 * MMAX + 2 * MMAX + j]));
        if (v > best || (v == best && ii < bi)) { best = v; bi = ii; }
      }
      const float ybi = (bi < n) ? __ldcg(&a.W[(int64_t)bi * a.k + j]) : 1.f;
      scale[j] = (ybi < 0.f ? -1.f : 1.f) * (nr > 0.f ? rsqrtf(nr) : 1.f);
    }
    __syncthreads();
    for (int rb = b; rb < nrb; rb += nb)
      for (int e = tid; e < RB * a.k; e += blockDim.x) {
        const int rr = e % RB, j = e / RB, row = rb * RB + rr;
        if (row < n) a.Qout[row + (int64_t)n * j] = (double)(__ldcg(&a.W[(int64_t)row * a.k + j]) * scale[j]);
      }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
void launch_sqrt_weights(const double* w, int n, float* ws, cudaStream_t s) {
  k_sqrt_weights<<<std::max(1, std::min((n + 255) / 256, 64)), 256, 0, s>>>(w, n, ws);
  count_launch();
}

void launch_weight_data(const float* V, int p, const int64_t* N, const float* const* ws, int64_t S, float* Vw,
                        cudaStream_t s) {
  SqrtWeights sw;
  sw.p = p;
  for (int n = 0; n < kMaxModes; ++n) {
    sw.N[n] = n < p ? (int)N[n] : 1;
    sw.ws[n] = n < p ? ws[n] : nullptr;
  }
  const int blocks = (int)std::min<int64_t>((S + 255) / 256, 152 * 8);
  k_weight_data<<<blocks, 256, 0, s>>>(V, sw, (int)S, Vw);
  count_launch();
}

void launch_gram_weighted(const float* Vw, int64_t L, int64_t Nn, int64_t Q, double* part, size_t part_cap, double* C64,
                          float* Cc, cudaStream_t s) {
  const int ntile = (int)((Nn + SY_T - 1) / SY_T);
  const int npair = ntile * (ntile + 1) / 2;
  const int64_t ncol = L * Q;
  int ksplit = (int)std::max<int64_t>(1, std::min<int64_t>((152 + npair - 1) / npair, (ncol + 127) / 128));
  while ((size_t)npair * ksplit * SY_T * SY_T > part_cap && ksplit > 1) --ksplit;
  k_syrk_partial<<<dim3(npair, ksplit), 256, 0, s>>>(Vw, L, Nn, Q, ntile, ksplit, part);
  count_launch();
  const int blocks = (int)std::min<int64_t>((Nn * Nn + 255) / 256, 1024);
  k_syrk_finish<<<blocks, 256, 0, s>>>(Nn, ntile, ksplit, part, C64, Cc);
  count_launch();
}

size_t eig_si_scratch_floats(int n) {
  // Z (two buffers), Ritz vectors: n x MMAX each; partial Grams (two): 152 x MMAX^2; Xg: MMAX^2
  return (size_t)3 * n * MMAX + (size_t)2 * 152 * MMAX * MMAX + MMAX * MMAX;
}

tdb_status eig_si_float(const float* Cc, const double* C64, int n, int k, int iters, float* scratch, unsigned* bar,
                        unsigned* flags, double* ev, double* Q, double* trace, cudaStream_t s) {
  const int m = std::min(n, std::min(MMAX, k + 16));
  if (k > m || iters < 0) return TDB_ERR_INVALID_ARG;
  static int nsm = 0;
  static size_t smem_cap = 0;
  if (nsm == 0) {
    int dev = 0, coop = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) { nsm = 0; return TDB_ERR_UNSUPPORTED; }
    smem_cap = (size_t)optin - 2048;
  }
  const int mq = (m + 3) / 4, mp = mq * 4;
  const int nls = EIG_THREADS / (4 * mq);
  // C Z staging: ZCH rows of Z (a multiple of 16 when chunked, so float4 runs of C
  // rows stay aligned), C rows and the reduction buffer, after the m x m work area
  auto need = [&](int zch) {
    return ((size_t)EIG_WORK_FLOATS + (size_t)zch * mp + (size_t)RB * (zch + 1) + (size_t)nls * RB * mp) *
           sizeof(float);
  };
  int ZCH = n;
  while (ZCH > 64 && need(ZCH) > smem_cap) ZCH = ((ZCH / 2) + 15) & ~15;
  const size_t smem = need(ZCH);
  if (smem > smem_cap) return TDB_ERR_UNSUPPORTED;
  cudaFuncSetAttribute(k_eig_si, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eig_si, EIG_THREADS, smem);
  if (per_sm < 1) return TDB_ERR_UNSUPPORTED;
  const int nrb = (n + RB - 1) / RB;
  const int gstride = ((m * m + 3) / 4) * 4;
  // every CTA sums all partial Grams each iteration: bound their count
  const int cap = std::max(8, 131072 / gstride);
  const int grid = std::min(std::min(nsm, 152), std::min(nrb, cap));
  EigArgs a;
  a.C = Cc;
  a.C64 = C64;
  a.n = n;
  a.m = m;
  a.k = k;
  a.iters = iters;
  a.Z[0] = scratch;
  a.Z[1] = a.Z[0] + (size_t)n * MMAX;
  a.W = a.Z[1] + (size_t)n * MMAX;
  a.ldz = mp;
  a.Gp[0] = a.W + (size_t)n * MMAX;
  a.Gp[1] = a.Gp[0] + (size_t)152 * MMAX * MMAX;
  a.gstride = gstride;
  a.Xg = a.Gp[1] + (size_t)152 * MMAX * MMAX;
  a.ev = ev;
  a.Qout = Q;
  a.trace = trace;
  a.bar = bar;
  a.flags = flags;
  a.c_resident = (ZCH >= n && grid == nrb) ? 1 : 0;
  cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
  void* args[] = {(void*)&a, (void*)&ZCH};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_eig_si, grid, EIG_THREADS, args, smem, s);
  count_launch();
  return e == cudaSuccess ? TDB_OK : TDB_ERR_CUDA;
}

}  // namespace tdb
