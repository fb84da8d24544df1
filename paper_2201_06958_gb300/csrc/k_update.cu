// k_update.cu - the rank-sized algebra of one step in one cooperative launch.
//
// Rows of every mode are split in tiles of 32 over all CTAs, r x r work runs on
// one CTA per mode, and bounded grid barriers separate the phases.  Tc is the
// compute type (float or double); the state (U, T, R, R^{-1}, G^{-1}) is double.
//   1 rows : M = Y_(n) T_(n)^T, X = M G_n^{-1}, partial P = A^T X with A = W U   (Tc)
//            (pseudo-inverse and complement projector, Sec. 2.2; Eq. 2.16 times dt)
//   2 rows : P_n = sum of the partials, E = X - U P_n (Tc), U' = U + E (double;
//            Euler step, Sec. 2.3), partial C = U'^T W U' (Tc)
//   3 mode : C_n = R^T R and R^{-1} (weighted Cholesky-QR, the reading used to keep
//            Eq. 2.6 through the step)
//   4 rows : U'' = U' R^{-1} (double), A = W U'' and U'' in Tc;
//            core (T + dS) x_1 R_1 (double)
//   5      : core x_n R_n for n = 2..p (T x U is left unchanged)
//   6 tasks: partial G_n = T_(n) T_(n)^T over column slices (double)
//   7 mode : G_n, G_n^{-1} by Gauss-Jordan (double); sigma^2 (Eq. 2.18) by a float
//            Jacobi warm-started from the previous eigenvectors, then Rayleigh
//            quotients in double
// GB300 issues one double warp-instruction per 64 cycles per SM sub-partition,
// with the same latency: double work is spread over all CTAs where it is a
// throughput cost and kept off the long serial chains where it is a latency cost.
// In the float compute type, C_n = I + D is accumulated in float; R comes from a
// series in D when D is small (as after every regular step) and otherwise from a
// float Cholesky with R^{-1} from one double Newton step on its float inverse.
// Either way R^{-1} R = I to double rounding (the core compensation stays exact)
// while U^T W U = I holds to the accuracy of C_n.
#include "common.cuh"
#include "kernels.h"
#include "small_dev.cuh"
#include "tc_project.h"

namespace tdb {

namespace {

constexpr int LD = kMaxRank;
constexpr int UPD_THREADS = 1024;
constexpr size_t kUpdSmem = 48 * 1024;   // largest phase: the Gram finish, 45.6 KB
constexpr int GJ_THREADS = 256;          // threads 0..255 invert G_n by Gauss-Jordan
// Modes with more row tiles than this (more than 1024 points) have their per-tile partial
// sums of P_n and C_n reduced once by the whole grid (reduce_long) instead of by every
// tile's CTA (P_n) or the mode's one CTA (C_n).
constexpr int kTreeTiles = 32;

__device__ __forceinline__ void named_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Order-preserving integer key of a double (larger value, larger key).
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (long long)(b ^ 0x7fffffffffffffffLL);
}

// Packed upper-triangle index e -> (a <= b), e < r (r + 1) / 2, column by column.
__device__ __forceinline__ void tri_index(int e, int* a, int* b) {
  int bb = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
  while ((bb + 1) * (bb + 2) / 2 <= e) ++bb;
  while (bb * (bb + 1) / 2 > e) --bb;
  *b = bb;
  *a = e - bb * (bb + 1) / 2;
}

// ---------------------------------------------------------------------------
// Double Cholesky S = L L^T in place (lower) and L^{-1}, all threads of the CTA
// (the double compute type's Cholesky-QR).
// ---------------------------------------------------------------------------
__device__ bool chol_d(double* S, int r, bool* ok_sh, double* dinv_sh) {
  if (threadIdx.x == 0) *ok_sh = true;
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      double d = S[k + LD * k];
      if (!(d > 0.0)) { *ok_sh = false; d = 1.0; }
      const double inv = drsqrt(d);
      S[k + LD * k] = d * inv;
      *dinv_sh = inv;
    }
    __syncthreads();
    const double inv = *dinv_sh;
    for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) S[i + LD * k] *= inv;
    __syncthreads();
    const int m = r - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e % m, j = k + 1 + e / m;
      if (j <= i) S[i + LD * j] -= S[i + LD * k] * S[j + LD * k];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    if (j > i) S[i + LD * j] = 0.0;
  }
  __syncthreads();
  return *ok_sh;
}

__device__ void trinv_d(const double* L, double* Li, int r, double* dinv) {
  for (int i = threadIdx.x; i < r; i += blockDim.x) dinv[i] = drcp(L[i + LD * i]);
  __syncthreads();
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    for (int i = 0; i < r; ++i) {
      if (i < j) { Li[i + LD * j] = 0.0; continue; }
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) s -= L[i + LD * k] * Li[k + LD * j];
      Li[i + LD * j] = s * dinv[i];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Float Cholesky and triangular inverse by one warp (lane i owns row i; the
// float compute type's Cholesky-QR).  S is r x r, ld LD, in shared memory.
// ---------------------------------------------------------------------------
__device__ bool chol_warp_f(float* S, int r) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int k = 0; k < r; ++k) {
    float d = S[k + LD * k];
    if (!(d > 0.f)) { ok = false; d = 1.f; }
    const float inv = rsqrt_approx(d);
    __syncwarp();
    float lik = 0.f;
    if (lane > k && lane < r) {
      lik = S[lane + LD * k] * inv;
      S[lane + LD * k] = lik;
    }
    if (lane == k) S[k + LD * k] = d * inv;
    __syncwarp();
    if (lane > k && lane < r)
      for (int j = k + 1; j <= lane; ++j) S[lane + LD * j] = fmaf(-lik, S[j + LD * k], S[lane + LD * j]);
    __syncwarp();
  }
  for (int j = 1; j < r; ++j)
    if (lane < j) S[lane + LD * j] = 0.f;
  __syncwarp();
  return ok;
}

// Li = L^{-1} (lower) by column sweeps: lane j owns column j.
__device__ void trinv_warp_f(const float* L, float* Li, int r) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < r; ++i)
    if (lane < r) Li[i + LD * lane] = (i == lane) ? 1.f : 0.f;
  __syncwarp();
  for (int k = 0; k < r; ++k) {
    if (lane <= k && lane < r) {
      const float x = Li[k + LD * lane] / L[k + LD * k];
      Li[k + LD * lane] = x;
      for (int i = k + 1; i < r; ++i) Li[i + LD * lane] = fmaf(-L[i + LD * k], x, Li[i + LD * lane]);
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi on a symmetric float matrix (n <= 32, ld LD, shared) by a group of
// `gs` threads (gt = index in the group, hardware barrier `bar`), Brent-Luk
// round-robin ordering as jacobi_smem: eigenvalues end on the diagonal of A and the
// vectors in V.  Stops when the off-diagonal mass is below tol^2 of the diagonal
// mass, after max_sweeps, or when a sweep after the second no longer halves it
// (the float rounding floor).  red holds >= 2 * gs / 32 floats.
// ---------------------------------------------------------------------------
__device__ int jacobi_group(float* A, float* V, int n, int max_sweeps, float tol, float* cs, int* pq, float* red,
                            int gt, int gs, int bar) {
  const int nn = (n + 1) & ~1, half = nn / 2;
  const int nw = gs >> 5, gl = gt & 31, gw = gt >> 5;
  for (int e = gt; e < nn * nn; e += gs) {
    const int i = e % nn, j = e / nn;
    if (i >= n || j >= n) A[i + LD * j] = 0.f;
    V[i + LD * j] = (i == j) ? 1.f : 0.f;
  }
  // the block (I, J) and the V entries (i, J) owned by this thread, fixed for all rounds
  const int bI = gt % half, bJ = gt / half;
  const bool has_b = gt < half * half;
  const int nv = nn * half;
  named_bar(bar, gs);
  const float thr = tol * 1e-3f;
  float off_prev = 0.f;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    float off = 0.f, dia = 0.f;
    for (int e = gt; e < nn * nn; e += gs) {
      const int i = e % nn, j = e / nn;
      const float v = A[i + LD * j];
      if (i == j) dia += v * v; else off += v * v;
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if (gl == 0) { red[gw] = off; red[nw + gw] = dia; }
    named_bar(bar, gs);
    off = 0.f;
    dia = 0.f;
    for (int w = 0; w < nw; ++w) { off += red[w]; dia += red[nw + w]; }
    named_bar(bar, gs);
    if (off <= tol * tol * dia || dia == 0.f) break;
    if (sweep >= 2 && off > 0.5f * off_prev) break;
    off_prev = off;
    for (int rd = 0; rd < nn - 1; ++rd) {
      if (gt < half) {
        const int k = gt;
        int p = rd, q = nn - 1;
        if (k > 0) {
          p = rd + k;
          if (p >= nn - 1) p -= nn - 1;
          q = rd - k;
          if (q < 0) q += nn - 1;
        }
        const float app = A[p + LD * p], aqq = A[q + LD * q], apq = A[p + LD * q];
        float c = 1.f, s = 0.f;
        if (apq != 0.f && apq * apq > thr * thr * fabsf(app * aqq)) {
          // tan of the rotation angle, t = sign(theta) / (|theta| + sqrt(theta^2 + 1)),
          // with approximate reciprocals: c^2 + s^2 = 1 holds whatever t's rounding
          const float theta = (aqq - app) * rcp_approx(2.f * apq);
          const float at = fabsf(theta);
          const float x = fmaf(at, at, 1.f);
          const float root = (at < 1e18f) ? x * rsqrt_approx(x) : at;
          const float t = copysignf(rcp_approx(at + root), theta);
          c = rsqrt_approx(fmaf(t, t, 1.f));
          s = t * c;
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
        pq[2 * k] = p;
        pq[2 * k + 1] = q;
      }
      named_bar(bar, gs);
      if (has_b) {
        const int pI = pq[2 * bI], qI = pq[2 * bI + 1], pJ = pq[2 * bJ], qJ = pq[2 * bJ + 1];
        const float cI = cs[2 * bI], sI = cs[2 * bI + 1], cJ = cs[2 * bJ], sJ = cs[2 * bJ + 1];
        const float b00 = A[pI + LD * pJ], b01 = A[pI + LD * qJ], b10 = A[qI + LD * pJ], b11 = A[qI + LD * qJ];
        const float c00 = cJ * b00 - sJ * b01, c01 = sJ * b00 + cJ * b01;
        const float c10 = cJ * b10 - sJ * b11, c11 = sJ * b10 + cJ * b11;
        A[pI + LD * pJ] = cI * c00 - sI * c10;
        A[pI + LD * qJ] = cI * c01 - sI * c11;
        A[qI + LD * pJ] = sI * c00 + cI * c10;
        A[qI + LD * qJ] = sI * c01 + cI * c11;
      }
      for (int e = gt; e < nv; e += gs) {
        const int i = e % nn, J = e / nn;
        const int pJ = pq[2 * J], qJ = pq[2 * J + 1];
        const float cJ = cs[2 * J], sJ = cs[2 * J + 1];
        const float vp = V[i + LD * pJ], vq = V[i + LD * qJ];
        V[i + LD * pJ] = cJ * vp - sJ * vq;
        V[i + LD * qJ] = sJ * vp + cJ * vq;
      }
      named_bar(bar, gs);
    }
  }
  return sweep;
}

// Gauss-Jordan inversion of the SPD matrix in A0 (r x r, ld LD, shared) by the
// threads [0, nthr) with hardware barrier `bar`, no pivoting (the pivots are the
// positive Schur-complement diagonals).  Step k reads one buffer and writes the
// other, so a step needs one barrier; returns the buffer holding the inverse.  The
// reciprocal of the next pivot is formed once, by the thread that updates that
// diagonal entry, into ipk[(k+1) & 1] (FP64 issues one warp-instruction per 64 cycles
// per SM sub-partition, so every thread forming it would cost the step more than the
// update itself).  *ok is false if a pivot is not a positive finite number.
__device__ double* gj_inverse(double* A0, double* A1, int r, int nthr, int bar, bool* ok, double* ipk, int* bad) {
  const int tid = threadIdx.x;
  double* cur = A0;
  double* nxt = A1;
  auto pivot_rcp = [&](double p, int slot) {
    const int hi = __double2hiint(p);
    if (hi <= 0 || ((hi >> 20) & 0x7ff) == 0x7ff) { *bad = 1; p = 1.0; }
    ipk[slot] = drcp(p);
  };
  if (tid == 0) {
    *bad = 0;
    pivot_rcp(cur[0], 0);
  }
  // this thread's entries (i, j), the same in every step (packed i | j << 8, -1 none)
  constexpr int EPT = LD * LD / GJ_THREADS;
  int ent[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int e = tid + nthr * u;
    ent[u] = e < r * r ? ((e % r) | ((e / r) << 8)) : -1;
  }
  named_bar(bar, nthr);
  for (int k = 0; k < r; ++k) {
    const double ip = ipk[k & 1];
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      if (ent[u] < 0) continue;
      const int i = ent[u] & 255, j = ent[u] >> 8;
      const double akj = (j == k) ? ip : cur[k + LD * j] * ip;     // row k after the step
      const double v = (i == k) ? akj : (j == k ? 0.0 : cur[i + LD * j]) - cur[i + LD * k] * akj;
      nxt[i + LD * j] = v;
      if (i == k + 1 && j == k + 1) pivot_rcp(v, (k + 1) & 1);
    }
    named_bar(bar, nthr);
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  *ok = *bad == 0;
  return cur;
}

// Bounded grid barrier; every CTA is resident (cooperative launch, <= 1 CTA per SM).
// The counter (zeroed before the launch) only grows: the k-th barrier (k from 1)
// waits for k * nblocks arrivals.  Release on arrival and acquire on the spin order
// the CTA's writes before and its reads after the barrier.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
constexpr long long kGridWaitCycles = 4000000000ll;   // ~2 s at 2 GHz
__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned k, unsigned nblocks, unsigned* flags,
                                          volatile int* abort_sh, long long limit = kGridWaitCycles) {
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_gpu(count, 1u);
    const unsigned target = k * nblocks;
    const long long t0 = clock64();
    unsigned it = 0;
    // one load per poll; the clock and another CTA's timeout flag every 32nd
    while (ld_acquire_gpu(count) < target) {
      if ((++it & 31) == 0 && (clock64() - t0 > limit || (ld_acquire_gpu(flags) & kFlagTimeout))) {
        atomicOr(flags, kFlagTimeout);
        *abort_sh = 1;
        break;
      }
    }
  }
  __syncthreads();
  return *abort_sh == 0;
}

// Profiling: CTA 0 reads the global timer at the start, after every grid barrier
// and at its end into shared memory; at the end it adds the phase durations to
// st[16 + k] (nanoseconds summed over launches; st null when profiling is off).
__device__ __forceinline__ void stamp(unsigned long long* sh, const unsigned long long* st, int k) {
  if (st && blockIdx.x == 0 && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    sh[k] = t;
  }
}
__device__ __forceinline__ void stamp_flush(const unsigned long long* sh, unsigned long long* st, int nst) {
  if (st && blockIdx.x == 0 && threadIdx.x == 0)
    for (int k = 1; k <= nst; ++k) atomicAdd(&st[16 + k - 1], sh[k] - sh[k - 1]);
}

}  // namespace

// ---------------------------------------------------------------------------
// Gram refresh, shared by the fused update and the standalone launches.
// ---------------------------------------------------------------------------

// Partial G_n = T_(n) T_(n)^T over column slice `sp` of mode n: the slice is staged
// in shared memory 32 columns at a time; one thread per upper-triangle entry.
__device__ void gram_partial(const ModeDesc& d, const double* T, double* gpart, int gsplit, int n, int sp,
                             double (*S)[33]) {
  const int r = d.r[n];
  const int64_t L = prod_r_below(d, n), Q = prod_r_above(d, n);
  const int64_t ncol = L * Q;
  const int64_t c0 = ncol * sp / gsplit, c1 = ncol * (sp + 1) / gsplit;
  const int ntri = r * (r + 1) / 2;
  int ta = 0, tb = 0;
  if ((int)threadIdx.x < ntri) tri_index(threadIdx.x, &ta, &tb);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double s = 0.0;
  for (int64_t cb = c0; cb < c1; cb += 32) {
    const int64_t c = cb + tx;
    double v = 0.0;
    if (c < c1 && ty < r) {
      const int64_t l = c % L, q = c / L;
      v = __ldcg(&T[l + L * (ty + (int64_t)r * q)]);
    }
    S[ty][tx] = v;
    __syncthreads();
    if ((int)threadIdx.x < ntri) {
#pragma unroll 8
      for (int x = 0; x < 32; ++x) s = fma(S[ta][x], S[tb][x], s);
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < ntri) gpart[((int64_t)n * gsplit + sp) * LD * LD + ta + LD * tb] = s;
}

// Mode n: sum the partials into G_n; G_n^{-1} by Gauss-Jordan (threads 0..255)
// while threads 256..511 run the float Jacobi on Vp^T (G / scale) Vp (Vp the previous
// eigenvectors, identity when cold); then Rayleigh quotients v^T G v / v^T v in
// double, sorted descending by an integer key; the sorted eigenvectors become the
// next warm start.  One CTA of UPD_THREADS threads; smraw holds >= 46 KB.
__device__ __noinline__ void gram_finish(const ModeDesc& d, int n, const double* gpart, int gsplit, double* Gout,
                                         double* Ginv, float* Ginvf, double* sig2, float* Vprev, int warm,
                                         unsigned* flags, unsigned char* smraw) {
  const int r = d.r[n];
  double* G = (double*)smraw;          // LD*LD
  double* Ai = G + LD * LD;            // LD*LD: Gauss-Jordan buffers, then G W
  double* Ai2 = Ai + LD * LD;          // LD*LD
  double* lam = Ai2 + LD * LD;         // LD
  float* Gf = (float*)(lam + LD);      // LD*LD: G / scale in float
  float* Vps = Gf + LD * LD;           // LD*LD: previous eigenvectors
  float* Af = Vps + LD * LD;           // LD*LD
  float* Vf = Af + LD * LD;            // LD*LD  (Af and Vf later hold W in double)
  float* Wf = Vf + LD * LD;            // LD*LD
  float* cs = Wf + LD * LD;            // 64
  float* red = cs + 64;                // 64
  int* pq = (int*)(red + 64);          // 64
  int* slot = pq + 64;                 // LD
  double* GW = Ai;
  double* Wd = (double*)Af;
  __shared__ int bad_sh, gjbad_sh;
  __shared__ float scale_sh;
  __shared__ double ipk_sh[2];
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  constexpr int JG = 256;              // Jacobi group: threads [JG, 2 JG)
  float* Vp = Vprev + (int64_t)n * LD * LD;
  if (tid == 0) bad_sh = 0;
  for (int e = tid; e < LD * LD; e += blockDim.x) {
    const int ra = e % LD, rb = e / LD;
    double s = 0.0;
    if (ra < r && rb < r) {
      const int aa = ra <= rb ? ra : rb, bb = ra <= rb ? rb : ra;
      const double* src = gpart + (int64_t)n * gsplit * LD * LD + aa + LD * bb;
#pragma unroll 8
      for (int k = 0; k < gsplit; ++k) s += __ldcg(&src[(int64_t)k * LD * LD]);
    }
    G[e] = s;
    Ai[e] = s;
    Vps[e] = (warm && ra < r && rb < r) ? Vp[e] : 0.f;
  }
  __syncthreads();
  if (wid == 0) {
    float m = 0.f;
    for (int k = lane; k < r; k += 32) m = fmaxf(m, (float)G[k + LD * k]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) scale_sh = m > 0.f ? 1.f / m : 1.f;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int a = e % r, b = e / r;
    Gf[a + LD * b] = (float)G[a + LD * b] * scale_sh;
  }
  __syncthreads();
  __shared__ double* inv_sh;
  if (tid < GJ_THREADS) {
    bool good;
    double* res = gj_inverse(Ai, Ai2, r, GJ_THREADS, 1, &good, ipk_sh, &gjbad_sh);
    if (tid == 0) {
      inv_sh = res;
      if (!good) bad_sh = 1;
    }
  } else if (tid < GJ_THREADS + JG) {
    const int gt = tid - GJ_THREADS;
    if (warm) {
      for (int e = gt; e < r * r; e += JG) {             // Wf = (G / scale) Vp
        const int i = e % r, b = e / r;
        float s = 0.f;
        for (int j = 0; j < r; ++j) s = fmaf(Gf[i + LD * j], Vps[j + LD * b], s);
        Wf[i + LD * b] = s;
      }
      named_bar(2, JG);
      for (int e = gt; e < r * r; e += JG) {             // Af = Vp^T Wf
        const int a = e % r, b = e / r;
        float s = 0.f;
        for (int i = 0; i < r; ++i) s = fmaf(Vps[i + LD * a], Wf[i + LD * b], s);
        Af[a + LD * b] = s;
      }
    } else {
      for (int e = gt; e < r * r; e += JG) {
        const int a = e % r, b = e / r;
        Af[a + LD * b] = Gf[a + LD * b];
      }
    }
    named_bar(2, JG);
    jacobi_group(Af, Vf, r, warm ? 2 : 30, 1e-6f, cs, pq, red, gt, JG, 2);
    for (int e = gt; e < r * r; e += JG) {               // eigenvectors in the original basis
      const int a = e % r, b = e / r;
      float s = Vf[a + LD * b];
      if (warm) {
        s = 0.f;
        for (int k = 0; k < r; ++k) s = fmaf(Vps[a + LD * k], Vf[k + LD * b], s);
      }
      Wf[a + LD * b] = s;
    }
  }
  __syncthreads();
  if (bad_sh && tid == 0) atomicOr(flags, kFlagCholGram);
  for (int e = tid; e < LD * LD; e += blockDim.x) {
    const int a = e % LD, b = e / LD;
    const bool in = a < r && b < r;
    const double gi = in ? inv_sh[e] : 0.0;
    Gout[(int64_t)n * LD * LD + e] = G[e];
    Ginv[(int64_t)n * LD * LD + e] = gi;
    if (Ginvf) Ginvf[(int64_t)n * LD * LD + e] = in ? (float)gi : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int a = e % r, b = e / r;
    Wd[a + LD * b] = (double)Wf[a + LD * b];
  }
  __syncthreads();
  // Rayleigh quotients: GW = G W, then warp j reduces column j
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    double s = 0.0;
    for (int k = 0; k < r; ++k) s = fma(G[i + LD * k], Wd[k + LD * j], s);
    GW[i + LD * j] = s;
  }
  __syncthreads();
  if (wid < r) {
    const int j = wid;
    double num = 0.0, den = 0.0;
    if (lane < r) {
      const double v = Wd[lane + LD * j];
      num = v * GW[lane + LD * j];
      den = v * v;
    }
    num = warp_sum(num);
    den = warp_sum(den);
    if (lane == 0) lam[j] = den > 0.0 ? num * drcp(den) : 0.0;
  }
  __syncthreads();
  if (tid < r) {                                         // descending rank by integer keys
    const long long kj = order_key(lam[tid]);
    int rank = 0;
    for (int k = 0; k < r; ++k) {
      const long long kk = order_key(lam[k]);
      rank += (kk > kj) || (kk == kj && k < tid);
    }
    slot[tid] = rank;
    sig2[(int64_t)n * LD + rank] = lam[tid];
  } else if (tid < LD) {
    sig2[(int64_t)n * LD + tid] = 0.0;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    Vp[i + LD * slot[j]] = Wf[i + LD * j];
  }
}

// ---------------------------------------------------------------------------
// Row-tile phases
// ---------------------------------------------------------------------------

// Phase 1 on one tile of mode n: M = Y_(n) T_(n)^T, X = M G^{-1}, partial P = A^T X.
template <typename Tc>
__device__ void rows_mxp(const UpdArgs& a, int n, int64_t i0, int tile, unsigned char* sm) {
  const ModeDesc& d = a.d;
  const int r = d.r[n];
  const int64_t N = d.N[n];
  const int li = threadIdx.x & 31, ca = threadIdx.x >> 5;
  const int64_t i = i0 + li;
  Tc (*Ysh)[33] = (Tc(*)[33])sm;
  Tc (*Tsh)[33] = Ysh + 32;
  Tc (*Msh)[33] = Tsh + 32;
  Tc* Gi = (Tc*)(Msh + 32);
  const int64_t L = prod_r_below(d, n), Q = prod_r_above(d, n);
  const Tc* Y = (const Tc*)a.Y[n];
  const Tc* Tm = (const Tc*)a.Tcore;
  if (sizeof(Tc) == 8) {
    for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) Gi[e] = (Tc)a.Ginv[(int64_t)n * LD * LD + e];
  } else {
    for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) Gi[e] = (Tc)a.Ginvf[(int64_t)n * LD * LD + e];
  }
  const int64_t ncol = L * Q;
  Tc s = Tc(0);
  // staging: for L == 1 the rows of Y_(n) (and the ranks of T_(n)) are contiguous, so
  // lanes run along rows; otherwise along columns.  The next chunk is loaded into
  // registers while the current one is multiplied.
  const bool rows_fast = (L == 1);
  const int u = threadIdx.x & 31, v = threadIdx.x >> 5;
  const int srow = rows_fast ? u : v, scol = rows_fast ? v : u;
  auto fetch = [&](int64_t c0, Tc* vy, Tc* vt) {
    const int64_t c = c0 + scol;
    const int64_t ii = i0 + srow;
    *vy = Tc(0);
    *vt = Tc(0);
    if (c < ncol) {
      const int64_t l = c % L, q = c / L;
      if (ii < N) *vy = Y[l + L * (ii + N * q)];
      if (srow < r) *vt = Tm[l + L * (srow + (int64_t)r * q)];
    }
  };
  Tc vy, vt;
  fetch(0, &vy, &vt);
  for (int64_t c0 = 0; c0 < ncol; c0 += 32) {
    Ysh[srow][scol] = vy;
    Tsh[srow][scol] = vt;
    __syncthreads();
    if (c0 + 32 < ncol) fetch(c0 + 32, &vy, &vt);
    if (ca < r) {
#pragma unroll 8
      for (int x = 0; x < 32; ++x) s += Ysh[li][x] * Tsh[ca][x];
    }
    __syncthreads();
  }
  if (ca < r) Msh[li][ca] = s;
  Tc (*Ash)[33] = Ysh;
  Tc (*Xsh)[33] = Tsh;
  Ash[li][ca] = (ca < r && i < N) ? ((const Tc*)a.A[n])[i + N * ca] : Tc(0);
  __syncthreads();
  Tc x = Tc(0);
  if (ca < r && i < N) {
    for (int b = 0; b < r; ++b) x += Msh[li][b] * Gi[b + LD * ca];
    ((Tc*)a.X[n])[i + N * ca] = x;
  }
  Xsh[li][ca] = x;
  __syncthreads();
  if ((int)threadIdx.x < r * r) {
    const int ra = threadIdx.x % r, rb = threadIdx.x / r;
    Tc acc = Tc(0);
#pragma unroll 8
    for (int t = 0; t < 32; ++t) acc += Ash[t][ra] * Xsh[t][rb];
    ((Tc*)a.part)[((int64_t)n * a.ntile + tile) * LD * LD + ra + LD * rb] = acc;
  }
  __syncthreads();
}

// Phase 2 on one tile of mode n: P_n, E = X - U P_n, U' = U + E (Heun's second stage:
// U' = (U0 + U + E) / 2; the midpoint scheme's second stage: U' = U0 + E), partial
// C = U'^T W U'.
template <typename Tc>
__device__ void rows_u1(const UpdArgs& a, int n, int64_t i0, int tile, unsigned char* sm) {
  const ModeDesc& d = a.d;
  const int r = d.r[n];
  const int64_t N = d.N[n];
  const int li = threadIdx.x & 31, ca = threadIdx.x >> 5;
  const int64_t i = i0 + li;
  Tc* Psh = (Tc*)sm;                         // LD*LD
  Tc (*Ush)[33] = (Tc(*)[33])(Psh + LD * LD);
  Tc* wsh = (Tc*)(Ush + 32);                 // 32
  const Tc* part = (const Tc*)a.part;
  const int nt = (int)((N + 31) / 32);
  {
    const int e = threadIdx.x, ra = e % LD, rb = e / LD;
    Tc s = Tc(0);
    if (ra < r && rb < r) {
      if (nt > kTreeTiles) {
        s = __ldcg(&((const Tc*)a.red)[(int64_t)n * LD * LD + e]);
      } else {
        const Tc* src = part + (int64_t)n * a.ntile * LD * LD + e;
#pragma unroll 8
        for (int t = 0; t < nt; ++t) s += __ldcg(&src[(int64_t)t * LD * LD]);
      }
    }
    Psh[e] = s;
  }
  Ush[li][ca] = (ca < r && i < N) ? ((const Tc*)a.Uc[n])[i + N * ca] : Tc(0);
  if (threadIdx.x < 32) wsh[li] = (i < N) ? (Tc)a.w[n][i] : Tc(0);
  __syncthreads();
  Tc upc = Tc(0);
  if (ca < r && i < N) {
    Tc e = __ldcg(&((const Tc*)a.X[n])[i + N * ca]);
    for (int b = 0; b < r; ++b) e -= Ush[li][b] * Psh[b + LD * ca];
    const int64_t ix = i + N * ca;
    const double up = !a.T0             ? a.U[n][ix] + (double)e
                      : a.combine == 2 ? a.U0[n][ix] + (double)e
                                       : 0.5 * ((a.U[n][ix] + a.U0[n][ix]) + (double)e);
    a.Up[n][i + N * ca] = up;
    upc = (Tc)up;
  }
  __syncthreads();
  Ush[li][ca] = upc;
  __syncthreads();
  if ((int)threadIdx.x < r * r) {
    const int ra = threadIdx.x % r, rb = threadIdx.x / r;
    Tc acc = Tc(0);
#pragma unroll 8
    for (int t = 0; t < 32; ++t) acc += Ush[t][ra] * wsh[t] * Ush[t][rb];
    ((Tc*)a.part)[(int64_t)a.d.p * a.ntile * LD * LD + ((int64_t)n * a.ntile + tile) * LD * LD + ra + LD * rb] = acc;
  }
  __syncthreads();
}

// Phases 1b / 2b, only for modes with more than kTreeTiles row tiles: the per-tile
// partials of P_n (which = 0) or C_n (which = 1) summed by the whole grid, a warp per
// entry, its lanes over every 32nd tile, then a butterfly of shuffles (the same order on
// every run).  Results go to red[which][n], read by every tile of phase 2 (P_n) or by
// the Cholesky-QR of phase 3 (C_n).
template <typename Tc>
__device__ void reduce_long(const UpdArgs& a, int which) {
  const ModeDesc& d = a.d;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const Tc* part = (const Tc*)a.part + (int64_t)which * d.p * a.ntile * LD * LD;
  Tc* red = (Tc*)a.red + (int64_t)which * kMaxModes * LD * LD;
  for (int64_t task = gw; task < (int64_t)d.p * LD * LD; task += nw) {
    const int n = (int)(task / (LD * LD)), e = (int)(task % (LD * LD));
    const int nt = (int)((d.N[n] + 31) / 32);
    const int r = d.r[n], ra = e % LD, rb = e / LD;
    if (nt <= kTreeTiles || ra >= r || rb >= r) continue;     // the same for the whole warp
    const Tc* src = part + (int64_t)n * a.ntile * LD * LD + e;
    Tc s = Tc(0);
    for (int t = lane; t < nt; t += 32) s += __ldcg(&src[(int64_t)t * LD * LD]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[(int64_t)n * LD * LD + e] = s;
  }
}

// Phase 3 for mode n (one CTA): C_n from the partials, R (upper, C = R^T R) and R^{-1}.
template <typename Tc>
__device__ void mode_cholqr(const UpdArgs& a, int n, unsigned char* sm) {
  const ModeDesc& d = a.d;
  const int r = d.r[n];
  const int nt = (int)((d.N[n] + 31) / 32);
  const Tc* part = (const Tc*)a.part + (int64_t)d.p * a.ntile * LD * LD + (int64_t)n * a.ntile * LD * LD;
  double* Rg = a.R + (int64_t)n * LD * LD;
  double* Rig = a.Rinv + (int64_t)n * LD * LD;
  __shared__ bool ok_sh;
  __shared__ double dinv_sh;
  if (!a.reorth) {
    for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) Rg[e] = Rig[e] = (e % LD == e / LD) ? 1.0 : 0.0;
    return;
  }
  if (sizeof(Tc) == 8) {
    double* C = (double*)sm;
    double* Li = C + LD * LD;
    double* dinv = Li + LD * LD;
    for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
      const int ra = e % LD, rb = e / LD;
      double s = 0.0;
      if (ra < r && rb < r) {
        if (nt > kTreeTiles)
          s = (double)__ldcg(&((const Tc*)a.red)[(int64_t)(kMaxModes + n) * LD * LD + e]);
        else
#pragma unroll 8
          for (int t = 0; t < nt; ++t) s += (double)__ldcg(&part[(int64_t)t * LD * LD + e]);
      }
      C[e] = s;
    }
    __syncthreads();
    if (!chol_d(C, r, &ok_sh, &dinv_sh) && threadIdx.x == 0) atomicOr(a.flags, kFlagCholQR);
    trinv_d(C, Li, r, dinv);
    for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
      const int ra = e % LD, rb = e / LD;
      Rg[e] = (ra < r && rb < r) ? C[rb + LD * ra] : 0.0;     // R = L^T
      Rig[e] = (ra < r && rb < r) ? Li[rb + LD * ra] : 0.0;   // R^{-1} = L^{-T}
    }
  } else {
    float* Cf = (float*)sm;                 // LD*LD
    float* Lif = Cf + LD * LD;              // LD*LD
    double* R0 = (double*)(Lif + LD * LD);  // LD*LD
    double* Z0 = R0 + LD * LD;              // LD*LD
    double* E = Z0 + LD * LD;               // LD*LD
    __shared__ float fmax_sh;
    for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
      const int ra = e % LD, rb = e / LD;
      float s = 0.f;
      if (ra < r && rb < r) {
        if (nt > kTreeTiles)
          s = (float)__ldcg(&((const Tc*)a.red)[(int64_t)(kMaxModes + n) * LD * LD + e]);
        else
#pragma unroll 8
          for (int t = 0; t < nt; ++t) s += (float)__ldcg(&part[(int64_t)t * LD * LD + e]);
      }
      Cf[e] = s;
    }
    __syncthreads();
    // C = I + D with D small after a step: R = I + F, F = Phi(D - F1^T F1), F1 = Phi(D),
    // Phi = upper triangle with the diagonal halved (R^T R = C up to O(|D|^3)), and
    // R^{-1} = I - F + F^2 - F^3 + F^4 (R R^{-1} = I + F^5).  Taken when max |F1| <= 2^-14,
    // so that |F^5| < 4e-14 for r <= 32.
    float* F1 = Lif;
    for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
      const int ra = e % LD, rb = e / LD;
      float f = 0.f;
      if (ra < r && rb < r && ra <= rb) f = (ra == rb) ? 0.5f * (Cf[e] - 1.f) : Cf[e];
      F1[e] = f;
    }
    if (threadIdx.x == 0) fmax_sh = 0.f;
    __syncthreads();
    {
      float m = 0.f;
      for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
        const float v = fabsf(F1[e]);
        m = (v == v) ? fmaxf(m, v) : 3.0e38f;      // a NaN takes the Cholesky path, which flags it
      }
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax((int*)&fmax_sh, __float_as_int(m));
    }
    __syncthreads();
    if (fmax_sh <= 6.103515625e-05f) {
      float* Fs = (float*)R0;                // LD*LD float: F
      float* F2 = Fs + LD * LD;              // F^2
      float* F3 = F2 + LD * LD;              // F^3
      float* F4 = F3 + LD * LD;              // F^4
      for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {   // F = Phi(D - F1^T F1)
        const int ra = e % LD, rb = e / LD;
        float f = 0.f;
        if (ra < r && rb < r && ra <= rb) {
          float q = 0.f;
          for (int k = 0; k <= ra; ++k) q = fmaf(F1[k + LD * ra], F1[k + LD * rb], q);
          f = (ra == rb) ? F1[e] - 0.5f * q : Cf[e] - q;
        }
        Fs[e] = f;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
        const int ra = e % LD, rb = e / LD;
        float q = 0.f;
        if (ra < r && rb < r && ra <= rb)
          for (int k = ra; k <= rb; ++k) q = fmaf(Fs[ra + LD * k], Fs[k + LD * rb], q);
        F2[e] = q;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
        const int ra = e % LD, rb = e / LD;
        float q = 0.f;
        if (ra < r && rb < r && ra <= rb)
          for (int k = ra; k <= rb; ++k) q = fmaf(F2[ra + LD * k], Fs[k + LD * rb], q);
        F3[e] = q;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
        const int ra = e % LD, rb = e / LD;
        float q = 0.f;
        if (ra < r && rb < r && ra <= rb)
          for (int k = ra; k <= rb; ++k) q = fmaf(F2[ra + LD * k], F2[k + LD * rb], q);
        F4[e] = q;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
        const int ra = e % LD, rb = e / LD;
        const double id = (ra == rb && ra < r) ? 1.0 : 0.0;
        Rg[e] = id + (double)Fs[e];
        Rig[e] = (((id - (double)Fs[e]) + (double)F2[e]) - (double)F3[e]) + (double)F4[e];
      }
      return;
    }
    if (threadIdx.x < 32) {
      const bool good = chol_warp_f(Cf, r);
      if (!good && threadIdx.x == 0) atomicOr(a.flags, kFlagCholQR);
      trinv_warp_f(Cf, Lif, r);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
      const int ra = e % LD, rb = e / LD;
      const bool in = ra < r && rb < r;
      R0[e] = in ? (double)Cf[rb + LD * ra] : 0.0;            // R0 = L^T (upper)
      Z0[e] = in ? (double)Lif[rb + LD * ra] : 0.0;           // Z0 = L^{-T}, float accurate
    }
    __syncthreads();
    // one Newton step in double: Z1 = Z0 + Z0 (I - R0 Z0); all three are upper triangular
    const int ntri = r * (r + 1) / 2;
    for (int e = threadIdx.x; e < ntri; e += blockDim.x) {
      int ia, jb;
      tri_index(e, &ia, &jb);
      double s = (ia == jb) ? 1.0 : 0.0;
      for (int k = ia; k <= jb; ++k) s = fma(-R0[ia + LD * k], Z0[k + LD * jb], s);
      E[ia + LD * jb] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) {
      const int ia = e % LD, jb = e / LD;
      double z = 0.0;
      if (ia < r && jb < r && ia <= jb) {
        z = Z0[e];
        for (int k = ia; k <= jb; ++k) z = fma(Z0[ia + LD * k], E[k + LD * jb], z);
      }
      Rg[e] = R0[e];
      Rig[e] = z;
    }
  }
}

// Phase 4 on one tile of mode n: U'' = U' R^{-1}, A = W U'' and U'' in the compute type.
template <typename Tc>
__device__ void rows_u2(const UpdArgs& a, int n, int64_t i0, unsigned char* sm) {
  const ModeDesc& d = a.d;
  const int r = d.r[n];
  const int64_t N = d.N[n];
  const int li = threadIdx.x & 31, ca = threadIdx.x >> 5;
  const int64_t i = i0 + li;
  double (*Ush)[LD + 1] = (double(*)[LD + 1])sm;
  double* Rsh = (double*)(Ush + 32);
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) Rsh[e] = __ldcg(&a.Rinv[(int64_t)n * LD * LD + e]);
  if (ca < r) Ush[li][ca] = (i < N) ? __ldcg(&a.Up[n][i + N * ca]) : 0.0;
  __syncthreads();
  if (ca < r && i < N) {
    double s = 0.0;
    for (int b = 0; b <= ca; ++b) s = fma(Ush[li][b], Rsh[b + LD * ca], s);
    a.U[n][i + N * ca] = s;
    ((Tc*)a.A[n])[i + N * ca] = (Tc)(a.w[n][i] * s);
    ((Tc*)a.Uc[n])[i + N * ca] = (Tc)s;
  }
  __syncthreads();
}

// Core mode product dst = src x_n R_n (R_n upper triangular); the first mode adds dS
// to T (Heun's second stage: forms (T0 + T + dS) / 2; the midpoint scheme's: T0 + dS).  Work is split by mode-n fibers (the r_n entries at fixed other indices):
// each pass stages F fibers per CTA in shared memory (one coalesced load per
// thread), F chosen so that every CTA of the grid has some.
template <typename Tc>
__device__ void core_mode(const UpdArgs& a, int n, const double* src, double* dst, unsigned char* sm) {
  const ModeDesc& d = a.d;
  const int r = d.r[n];
  const int64_t L = prod_r_below(d, n);
  const int64_t nfib = prod_r(d) / r;
  const int64_t per_cta = (nfib + gridDim.x - 1) / gridDim.x;
  const int F = (int)(per_cta < UPD_THREADS / r ? per_cta : UPD_THREADS / r);
  double* Rsh = (double*)sm;            // LD*LD
  double* Xs = Rsh + LD * LD;           // r x F <= UPD_THREADS
  for (int e = threadIdx.x; e < LD * LD; e += blockDim.x) Rsh[e] = __ldcg(&a.R[(int64_t)n * LD * LD + e]);
  const Tc* dS = (const Tc*)a.dS;
  const int t = threadIdx.x, fl = t % F, j = t / F;
  for (int64_t f0 = blockIdx.x * (int64_t)F; f0 < nfib; f0 += (int64_t)gridDim.x * F) {
    const int64_t f = f0 + fl;
    const bool act = j < r && f < nfib;
    int64_t idx = 0;
    if (act) {
      const int64_t l = f % L, q = f / L;
      idx = l + L * (j + (int64_t)r * q);
      if (n != 0)
        Xs[j * F + fl] = __ldcg(&src[idx]);
      else if (a.T0 && a.combine == 2)
        Xs[j * F + fl] = a.T0[idx] + (double)dS[idx];
      else if (a.T0)
        Xs[j * F + fl] = 0.5 * ((src[idx] + a.T0[idx]) + (double)dS[idx]);
      else
        Xs[j * F + fl] = src[idx] + (double)dS[idx];
    }
    __syncthreads();
    if (act) {
      double s = 0.0;
      for (int k = j; k < r; ++k) s = fma(Rsh[j + LD * k], Xs[k * F + fl], s);
      dst[idx] = s;
    }
    __syncthreads();
  }
}

template <typename Tc>
__global__ void __launch_bounds__(UPD_THREADS, 1) k_update(UpdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int abort_sh;
  if (threadIdx.x == 0) abort_sh = 0;
  __syncthreads();
  __shared__ unsigned long long st_sh[16];
  int nst = 0;
  unsigned nbar = 0;
  stamp(st_sh, a.stamps, 0);
  const ModeDesc& d = a.d;
  const int p = d.p;
  const unsigned nb = gridDim.x;

  int ntiles_total = 0, tile_base[kMaxModes + 1];
  for (int n = 0; n < p; ++n) {
    tile_base[n] = ntiles_total;
    ntiles_total += (int)((d.N[n] + 31) / 32);
  }
  tile_base[p] = ntiles_total;
  bool tree = false;
  for (int n = 0; n < p; ++n) tree |= (d.N[n] + 31) / 32 > kTreeTiles;
  auto tile_of = [&](int task, int* n_out, int* t_out) {
    int n = 0;
    while (task >= tile_base[n + 1]) ++n;
    *n_out = n;
    *t_out = task - tile_base[n];
  };

  // 1: M, X, partial P; dS = Y_2 x_2 A_2^T when the projection left it
  for (int task = blockIdx.x; task < ntiles_total; task += nb) {
    int n, t;
    tile_of(task, &n, &t);
    rows_mxp<Tc>(a, n, (int64_t)t * 32, t, smraw);
  }
  if (a.ds_y2) {
    // dS = Y_2 x_2 A_2^T (Eqs. 2.15/2.16: dS = Y_n x_n A_n^T for every n), read from
    // phase 4 on.  Eight consecutive threads share one element (every CTA takes a share
    // of the elements): each sums every eighth i2 with all its loads in flight, then the
    // eight partial sums are added by shuffles in a fixed order.
    const Tc* Y2 = (const Tc*)a.ds_y2;
    const Tc* A2 = (const Tc*)a.A[1];
    const int r1 = d.r[0], r2 = d.r[1];
    const int N2 = (int)d.N[1];
    const int64_t tot = prod_r(d);
    const int grp = threadIdx.x >> 3, part = threadIdx.x & 7;
    const int ngrp = blockDim.x >> 3;
    const int64_t stride = (int64_t)nb * ngrp;
    const int64_t rounds = (tot + stride - 1) / stride;
    for (int64_t k = 0; k < rounds; ++k) {
      const int64_t e = blockIdx.x + (int64_t)nb * grp + stride * k;
      Tc acc = Tc(0);
      if (e < tot) {
        const int a1 = (int)(e % r1);
        const int64_t rest = e / r1;
        const int b = (int)(rest % r2);
        const int64_t q = rest / r2;
        const Tc* y = Y2 + a1 + (int64_t)r1 * N2 * q;      // Y_2[a1 + r1 (i2 + N2 q)]
        const Tc* A = A2 + (int64_t)N2 * b;
#pragma unroll 16
        for (int i2 = part; i2 < N2; i2 += 8) acc += __ldcg(&y[(int64_t)r1 * i2]) * A[i2];
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (e < tot && part == 0) ((Tc*)a.dS_out)[e] = acc;
    }
  }
  if (!grid_sync(a.bar, ++nbar, nb, a.flags, &abort_sh)) return;
  stamp(st_sh, a.stamps, ++nst);
  if (tree) {
    reduce_long<Tc>(a, 0);
    if (!grid_sync(a.bar, ++nbar, nb, a.flags, &abort_sh)) return;
  }

  // 2: P, U', partial C
  for (int task = blockIdx.x; task < ntiles_total; task += nb) {
    int n, t;
    tile_of(task, &n, &t);
    rows_u1<Tc>(a, n, (int64_t)t * 32, t, smraw);
  }
  if (!grid_sync(a.bar, ++nbar, nb, a.flags, &abort_sh)) return;
  stamp(st_sh, a.stamps, ++nst);
  if (tree && a.reorth) {
    reduce_long<Tc>(a, 1);
    if (!grid_sync(a.bar, ++nbar, nb, a.flags, &abort_sh)) return;
  }

  // 3: Cholesky-QR factors, one CTA per mode
  for (int n = blockIdx.x; n < p; n += nb) mode_cholqr<Tc>(a, n, smraw);
  if (!grid_sync(a.bar, ++nbar, nb, a.flags, &abort_sh)) return;
  stamp(st_sh, a.stamps, ++nst);

  // 4: U'' and the core product of mode 1; 5: the other modes (T -> T2 -> T ...)
  for (int task = blockIdx.x; task < ntiles_total; task += nb) {
    int n, t;
    tile_of(task, &n, &t);
    rows_u2<Tc>(a, n, (int64_t)t * 32, smraw);
  }
  for (int n = 0; n < p; ++n) {
    const double* src = (n & 1) ? a.T2 : a.T;
    double* dst = (n & 1) ? a.T : a.T2;
    core_mode<Tc>(a, n, src, dst, smraw);
    if (!grid_sync(a.bar, ++nbar, nb, a.flags, &abort_sh)) return;
    stamp(st_sh, a.stamps, ++nst);
  }

  // 6: final core in T, compute-type copy, Gram partials
  {
    const double* Tfin = (p & 1) ? a.T2 : a.T;
    const int64_t Rprod = prod_r(d);
    const int64_t gstr = (int64_t)nb * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Rprod; e += gstr) {
      const double v = __ldcg(&Tfin[e]);
      if (p & 1) a.T[e] = v;
      if (sizeof(Tc) == 4) ((float*)a.Tcore)[e] = (float)v;
    }
    for (int task = blockIdx.x; task < p * a.gsplit; task += nb)
      gram_partial(d, Tfin, a.gpart, a.gsplit, task / a.gsplit, task % a.gsplit, (double(*)[33])smraw);
  }
  if (!grid_sync(a.bar, ++nbar, nb, a.flags, &abort_sh)) return;
  stamp(st_sh, a.stamps, ++nst);

  // 7: G, G^{-1}, sigma^2 (or a separate launch beside the exact error)
  if (!a.skip_finish)
    for (int n = blockIdx.x; n < p; n += nb)
      gram_finish(d, n, a.gpart, a.gsplit, a.G, a.Ginv, a.Ginvf, a.sig2, a.Vprev, a.warm, a.flags, smraw);
  stamp(st_sh, a.stamps, ++nst);
  stamp_flush(st_sh, a.stamps, nst);
}

// The Gram refresh of phases 6-7 as two ordinary launches (after (re)initialisation
// and state loads), bit-identical to the fused path.
__global__ void __launch_bounds__(UPD_THREADS, 1) k_gram_partial(ModeDesc d, const double* T, double* gpart,
                                                                 int gsplit) {
  __shared__ double S[32][33];
  gram_partial(d, T, gpart, gsplit, blockIdx.x / gsplit, blockIdx.x % gsplit, S);
}

__global__ void __launch_bounds__(UPD_THREADS, 1) k_gram_finish(ModeDesc d, const double* gpart, int gsplit, double* G,
                                                                double* Ginv, float* Ginvf, double* sig2,
                                                                float* Vprev, int warm, unsigned* flags) {
  extern __shared__ __align__(16) unsigned char smraw[];
  gram_finish(d, blockIdx.x, gpart, gsplit, G, Ginv, Ginvf, sig2, Vprev, warm, flags, smraw);
}

void launch_gram_finish(const ModeDesc& d, const double* Gpart, int nsplit, double* G, double* Ginv, float* Ginvf,
                        double* sig2, float* Vprev, int warm, unsigned* flags, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gram_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpdSmem);
    attr = true;
  }
  k_gram_finish<<<d.p, UPD_THREADS, kUpdSmem, s>>>(d, Gpart, nsplit, G, Ginv, Ginvf, sig2, Vprev, warm, flags);
  count_launch();
}

void launch_gram(const ModeDesc& d, const double* T, double* Gpart, int nsplit, double* G, double* Ginv,
                 float* Ginvf, double* sig2, float* Vprev, int warm, unsigned* flags, cudaStream_t s) {
  k_gram_partial<<<d.p * nsplit, UPD_THREADS, 0, s>>>(d, T, Gpart, nsplit); count_launch();
  launch_gram_finish(d, Gpart, nsplit, G, Ginv, Ginvf, sig2, Vprev, warm, flags, s);
}

template <typename Tc>
tdb_status launch_update(UpdArgs& a, int grid_hint, cudaStream_t s) {
  static int nsm_cache[2] = {0, 0};
  int& nsm = nsm_cache[sizeof(Tc) == 8 ? 1 : 0];
  if (nsm == 0) {
    int dev = 0, n = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return TDB_ERR_UNSUPPORTED;
    cudaFuncSetAttribute(k_update<Tc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpdSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update<Tc>, UPD_THREADS, kUpdSmem);
    if (per_sm < 1) return TDB_ERR_UNSUPPORTED;
    nsm = n;
  }
  // every CTA is resident (one per SM at most), so the grid barriers cannot deadlock
  const int grid = std::max(a.d.p, std::min(nsm, grid_hint));
  cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s);
  // cooperative launch through the extensible API, which stream capture records as a
  // cooperative kernel node
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(UPD_THREADS);
  cfg.dynamicSmemBytes = kUpdSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_update<Tc>, a);
  count_launch();
  return e == cudaSuccess ? TDB_OK : TDB_ERR_CUDA;
}
template tdb_status launch_update<float>(UpdArgs&, int, cudaStream_t);
template tdb_status launch_update<double>(UpdArgs&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Diagnostics (tdb_selftest_recip, tdb_selftest_timeout): the double reciprocal helpers
// over an array, and the update kernel's grid barrier waiting for one CTA more than the
// grid holds - an arrival that never comes - so that its bounded wait runs out.
// ---------------------------------------------------------------------------
__global__ void k_selftest_recip(const double* __restrict__ x, double* __restrict__ rcp, double* __restrict__ rs,
                                 int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    rcp[i] = drcp(v);
    rs[i] = v > 0.0 ? drsqrt(v) : 0.0;
  }
}

__global__ void k_selftest_gridwait(unsigned* bar, unsigned* flags, long long limit) {
  __shared__ int abort_sh;
  if (threadIdx.x == 0) abort_sh = 0;
  grid_sync(bar, 1u, gridDim.x + 1u, flags, &abort_sh, limit);
}

}  // namespace tdb

extern "C" tdb_status tdb_selftest_recip(const double* x, double* rcp, double* rsqrt, int64_t n, void* stream) {
  using namespace tdb;
  if (!x || !rcp || !rsqrt || n < 0) return TDB_ERR_INVALID_ARG;
  if (n == 0) return TDB_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  k_selftest_recip<<<blocks, 256, 0, s>>>(x, rcp, rsqrt, n);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return TDB_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? TDB_OK : TDB_ERR_CUDA;
}

extern "C" tdb_status tdb_selftest_timeout(int which, int64_t limit_cycles, unsigned* scratch, void* stream) {
  using namespace tdb;
  if (!scratch || limit_cycles < 1 || limit_cycles > 4000000000ll || (which != 0 && which != 1))
    return TDB_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(scratch, 0, 4 * sizeof(unsigned), s) != cudaSuccess) return TDB_ERR_CUDA;
  unsigned* flags = scratch + 2;
  if (which == 0) {
    // two co-resident CTAs (cooperative launch): the barrier's target is three arrivals
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(32);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_selftest_gridwait, scratch, flags, (long long)limit_cycles) != cudaSuccess)
      return TDB_ERR_CUDA;
    count_launch();
  } else {
    const tdb_status st = tc_selftest_mbar_wait(flags, (long long)limit_cycles, s);
    if (st != TDB_OK) return st;
  }
  unsigned h = 0;
  if (cudaMemcpyAsync(&h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TDB_ERR_CUDA;
  return (h & kFlagTimeout) ? TDB_ERR_TIMEOUT : TDB_OK;
}
