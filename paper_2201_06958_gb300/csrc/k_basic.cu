// k_basic.cu - elementwise kernels, weighted norms and the generic n-mode product.
//
// The n-mode product (Sec. 2.1) out = in x_n M, with M of shape J x K, is taken on
// the view in = (L, K, Q), out = (L, J, Q) (column-major, l fastest), where
// L = prod of the sizes before mode n and Q = prod of the sizes after it:
//     out[l + L (j + J q)] = sum_k M[j sMj + k sMk] in[l + L (k + K q)].
// It serves the unfused projection (M = A_n^T = (W_n U_n)^T, Eqs. 2.15/2.16),
// the reconstruction (M = U_n, Eq. 2.5) and the core compensation (M = R_n).
#include "common.cuh"
#include "kernels.h"

#include <atomic>

namespace tdb {

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Elementwise
// ---------------------------------------------------------------------------

// out = scale (a - b): the snapshot difference (scale 1), or a scaled central difference
template <typename T>
__global__ void k_diff(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out, int64_t n, T scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (a[i] - b[i]) * scale;
}

template <typename T>
void launch_diff(const T* a, const T* b, T* out, int64_t n, cudaStream_t s, T scale) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_diff<T><<<blocks, 256, 0, s>>>(a, b, out, n, scale); count_launch();
}
template void launch_diff<float>(const float*, const float*, float*, int64_t, cudaStream_t, float);
template void launch_diff<double>(const double*, const double*, double*, int64_t, cudaStream_t, double);

// A = W U in the compute type: A[i + N a] = w[i] U[i + N a]  (Eq. 2.17).
template <typename T>
__global__ void k_weighted_bases(const double* __restrict__ U, const double* __restrict__ w, T* __restrict__ A,
                                 int64_t N, int r) {
  const unsigned n = (unsigned)N, tot = (unsigned)(N * r);
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x)
    A[e] = (T)(w[e % n] * U[e]);
}

template <typename T>
void launch_weighted_bases(const double* U, const double* w, T* A, int64_t N, int r, cudaStream_t s) {
  int64_t n = N * r;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  k_weighted_bases<T><<<blocks, 256, 0, s>>>(U, w, A, N, r); count_launch();
}
template void launch_weighted_bases<float>(const double*, const double*, float*, int64_t, int, cudaStream_t);
template void launch_weighted_bases<double>(const double*, const double*, double*, int64_t, int, cudaStream_t);

template <typename Ts, typename Td>
__global__ void k_cast(const Ts* __restrict__ a, Td* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (Td)a[i];
}
template <typename Ts, typename Td>
void launch_cast(const Ts* a, Td* b, int64_t n, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  if (blocks < 1) blocks = 1;
  k_cast<Ts, Td><<<blocks, 256, 0, s>>>(a, b, n); count_launch();
}
template void launch_cast<double, float>(const double*, float*, int64_t, cudaStream_t);
template void launch_cast<float, double>(const float*, double*, int64_t, cudaStream_t);
template void launch_cast<double, double>(const double*, double*, int64_t, cudaStream_t);

// out = a + (double) b   (core Euler update T + dS, Sec. 2.3)
template <typename Tb>
__global__ void k_add(const double* __restrict__ a, const Tb* __restrict__ b, double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] + (double)b[i];
}
template <typename Tb>
void launch_add(const double* a, const Tb* b, double* out, int64_t n, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  if (blocks < 1) blocks = 1;
  k_add<Tb><<<blocks, 256, 0, s>>>(a, b, out, n); count_launch();
}
template void launch_add<float>(const double*, const float*, double*, int64_t, cudaStream_t);
template void launch_add<double>(const double*, const double*, double*, int64_t, cudaStream_t);

// ---------------------------------------------------------------------------
// Weighted squared norms (Eq. 2.2 with the quadrature of Eq. 2.17), deterministic:
// block partials in fixed order, then one block sums the partials in fixed order.
//   sum_i w_1(i_1) ... w_p(i_p) (x[i] - y[i])^2      (y may be null)
// Grid-stride over mode-1 columns; the product of the other weights is formed
// once per column.
// ---------------------------------------------------------------------------


template <typename T>
__global__ void k_wnorm2_partial(const T* __restrict__ x, const T* __restrict__ y, WeightView wv,
                                 double* __restrict__ partial, unsigned* flags) {
  __shared__ double sh[32];
  const int64_t N1 = wv.N[0];
  int64_t ncol = 1;
  for (int m = 1; m < wv.p; ++m) ncol *= wv.N[m];
  double acc = 0.0;
  bool bad = false;
  for (int64_t c = blockIdx.x; c < ncol; c += gridDim.x) {
    double wc = 1.0;
    unsigned rem = (unsigned)c;
    for (int m = 1; m < wv.p; ++m) {
      const unsigned nm = (unsigned)wv.N[m];
      wc *= wv.w[m][rem % nm];
      rem /= nm;
    }
    const T* xc = x + c * N1;
    const T* yc = y ? y + c * N1 : nullptr;
    T s = 0;                 // per-thread partial over <= N1 / blockDim terms in the data type
    for (int64_t i = threadIdx.x; i < N1; i += blockDim.x) {
      T d = xc[i] - (yc ? yc[i] : T(0));
      bad |= !isfinite((double)d);
      s += (T)wv.w[0][i] * d * d;
    }
    acc += wc * (double)s;
  }
  acc = block_sum(acc, sh);
  if (bad && flags) atomicOr(flags, kFlagNonFinite);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

template <typename T>
void launch_wnorm2(const T* x, const T* y, const WeightView& wv, double* partial, int nblocks, double* out,
                   unsigned* flags, cudaStream_t s) {
  k_wnorm2_partial<T><<<nblocks, 256, 0, s>>>(x, y, wv, partial, flags); count_launch();
  k_sum_partials<<<1, 256, 0, s>>>(partial, nblocks, out); count_launch();
}
template void launch_wnorm2<float>(const float*, const float*, const WeightView&, double*, int, double*, unsigned*,
                                   cudaStream_t);
template void launch_wnorm2<double>(const double*, const double*, const WeightView&, double*, int, double*,
                                    unsigned*, cudaStream_t);

// Exact error of Eq. 2.20 without materialising V^TDB: with H = T x_2 U_2 ... x_p U_p
// (r_1 x N_2 x ... x N_p), every mode-1 column of the reconstruction is U_1 H[:, c].
// One warp per column, U_1 and w_1 staged in shared memory when they fit, the
// column's H values broadcast by shuffles; w_1 and the column weights
// w_c = prod_{m>1} w_m(i_m) in the compute type; per-column sums in the compute type,
// double across columns.  Float with N_1 % 4 == 0: lanes own float4 row groups and a
// warp works on two columns at once with all their loads issued before the
// arithmetic (the pass is bound by how many bytes of V are in flight).  The last CTA
// to finish adds the per-CTA partials in a fixed order and writes *out (no second
// launch); `counter` is zero before and after.
template <typename T>
__global__ void __launch_bounds__(256) k_recon_err(const T* __restrict__ V, const T* __restrict__ U1,
                                                   const T* __restrict__ H, int r1, int N1, unsigned ncol,
                                                   const T* __restrict__ w1, const T* __restrict__ wcol,
                                                   int stage_u1, double* __restrict__ partial,
                                                   unsigned* __restrict__ counter, double* __restrict__ out,
                                                   unsigned* flags, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;          // the estimator ruled this evaluation out
  extern __shared__ __align__(16) unsigned char sm_re[];
  T* U1s = (T*)sm_re;
  T* w1s = U1s + (size_t)N1 * r1;
  __shared__ double sh[32];
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const T* Usrc = U1;
  const T* wsrc = w1;
  if (stage_u1) {
    // every load of the staging issued before the first store (eight per thread in flight)
    bool vec = false;
    if constexpr (sizeof(T) == 4) vec = (N1 & 3) == 0;
    if (vec) {
      const float4* su = reinterpret_cast<const float4*>(U1);
      float4* du = reinterpret_cast<float4*>(U1s);
      const int nu4 = N1 * r1 / 4, nw4 = N1 / 4;
#pragma unroll 8
      for (int e = tid; e < nu4; e += blockDim.x) du[e] = __ldg(&su[e]);
#pragma unroll 4
      for (int e = tid; e < nw4; e += blockDim.x)
        reinterpret_cast<float4*>(w1s)[e] = __ldg(&reinterpret_cast<const float4*>(w1)[e]);
    } else {
#pragma unroll 8
      for (int e = tid; e < N1 * r1; e += blockDim.x) U1s[e] = U1[e];
#pragma unroll 4
      for (int e = tid; e < N1; e += blockDim.x) w1s[e] = w1[e];
    }
    __syncthreads();
    Usrc = U1s;
    wsrc = w1s;
  }
  double acc = 0.0;
  bool bad = false;
  const unsigned gw = blockIdx.x * nw + warp, tw = gridDim.x * nw;
  bool done = false;
  if constexpr (sizeof(T) == 4) {
    if (stage_u1 && (N1 & 3) == 0) {
      const int n4 = N1 >> 2;
      const float4* U4 = reinterpret_cast<const float4*>(Usrc);
      const float4* w4 = reinterpret_cast<const float4*>(wsrc);
      const float4* V4 = reinterpret_cast<const float4*>(V);
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (unsigned c0 = gw; c0 < ncol; c0 += 2 * tw) {
        const unsigned c1 = c0 + tw;
        const bool has1 = c1 < ncol;
        const float hl0 = lane < r1 ? H[lane + (size_t)r1 * c0] : 0.f;
        const float hl1 = (has1 && lane < r1) ? H[lane + (size_t)r1 * c1] : 0.f;
        float s0 = 0.f, s1 = 0.f;
        for (int g0 = 0; g0 < n4; g0 += 128) {
          float4 v0[4], v1[4], q0[4], q1[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int g = g0 + lane + 32 * t;
            v0[t] = g < n4 ? V4[(size_t)n4 * c0 + g] : z4;
            v1[t] = (has1 && g < n4) ? V4[(size_t)n4 * c1 + g] : z4;
            q0[t] = z4;
            q1[t] = z4;
          }
          for (int a = 0; a < r1; ++a) {
            const float h0 = __shfl_sync(0xffffffffu, hl0, a), h1 = __shfl_sync(0xffffffffu, hl1, a);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int g = g0 + lane + 32 * t;
              if (g < n4) {
                const float4 u = U4[(size_t)n4 * a + g];
                q0[t].x = fmaf(u.x, h0, q0[t].x); q0[t].y = fmaf(u.y, h0, q0[t].y);
                q0[t].z = fmaf(u.z, h0, q0[t].z); q0[t].w = fmaf(u.w, h0, q0[t].w);
                q1[t].x = fmaf(u.x, h1, q1[t].x); q1[t].y = fmaf(u.y, h1, q1[t].y);
                q1[t].z = fmaf(u.z, h1, q1[t].z); q1[t].w = fmaf(u.w, h1, q1[t].w);
              }
            }
          }
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int g = g0 + lane + 32 * t;
            if (g < n4) {
              const float4 w = w4[g];
              const float d0[4] = {v0[t].x - q0[t].x, v0[t].y - q0[t].y, v0[t].z - q0[t].z, v0[t].w - q0[t].w};
              const float d1[4] = {v1[t].x - q1[t].x, v1[t].y - q1[t].y, v1[t].z - q1[t].z, v1[t].w - q1[t].w};
              const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                bad |= !isfinite(d0[u]) || !isfinite(d1[u]);
                s0 += wv[u] * d0[u] * d0[u];
                s1 += wv[u] * d1[u] * d1[u];
              }
            }
          }
        }
        acc += (double)(wcol[c0] * s0);
        if (has1) acc += (double)(wcol[c1] * s1);
      }
      done = true;
    }
  }
  if (!done) {
    for (unsigned c = gw; c < ncol; c += tw) {
      const T hl = lane < r1 ? H[lane + (size_t)r1 * c] : T(0);
      T h[32];
#pragma unroll
      for (int a = 0; a < 32; ++a) h[a] = __shfl_sync(0xffffffffu, hl, a);
      const T* vc = V + (size_t)N1 * c;
      T s = T(0);
      for (int i = lane; i < N1; i += 32) {
        T rec = T(0);
#pragma unroll
        for (int a = 0; a < 32; ++a)
          if (a < r1) rec += Usrc[i + N1 * a] * h[a];
        const T d = vc[i] - rec;
        bad |= !isfinite(d);
        s += wsrc[i] * d * d;
      }
      acc += (double)(wcol[c] * s);
    }
  }
  acc = block_sum(acc, sh);
  if (bad && flags) atomicOr(flags, kFlagNonFinite);
  if (tid == 0) {
    partial[blockIdx.x] = acc;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int k = tid; k < (int)gridDim.x; k += blockDim.x) t += __ldcg(&partial[k]);
  t = block_sum(t, sh);
  if (tid == 0) {
    *out = t;
    atomicExch(counter, 0u);
  }
}

// Float exact error, row-major variant: lane l of a warp owns rows i0 + R l .. i0 + R l + R - 1
// of a block of 32 R rows, with U_1 of those rows (R x r_1) and w_1 in registers, and walks a
// contiguous range of columns c.  Each column's R rows per lane, H[:, c] (lanes < r_1) and
// w_c (lane 0) arrive by cp.async into a ring of D column slots per warp (D columns in
// flight per warp, no registers held); H[:, c] is broadcast by shuffles.  Per column the
// lane forms U_1 H[:, c] for its rows, the weighted squared difference, and adds w_c times
// it to a float sum that goes into the double accumulator every D columns.
constexpr int RE_D = 8;           // columns in flight per warp
template <int R>
__device__ __forceinline__ void cp_async_rows(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 4 * R : 0;
  if (R == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
  else if (R == 2)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int R, int RM>
__global__ void __launch_bounds__(256, 2) k_recon_err_rows(const float* __restrict__ V, const float* __restrict__ U1,
                                                         const float* __restrict__ H, int r1, int N1, unsigned ncol,
                                                         const float* __restrict__ w1, const float* __restrict__ wcol,
                                                         int vec, double* __restrict__ partial,
                                                         unsigned* __restrict__ counter, double* __restrict__ out,
                                                         unsigned* flags, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;          // the estimator ruled this evaluation out
  constexpr int SLOT = 32 * R + RM + 4;    // floats per column slot: rows, H[:, c] (zero past r_1), w_c
  __shared__ __align__(16) float ring[8][RE_D][SLOT];
  __shared__ double sh[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float (*slot)[SLOT] = ring[wib];
  // H entries past r_1 are never copied: zero them once (they meet zero rows of U_1)
  for (int e = lane; e < RE_D * RM; e += 32) slot[e / RM][32 * R + e % RM] = 0.f;
  __syncwarp();
  const int nrb = (N1 + 32 * R - 1) / (32 * R);
  const unsigned gw = blockIdx.x * (blockDim.x >> 5) + wib, tw = gridDim.x * (blockDim.x >> 5);
  const unsigned wpr = tw >= (unsigned)nrb ? tw / nrb : 1u;   // warps per row block
  double acc = 0.0;
  bool bad = false;
  const unsigned kk = gw % wpr;
  const unsigned c_lo = (unsigned)((uint64_t)ncol * kk / wpr), c_hi = (unsigned)((uint64_t)ncol * (kk + 1) / wpr);
  if (gw < wpr * (unsigned)nrb && c_lo < c_hi) {
    const int rb = (int)(gw / wpr);
    const int i0 = rb * 32 * R + R * lane;
    float u[R][RM], wr[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = i0 + q;
      wr[q] = i < N1 ? w1[i] : 0.f;
#pragma unroll
      for (int a = 0; a < RM; ++a) u[q][a] = (i < N1 && a < r1) ? U1[i + (size_t)N1 * a] : 0.f;
    }
    // source pointers of the next column to issue, advanced by one column per issue; past
    // c_hi the copies read nothing (zero bytes) from the last valid column
    const bool rows_in = i0 < N1;
    const float* vsrc = V + (size_t)N1 * c_lo + (rows_in ? i0 : 0);
    const float* hsrc = H + (size_t)r1 * c_lo + (lane < r1 ? lane : 0);
    const float* wsrc = wcol + c_lo;
    unsigned cnext = c_lo;
    auto issue = [&](int sl) {
      const bool in = cnext < c_hi;
      if (vec) {
        cp_async_rows<R>(&slot[sl][R * lane], vsrc, in && rows_in);
      } else {
#pragma unroll
        for (int q = 0; q < R; ++q) cp_async4(&slot[sl][R * lane + q], vsrc + (i0 + q < N1 ? q : 0), in && i0 + q < N1);
      }
      if (lane < r1) cp_async4(&slot[sl][32 * R + lane], hsrc, in);
      if (lane == 0) cp_async4(&slot[sl][32 * R + RM], wsrc, in);
      cp_async_commit();
      if (in && cnext + 1 < c_hi) {
        vsrc += N1;
        hsrc += r1;
        wsrc += 1;
      }
      ++cnext;
    };
#pragma unroll
    for (int t = 0; t < RE_D; ++t) issue(t);
    float csum = 0.f;
    int sl = 0;
    for (unsigned c = c_lo; c < c_hi; ++c) {
      cp_async_wait<RE_D - 1>();           // this column's copies (the oldest group) have landed
      __syncwarp();
      float v[R], h[RM];
      if (R == 4) {
        const float4 t4 = *reinterpret_cast<const float4*>(&slot[sl][4 * lane]);
        v[0] = t4.x; v[1 % R] = t4.y; v[2 % R] = t4.z; v[3 % R] = t4.w;
      } else if (R == 2) {
        const float2 t2 = *reinterpret_cast<const float2*>(&slot[sl][2 * lane]);
        v[0] = t2.x; v[1 % R] = t2.y;
      } else {
        v[0] = slot[sl][lane];
      }
#pragma unroll
      for (int j = 0; j < RM / 4; ++j) {
        const float4 t4 = *reinterpret_cast<const float4*>(&slot[sl][32 * R + 4 * j]);
        h[4 * j] = t4.x; h[4 * j + 1] = t4.y; h[4 * j + 2] = t4.z; h[4 * j + 3] = t4.w;
      }
      const float wc = slot[sl][32 * R + RM];
      __syncwarp();
      issue(sl);                           // the slot refills with the column D ahead
      float rec[R];
#pragma unroll
      for (int q = 0; q < R; ++q) rec[q] = 0.f;
#pragma unroll
      for (int a = 0; a < RM; ++a)
#pragma unroll
        for (int q = 0; q < R; ++q) rec[q] = fmaf(u[q][a], h[a], rec[q]);
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const float d = v[q] - rec[q];
        s = fmaf(wr[q] * d, d, s);
      }
      csum = fmaf(wc, s, csum);
      if (++sl == RE_D) {
        sl = 0;
        bad |= !isfinite(csum);
        acc += (double)csum;
        csum = 0.f;
      }
    }
    cp_async_wait<0>();
    bad |= !isfinite(csum);
    acc += (double)csum;
  }
  acc = block_sum(acc, sh);
  if (bad && flags) atomicOr(flags, kFlagNonFinite);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = acc;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(&partial[b]);
  t = block_sum(t, sh);
  if (threadIdx.x == 0) {
    *out = t;
    atomicExch(counter, 0u);
  }
}

template <typename T>
void launch_recon_err(const T* V, const T* U1, const T* H, int r1, int N1, int64_t ncol, const T* w1, const T* wcol,
                      double* partial, unsigned* counter, int nblocks, double* out, unsigned* flags, cudaStream_t s,
                      const int* gate) {
  if constexpr (sizeof(T) == 4) {
    // the row-major variant: U_1 in registers, cp.async column ring
    const uintptr_t va = (uintptr_t)V;
    const int vec4 = (N1 % 4) == 0 && va % 16 == 0, vec2 = (N1 % 2) == 0 && va % 8 == 0;
    const int blocks = std::max(1, std::min(nblocks, 2 * 152));
    if (r1 <= 8)
      k_recon_err_rows<4, 8><<<blocks, 256, 0, s>>>(V, U1, H, r1, N1, (unsigned)ncol, w1, wcol, vec4, partial,
                                                    counter, out, flags, gate);
    else if (r1 <= 16)
      k_recon_err_rows<4, 16><<<blocks, 256, 0, s>>>(V, U1, H, r1, N1, (unsigned)ncol, w1, wcol, vec4, partial,
                                                     counter, out, flags, gate);
    else
      k_recon_err_rows<2, 32><<<blocks, 256, 0, s>>>(V, U1, H, r1, N1, (unsigned)ncol, w1, wcol, vec2, partial,
                                                     counter, out, flags, gate);
    count_launch();
    return;
  }
  const size_t st_bytes = (size_t)N1 * (r1 + 1) * sizeof(T);
  const int stage = st_bytes <= 96 * 1024 ? 1 : 0;
  static bool attr[2] = {false, false};
  if (stage && !attr[sizeof(T) == 8]) {
    cudaFuncSetAttribute(k_recon_err<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr[sizeof(T) == 8] = true;
  }
  // float4 path: two columns per warp and iteration
  const int per_block = (sizeof(T) == 4 && stage && N1 % 4 == 0) ? 16 : 8;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(nblocks, (ncol + per_block - 1) / per_block));
  k_recon_err<T><<<blocks, 256, stage ? st_bytes : 0, s>>>(V, U1, H, r1, N1, (unsigned)ncol, w1, wcol, stage,
                                                           partial, counter, out, flags, gate);
  count_launch();
}
template void launch_recon_err<float>(const float*, const float*, const float*, int, int, int64_t, const float*,
                                      const float*, double*, unsigned*, int, double*, unsigned*, cudaStream_t,
                                      const int*);
template void launch_recon_err<double>(const double*, const double*, const double*, int, int, int64_t, const double*,
                                       const double*, double*, unsigned*, int, double*, unsigned*, cudaStream_t,
                                       const int*);

// Weights in the compute type: w_1 (N_1) and the column weights of the mode-1 unfolding,
// w_c = prod_{m>1} w_m(i_m) for c = i_2 + N_2 (i_3 + ...).
template <typename T>
__global__ void k_weights_T(WeightView wv, T* __restrict__ w1, T* __restrict__ wcol) {
  const unsigned N1 = (unsigned)wv.N[0];
  unsigned ncol = 1;
  for (int m = 1; m < wv.p; ++m) ncol *= (unsigned)wv.N[m];
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < N1 + ncol; e += gridDim.x * blockDim.x) {
    if (e < N1) {
      w1[e] = (T)wv.w[0][e];
    } else {
      unsigned rem = e - N1;
      double wc = 1.0;
      for (int m = 1; m < wv.p; ++m) {
        const unsigned nm = (unsigned)wv.N[m];
        wc *= wv.w[m][rem % nm];
        rem /= nm;
      }
      wcol[e - N1] = (T)wc;
    }
  }
}

template <typename T>
void launch_weights_T(const WeightView& wv, T* w1, T* wcol, cudaStream_t s) {
  k_weights_T<T><<<152, 256, 0, s>>>(wv, w1, wcol);
  count_launch();
}
template void launch_weights_T<float>(const WeightView&, float*, float*, cudaStream_t);
template void launch_weights_T<double>(const WeightView&, double*, double*, cudaStream_t);

void launch_sum_partials(const double* partial, int n, double* out, cudaStream_t s) {
  k_sum_partials<<<1, 256, 0, s>>>(partial, n, out); count_launch();
}

// ---------------------------------------------------------------------------
// Generic n-mode product
// ---------------------------------------------------------------------------

// K large, L == 1: one warp per output column q, lanes split k, JT accumulators.
template <typename Tin, typename Tm, typename Tacc, int JT>
__global__ void k_mp_reduce_col(const Tin* __restrict__ in, Tacc* __restrict__ out, const Tm* __restrict__ M, int K,
                                int J, int64_t Q, int64_t sMj, int64_t sMk) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = warp; q < Q; q += nwarps) {
    const Tin* col = in + q * K;
    for (int j0 = 0; j0 < J; j0 += JT) {
      Tacc acc[JT];
#pragma unroll
      for (int t = 0; t < JT; ++t) acc[t] = Tacc(0);
      for (int k = lane; k < K; k += 32) {
        Tacc v = (Tacc)col[k];
#pragma unroll
        for (int t = 0; t < JT; ++t)
          if (j0 + t < J) acc[t] += (Tacc)M[(j0 + t) * sMj + k * sMk] * v;
      }
#pragma unroll
      for (int t = 0; t < JT; ++t) {
        Tacc v = warp_sum(acc[t]);
        if (lane == 0 && j0 + t < J) out[(j0 + t) + (int64_t)J * q] = v;
      }
    }
  }
}

// K large, Q == 1, J <= 32: out (L x J) = in (L x K) M^T as a tiled product.  A CTA
// owns 64 consecutive l and all j; K in chunks of 32 staged in shared memory (in along
// l: coalesced; M once per chunk), the next chunk loaded into registers while the
// current one is multiplied; thread (tl, tj) accumulates l = 4 tl .. 4 tl + 3 and
// j = 2 tj, 2 tj + 1.  Fixed summation order over k.
template <typename Tin, typename Tm, typename Tacc>
__global__ void __launch_bounds__(256) k_mp_gemm(const Tin* __restrict__ in, Tacc* __restrict__ out,
                                                 const Tm* __restrict__ M, int64_t L, int K, int J, int64_t sMj,
                                                 int64_t sMk) {
  constexpr int BM = 64, BK = 32;
  __shared__ Tacc As[BK][BM + 1];
  __shared__ Tacc Bs[BK][33];
  const int tid = threadIdx.x;
  const int tl = tid & 15, tj = tid >> 4;
  for (int64_t l0 = blockIdx.x * (int64_t)BM; l0 < L; l0 += (int64_t)gridDim.x * BM) {
    Tacc acc[4][2];
#pragma unroll
    for (int x = 0; x < 4; ++x) acc[x][0] = acc[x][1] = Tacc(0);
    // register staging of one chunk: 8 entries of in, 4 of M per thread
    Tacc ra[8], rb[4];
    auto fetch = [&](int k0) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = tid + 256 * u, i = e % BM, kk = e / BM;
        const int64_t l = l0 + i;
        const int k = k0 + kk;
        ra[u] = (l < L && k < K) ? (Tacc)in[l + L * (int64_t)k] : Tacc(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + 256 * u, j = e % 32, kk = e / 32;
        const int k = k0 + kk;
        rb[u] = (j < J && k < K) ? (Tacc)M[j * sMj + (int64_t)k * sMk] : Tacc(0);
      }
    };
    fetch(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = tid + 256 * u;
        As[e / BM][e % BM] = ra[u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + 256 * u;
        Bs[e / 32][e % 32] = rb[u];
      }
      __syncthreads();
      if (k0 + BK < K) fetch(k0 + BK);
#pragma unroll 8
      for (int kk = 0; kk < BK; ++kk) {
        Tacc a[4], b[2];
#pragma unroll
        for (int x = 0; x < 4; ++x) a[x] = As[kk][4 * tl + x];
        b[0] = Bs[kk][2 * tj];
        b[1] = Bs[kk][2 * tj + 1];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          acc[x][0] = fma(a[x], b[0], acc[x][0]);
          acc[x][1] = fma(a[x], b[1], acc[x][1]);
        }
      }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const int64_t l = l0 + 4 * tl + x;
        const int j = 2 * tj + y;
        if (l < L && j < J) out[l + L * (int64_t)j] = acc[x][y];
      }
  }
}

// K large, L > 1: one thread per (l, q), l fastest (coalesced over l).
template <typename Tin, typename Tm, typename Tacc, int JT>
__global__ void k_mp_reduce_gen(const Tin* __restrict__ in, Tacc* __restrict__ out, const Tm* __restrict__ M,
                                int64_t L, int K, int J, int64_t Q, int64_t sMj, int64_t sMk) {
  const unsigned total = (unsigned)(L * Q), uL = (unsigned)L;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const unsigned l = e % uL, q = e / uL;
    const Tin* base = in + l + (size_t)uL * K * q;
    for (int j0 = 0; j0 < J; j0 += JT) {
      Tacc acc[JT];
#pragma unroll
      for (int t = 0; t < JT; ++t) acc[t] = Tacc(0);
      for (int k = 0; k < K; ++k) {
        Tacc v = (Tacc)base[(int64_t)k * L];
#pragma unroll
        for (int t = 0; t < JT; ++t)
          if (j0 + t < J) acc[t] += (Tacc)M[(j0 + t) * sMj + k * sMk] * v;
      }
#pragma unroll
      for (int t = 0; t < JT; ++t)
        if (j0 + t < J) out[l + L * ((j0 + t) + (int64_t)J * q)] = acc[t];
    }
  }
}

// K large, L * Q small: one warp per (l, q), lanes split k, JT accumulators.
template <typename Tin, typename Tm, typename Tacc, int JT>
__global__ void k_mp_reduce_warp(const Tin* __restrict__ in, Tacc* __restrict__ out, const Tm* __restrict__ M,
                                 int64_t L, int K, int J, int64_t Q, int64_t sMj, int64_t sMk) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned uL = (unsigned)L;
  for (int64_t w = warp; w < L * Q; w += nwarps) {
    const unsigned l = (unsigned)w % uL, q = (unsigned)w / uL;
    const Tin* base = in + l + (size_t)uL * K * q;
    for (int j0 = 0; j0 < J; j0 += JT) {
      Tacc acc[JT];
#pragma unroll
      for (int t = 0; t < JT; ++t) acc[t] = Tacc(0);
      for (int k = lane; k < K; k += 32) {
        Tacc v = (Tacc)base[(int64_t)k * L];
#pragma unroll
        for (int t = 0; t < JT; ++t)
          if (j0 + t < J) acc[t] += (Tacc)M[(j0 + t) * sMj + k * sMk] * v;
      }
#pragma unroll
      for (int t = 0; t < JT; ++t) {
        Tacc v = warp_sum(acc[t]);
        if (lane == 0 && j0 + t < J) out[l + L * ((j0 + t) + (int64_t)J * q)] = v;
      }
    }
  }
}

// K large, very few (l, q): one block per (l, q), threads split k, block reduction.
template <typename Tin, typename Tm, typename Tacc, int JT>
__global__ void k_mp_reduce_block(const Tin* __restrict__ in, Tacc* __restrict__ out, const Tm* __restrict__ M,
                                  int64_t L, int K, int J, int64_t Q, int64_t sMj, int64_t sMk) {
  __shared__ Tacc sh[JT][33];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned uL = (unsigned)L;
  for (unsigned w = blockIdx.x; w < (unsigned)(L * Q); w += gridDim.x) {
    const unsigned l = w % uL, q = w / uL;
    const Tin* base = in + l + (size_t)uL * K * q;
    for (int j0 = 0; j0 < J; j0 += JT) {
      Tacc acc[JT];
#pragma unroll
      for (int t = 0; t < JT; ++t) acc[t] = Tacc(0);
      for (int k = threadIdx.x; k < K; k += blockDim.x) {
        Tacc v = (Tacc)base[(size_t)k * uL];
#pragma unroll
        for (int t = 0; t < JT; ++t)
          if (j0 + t < J) acc[t] += (Tacc)M[(j0 + t) * sMj + k * sMk] * v;
      }
#pragma unroll
      for (int t = 0; t < JT; ++t) {
        Tacc v = warp_sum(acc[t]);
        if (lane == 0) sh[t][wid] = v;
      }
      __syncthreads();
      if (threadIdx.x < JT && j0 + (int)threadIdx.x < J) {
        Tacc v = Tacc(0);
        for (int x = 0; x < nw; ++x) v += sh[threadIdx.x][x];
        out[l + uL * ((j0 + threadIdx.x) + (size_t)J * q)] = v;
      }
      __syncthreads();
    }
  }
}

// K small: one thread per output element (l, j, q), l fastest.
template <typename Tin, typename Tm, typename Tacc>
__global__ void k_mp_expand(const Tin* __restrict__ in, Tacc* __restrict__ out, const Tm* __restrict__ M, int64_t L,
                            int K, int J, int64_t Q, int64_t sMj, int64_t sMk, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const unsigned total = (unsigned)(L * J * Q), uL = (unsigned)L, uJ = (unsigned)J;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const unsigned l = e % uL;
    const unsigned jq = e / uL;
    const unsigned j = jq % uJ;
    const unsigned q = jq / uJ;
    const Tin* base = in + l + (size_t)uL * K * q;
    const Tm* mrow = M + j * sMj;
    Tacc acc = Tacc(0);
    for (int k = 0; k < K; ++k) acc += (Tacc)mrow[k * sMk] * (Tacc)base[(size_t)k * uL];
    out[e] = acc;
  }
}

template <typename Tin, typename Tm, typename Tacc>
void launch_modeprod(const Tin* in, Tacc* out, const Tm* M, int64_t L, int K, int J, int64_t Q, int64_t sMj,
                     int64_t sMk, cudaStream_t s, const int* gate) {
  if (L <= 0 || K <= 0 || J <= 0 || Q <= 0) return;
  count_launch();
  if (K <= 64) {
    int64_t total = L * J * Q;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    k_mp_expand<Tin, Tm, Tacc><<<blocks, 256, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk, gate);
  } else if (Q == 1 && L >= 64 && J <= 32) {
    const int blocks = (int)std::min<int64_t>((L + 63) / 64, 152 * 8);
    k_mp_gemm<Tin, Tm, Tacc><<<blocks, 256, 0, s>>>(in, out, M, L, K, J, sMj, sMk);
  } else if (L > 1 && L * Q <= 1024) {
    int blocks = (int)std::min<int64_t>(L * Q, 152 * 8);
    if (J <= 8)
      k_mp_reduce_block<Tin, Tm, Tacc, 8><<<blocks, 256, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk);
    else if (J <= 16)
      k_mp_reduce_block<Tin, Tm, Tacc, 16><<<blocks, 256, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk);
    else
      k_mp_reduce_block<Tin, Tm, Tacc, 32><<<blocks, 256, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk);
  } else if (L > 1 && L * Q <= 32768) {
    int64_t warps = L * Q;
    int blocks = (int)std::min<int64_t>((warps * 32 + 255) / 256, 152 * 32);
    if (J <= 8)
      k_mp_reduce_warp<Tin, Tm, Tacc, 8><<<blocks, 256, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk);
    else if (J <= 16)
      k_mp_reduce_warp<Tin, Tm, Tacc, 16><<<blocks, 256, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk);
    else
      k_mp_reduce_warp<Tin, Tm, Tacc, 32><<<blocks, 256, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk);
  } else if (L == 1) {
    int64_t warps = Q;
    int blocks = (int)std::min<int64_t>((warps * 32 + 255) / 256, 152 * 32);
    if (J <= 8)
      k_mp_reduce_col<Tin, Tm, Tacc, 8><<<blocks, 256, 0, s>>>(in, out, M, K, J, Q, sMj, sMk);
    else if (J <= 16)
      k_mp_reduce_col<Tin, Tm, Tacc, 16><<<blocks, 256, 0, s>>>(in, out, M, K, J, Q, sMj, sMk);
    else
      k_mp_reduce_col<Tin, Tm, Tacc, 32><<<blocks, 256, 0, s>>>(in, out, M, K, J, Q, sMj, sMk);
  } else {
    int64_t total = L * Q;
    int blocks = (int)std::min<int64_t>((total + 127) / 128, 152 * 32);
    if (J <= 8)
      k_mp_reduce_gen<Tin, Tm, Tacc, 8><<<blocks, 128, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk);
    else if (J <= 16)
      k_mp_reduce_gen<Tin, Tm, Tacc, 16><<<blocks, 128, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk);
    else
      k_mp_reduce_gen<Tin, Tm, Tacc, 32><<<blocks, 128, 0, s>>>(in, out, M, L, K, J, Q, sMj, sMk);
  }
}

#define INST_MP(Tin, Tm, Tacc)                                                                                   \
  template void launch_modeprod<Tin, Tm, Tacc>(const Tin*, Tacc*, const Tm*, int64_t, int, int, int64_t, int64_t, \
                                               int64_t, cudaStream_t, const int*);
INST_MP(float, float, float)
INST_MP(double, double, double)
INST_MP(double, float, float)
INST_MP(float, double, double)
INST_MP(double, double, float)

}  // namespace tdb
