// k_mlp.cu - the learned error estimator: a two-hidden-layer perceptron
//   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3     (F -> 64 -> 64 -> 1)
// with mean-squared-error loss, back-propagation and Adam, in FP32.  The paper
// monitors the error by computing it (Eq. 2.20); the estimator predicts log10 of
// that error from reduced quantities so that most steps can skip the full pass,
// and the exact error stays the fallback and the only input to rank decisions.
//
// Parameter vector (float, MLP_NPARAM entries): W1 (H x F, row-major), b1 (H),
// W2 (H x H, row-major), b2 (H), w3 (H), b3 (1).
#include "common.cuh"
#include "kernels.h"
#include "mlp.h"

#include <cmath>

namespace tdb {

// One CTA of H = 64 threads walks a chunk of samples; thread j owns hidden unit j
// and accumulates its rows of the gradient in registers.
__global__ void __launch_bounds__(MLP_H) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                     const float* __restrict__ tgt, int n, int per_cta, float inv_n,
                                                     float* __restrict__ gpart, float* __restrict__ lpart) {
  constexpr int F = MLP_F, H = MLP_H;
  __shared__ float W2[H][H + 1];
  __shared__ float h1[H], da2[H], xs[F];
  __shared__ float red[2];
  const int j = threadIdx.x;
  const float* W1 = P;
  const float* b1 = W1 + H * F;
  const float* W2g = b1 + H;
  const float* b2 = W2g + H * H;
  const float* w3 = b2 + H;
  const float b3 = w3[H];
  for (int k = 0; k < H; ++k) W2[j][k] = W2g[j * H + k];
  float w1r[F];
#pragma unroll
  for (int f = 0; f < F; ++f) w1r[f] = W1[j * F + f];
  const float b1j = b1[j], b2j = b2[j], w3j = w3[j];
  float gW2[H], gW1[F];
#pragma unroll
  for (int k = 0; k < H; ++k) gW2[k] = 0.f;
#pragma unroll
  for (int f = 0; f < F; ++f) gW1[f] = 0.f;
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, loss = 0.f;
  __syncthreads();
  const int s0 = blockIdx.x * per_cta, s1 = min(n, s0 + per_cta);
  for (int s = s0; s < s1; ++s) {
    if (j < F) xs[j] = X[(size_t)s * F + j];
    __syncthreads();
    float a = b1j;
#pragma unroll
    for (int f = 0; f < F; ++f) a += w1r[f] * xs[f];
    const float h1j = tanhf(a);
    h1[j] = h1j;
    __syncthreads();
    float a2 = b2j;
#pragma unroll 16
    for (int k = 0; k < H; ++k) a2 += W2[j][k] * h1[k];
    const float h2j = tanhf(a2);
    float part = w3j * h2j;
    part = warp_sum(part);
    if ((j & 31) == 0) red[j >> 5] = part;
    __syncthreads();
    const float y = red[0] + red[1] + b3;
    const float r = y - tgt[s];
    const float dy = 2.f * r * inv_n;
    if (j == 0) { loss += r * r * inv_n; gb3 += dy; }
    gw3 += dy * h2j;
    const float d2 = dy * w3j * (1.f - h2j * h2j);
    da2[j] = d2;
    gb2 += d2;
#pragma unroll
    for (int k = 0; k < H; ++k) gW2[k] += d2 * h1[k];
    __syncthreads();
    // dh1_j = sum_i W2[i][j] da2_i
    float dh1 = 0.f;
#pragma unroll 16
    for (int i = 0; i < H; ++i) dh1 += W2[i][j] * da2[i];
    const float d1 = dh1 * (1.f - h1j * h1j);
    gb1 += d1;
#pragma unroll
    for (int f = 0; f < F; ++f) gW1[f] += d1 * xs[f];
    __syncthreads();
  }
  float* g = gpart + (size_t)blockIdx.x * MLP_NPARAM;
#pragma unroll
  for (int f = 0; f < F; ++f) g[j * F + f] = gW1[f];
  g[H * F + j] = gb1;
#pragma unroll
  for (int k = 0; k < H; ++k) g[H * F + H + j * H + k] = gW2[k];
  g[H * F + H + H * H + j] = gb2;
  g[H * F + H + H * H + H + j] = gw3;
  if (j == 0) {
    g[MLP_NPARAM - 1] = gb3;
    lpart[blockIdx.x] = loss;
  }
}

// Sum the per-CTA partial gradients (fixed order) and the loss.
__global__ void k_mlp_reduce(const float* __restrict__ gpart, const float* __restrict__ lpart, int nparts,
                             float* __restrict__ grad, float* __restrict__ loss) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < MLP_NPARAM; e += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int p = 0; p < nparts; ++p) s += gpart[(size_t)p * MLP_NPARAM + e];
    grad[e] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
    float s = 0.f;
    for (int p = 0; p < nparts; ++p) s += lpart[p];
    *loss = s;
  }
}

// Adam (Kingma and Ba) with bias correction; step counts from 1.
// omb1 = 1 - beta1 and omb2 = 1 - beta2 and the bias corrections c1, c2 are formed in
// double on the host (1 - 0.999f is not 1e-3 in float).
__global__ void k_mlp_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr, float beta1, float omb1, float beta2, float omb2, float c1,
                           float c2, float eps) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < MLP_NPARAM; e += gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = beta1 * m[e] + omb1 * ge;
    const float ve = beta2 * v[e] + omb2 * ge * ge;
    m[e] = me;
    v[e] = ve;
    P[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
  }
}

__global__ void __launch_bounds__(MLP_H) k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X,
                                                        int n, float* __restrict__ y) {
  constexpr int F = MLP_F, H = MLP_H;
  __shared__ float W2[H][H + 1];
  __shared__ float h1[H], xs[F];
  __shared__ float red[2];
  const int j = threadIdx.x;
  const float* W1 = P;
  const float* b1 = W1 + H * F;
  const float* W2g = b1 + H;
  const float* b2 = W2g + H * H;
  const float* w3 = b2 + H;
  for (int k = 0; k < H; ++k) W2[j][k] = W2g[j * H + k];
  __syncthreads();
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    if (j < F) xs[j] = X[(size_t)s * F + j];
    __syncthreads();
    float a = b1[j];
#pragma unroll
    for (int f = 0; f < F; ++f) a += W1[j * F + f] * xs[f];
    h1[j] = tanhf(a);
    __syncthreads();
    float a2 = b2[j];
    for (int k = 0; k < H; ++k) a2 += W2[j][k] * h1[k];
    float part = w3[j] * tanhf(a2);
    part = warp_sum(part);
    if ((j & 31) == 0) red[j >> 5] = part;
    __syncthreads();
    if (j == 0) y[s] = red[0] + red[1] + w3[H];
    __syncthreads();
  }
}

void mlp_loss_grad(const float* P, const float* X, const float* t, int n, float* gpart, float* lpart, int max_parts,
                   float* grad, float* loss, cudaStream_t s) {
  int parts = std::min(max_parts, std::max(1, (n + 31) / 32));
  int per = (n + parts - 1) / parts;
  k_mlp_grad<<<parts, MLP_H, 0, s>>>(P, X, t, n, per, 1.f / (float)n, gpart, lpart);
  count_launch();
  k_mlp_reduce<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(gpart, lpart, parts, grad, loss);
  count_launch();
}

void mlp_adam(float* P, const float* g, float* m, float* v, int step, float lr, cudaStream_t s) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, step)), c2 = (float)(1.0 - std::pow(b2, step));
  k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(P, g, m, v, lr, (float)b1, (float)(1.0 - b1), (float)b2,
                                                       (float)(1.0 - b2), c1, c2, 1e-8f);
  count_launch();
}

void mlp_forward(const float* P, const float* X, int n, float* y, cudaStream_t s) {
  k_mlp_forward<<<std::min(n, 1024), MLP_H, 0, s>>>(P, X, n, y);
  count_launch();
}

}  // namespace tdb

// ---------------------------------------------------------------------------
// Standalone C ABI of the estimator kernels (device buffers)
// ---------------------------------------------------------------------------
extern "C" {

int tdb_mlp_param_count(void) { return tdb::MLP_NPARAM; }

tdb_status tdb_mlp_forward(const float* params, const float* X, int n, float* y, void* stream) {
  if (!params || !X || !y || n < 0) return TDB_ERR_INVALID_ARG;
  if (n == 0) return TDB_OK;
  tdb::mlp_forward(params, X, n, y, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? TDB_OK : TDB_ERR_CUDA;
}

tdb_status tdb_mlp_loss_grad(const float* params, const float* X, const float* t, int n, float* scratch,
                             size_t scratch_floats, float* loss, float* grad, void* stream) {
  if (!params || !X || !t || !scratch || !grad || n < 1) return TDB_ERR_INVALID_ARG;
  int max_parts = (int)std::min<size_t>(1024, scratch_floats / (tdb::MLP_NPARAM + 1));
  if (max_parts < 1) return TDB_ERR_WORKSPACE;
  float* gpart = scratch;
  float* lpart = scratch + (size_t)max_parts * tdb::MLP_NPARAM;
  tdb::mlp_loss_grad(params, X, t, n, gpart, lpart, max_parts, grad, loss, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? TDB_OK : TDB_ERR_CUDA;
}

tdb_status tdb_mlp_adam_step(float* params, const float* grad, float* m, float* v, int step, float lr, void* stream) {
  if (!params || !grad || !m || !v || step < 1) return TDB_ERR_INVALID_ARG;
  tdb::mlp_adam(params, grad, m, v, step, lr, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? TDB_OK : TDB_ERR_CUDA;
}

}  // extern "C"

namespace tdb {

// Features (in this order): log10 of the previous step's error (exact, or the estimate
// when that step was skipped), log10 ||dV||_W, log10 of the residual sqrt(||dV||_W^2 -
// ||dS||^2) (the part of the step outside the current basis), log10 ||dS||, log10 of the
// smallest sigma_min / sigma_max over modes, log10 ||T||, log10(steps since the last
// re-initialisation + 1), log10 of the previous step's residual.  The network predicts
// the change of log10 error over the step, so the estimate chains from the previous
// error and the features do not depend on which steps were evaluated exactly.
__global__ void __launch_bounds__(256) k_est_features(const EstState* __restrict__ stp, const float* __restrict__ dS, int nds,
                                                      const double* __restrict__ dv2, const double* __restrict__ sig2,
                                                      int4 ranks, int p, const float* __restrict__ P,
                                                      const float* __restrict__ norm, float* __restrict__ feat,
                                                      double* __restrict__ est, int* __restrict__ need,
                                                      double* __restrict__ ds2_out) {
  // The features are float-valued and ||dS|| is only as accurate as the projection,
  // so everything is float except the difference ||dV||^2 - ||dS||^2 (double: it can
  // cancel).  One CTA; the launch is latency-bound, so every global load is issued up
  // front by the thread that uses it: the network's weights go straight to registers
  // (layer 1: thread j < H owns unit j; layer 2: four threads per unit, 16 inputs each),
  // warps 1 and 2 reduce the sigma^2 features while all threads sum ||dS||^2.
  constexpr int F = MLP_F, H = MLP_H;
  __shared__ double sh[32];
  __shared__ float xs[F], h1[H], red[8], nrm_s[2 * F + 2];
  __shared__ float tot_sh, smin_sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const float* W1 = P;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* w3 = b2 + H;
  const int j = tid >> 2, q = tid & 3;
  float w1r[F], w2r[H / 4];
  float b1v = 0.f;
  if (tid < H) {
#pragma unroll
    for (int f = 0; f < F; ++f) w1r[f] = W1[tid * F + f];
    b1v = b1[tid];
  }
#pragma unroll
  for (int k = 0; k < H / 4; ++k) w2r[k] = W2[j * H + q * (H / 4) + k];
  const float b2v = b2[j], w3v = w3[j];
  const float tiny = 1e-30f;
  const int rr[4] = {ranks.x, ranks.y, ranks.z, ranks.w};
  if (wid == 1) {                       // sum of the mode-1 sigma^2 (kept part)
    float v = lane < rr[0] ? fmaxf((float)sig2[lane], 0.f) : 0.f;
    v = warp_sum(v);
    if (lane == 0) tot_sh = v;
  } else if (wid == 2) {                // smallest sigma_min / sigma_max over the modes
    float v = 1.f;
    if (lane < p) {
      const double* sg = sig2 + lane * kMaxRank;
      const float mx = fmaxf((float)sg[0], tiny), mn = fmaxf((float)sg[rr[lane] - 1], tiny);
      v = sqrtf(mn / mx);
    }
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) smin_sh = v;
  } else if (wid == 3 && lane < 2 * F + 2) {
    nrm_s[lane] = norm[lane];
  }
  const EstState st = *stp;     // the host's estimator state of this step (device copy)
  // ||dS||^2: eight loads in flight per thread
  float sf = 0.f;
  for (int i0 = tid; i0 < nds; i0 += 8 * 256) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = i0 + k * 256 < nds ? dS[i0 + k * 256] : 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) sf = fmaf(v[k], v[k], sf);
  }
  const double s = block_sum((double)sf, sh);     // (its barriers also publish the values above)
  if (tid == 0) {
    const double d2 = *dv2;
    const float res2 = (float)fmax(d2 - s, 0.0);
    float f[F];
    f[0] = (float)st.last_log_eps;
    f[1] = log10f(sqrtf((float)d2) + tiny);
    f[2] = log10f(sqrtf(res2) + tiny);
    f[3] = log10f(sqrtf((float)s) + tiny);
    f[4] = log10f(smin_sh + tiny);
    f[5] = log10f(sqrtf(tot_sh) + tiny);
    f[6] = log10f((float)st.steps_since_reinit + 1.f);
    f[7] = (float)st.prev_res_log;
#pragma unroll
    for (int i = 0; i < F; ++i) {
      feat[i] = f[i];
      xs[i] = st.ready ? (f[i] - nrm_s[i]) / nrm_s[F + i] : 0.f;
    }
    *ds2_out = s;
  }
  __syncthreads();
  if (!st.ready) {
    if (tid == 0) { *need = 1; *est = nan(""); }
    return;
  }
  // forward pass of one sample
  if (tid < H) {
    float a = b1v;
#pragma unroll
    for (int f = 0; f < F; ++f) a = fmaf(w1r[f], xs[f], a);
    h1[tid] = tanhf(a);
  }
  __syncthreads();
  float a2 = 0.f;
#pragma unroll
  for (int k = 0; k < H / 4; ++k) a2 = fmaf(w2r[k], h1[q * (H / 4) + k], a2);
  a2 += __shfl_xor_sync(0xffffffffu, a2, 1);
  a2 += __shfl_xor_sync(0xffffffffu, a2, 2);
  float part = (q == 0) ? w3v * tanhf(a2 + b2v) : 0.f;
  part = warp_sum(part);
  if (lane == 0) red[wid] = part;
  __syncthreads();
  if (tid == 0) {
    float yz = w3[H];
    for (int w = 0; w < 8; ++w) yz += red[w];
    const float dlog = yz * nrm_s[2 * F + 1] + nrm_s[2 * F];
    const double e = (double)exp10f((float)st.last_log_eps + dlog);
    *est = e;
    bool novel = false;
    for (int i = 1; i < F; ++i)
      if (i != 6) novel |= fabsf(xs[i]) > (float)st.novelty_z;
    *need = (e > st.gate * st.eps_th ? 1 : 0) | (st.steps_since_exact >= st.max_skip ? 2 : 0) | (novel ? 4 : 0);
  }
}

void est_features(const EstState* st_dev, const float* dS, int nds, const double* dv2, const double* sig2,
                  const int* ranks, int p, const float* P, const float* norm, float* feat, double* est, int* need,
                  double* ds2, cudaStream_t s) {
  int4 rk = make_int4(ranks[0], p > 1 ? ranks[1] : 1, p > 2 ? ranks[2] : 1, p > 3 ? ranks[3] : 1);
  k_est_features<<<1, 256, 0, s>>>(st_dev, dS, nds, dv2, sig2, rk, p, P, norm, feat, est, need, ds2);
  count_launch();
}

// Standardise the trace in place: norm = [mean_f (F), sd_f (F), mean_t, sd_t].
__global__ void k_est_normalize(float* __restrict__ X, float* __restrict__ t, int n, float* __restrict__ norm) {
  __shared__ double sh[32];
  for (int c = 0; c <= MLP_F; ++c) {
    double s = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double v = c < MLP_F ? X[(size_t)i * MLP_F + c] : t[i];
      s += v;
      q += v * v;
    }
    s = block_sum(s, sh);
    q = block_sum(q, sh);
    const double mu = s / n;
    // scales floored at 0.05 (log10 units) so that a feature nearly constant in training
    // does not make every small drift look out of range
    const double sd = fmax(sqrt(fmax(q / n - mu * mu, 0.0)), 0.05);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (c < MLP_F) X[(size_t)i * MLP_F + c] = (float)((X[(size_t)i * MLP_F + c] - mu) / sd);
      else t[i] = (float)((t[i] - mu) / sd);
    }
    if (threadIdx.x == 0) {
      if (c < MLP_F) { norm[c] = (float)mu; norm[MLP_F + c] = (float)sd; }
      else { norm[2 * MLP_F] = (float)mu; norm[2 * MLP_F + 1] = (float)sd; }
    }
    __syncthreads();
  }
}

void est_normalize(float* X, float* t, int n, float* norm, cudaStream_t s) {
  k_est_normalize<<<1, 256, 0, s>>>(X, t, n, norm);
  count_launch();
}

// Glorot-uniform weights from a counter-based hash of (seed, index); zero biases.
__global__ void k_est_init(float* __restrict__ P, unsigned long long seed) {
  const int F = MLP_F, H = MLP_H;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < MLP_NPARAM; e += gridDim.x * blockDim.x) {
    unsigned long long h = seed * 0x9E3779B97F4A7C15ull + (unsigned long long)e * 0xBF58476D1CE4E5B9ull;
    h ^= h >> 31; h *= 0x94D049BB133111EBull; h ^= h >> 29;
    const float u = (float)((h >> 40) & 0xFFFFFF) / 16777216.0f * 2.f - 1.f;
    float a = 0.f;
    if (e < H * F) a = sqrtf(6.f / (F + H));
    else if (e >= H * F + H && e < H * F + H + H * H) a = sqrtf(6.f / (H + H));
    else if (e >= H * F + H + H * H + H && e < MLP_NPARAM - 1) a = sqrtf(6.f / (H + 1));
    P[e] = a * u;
  }
}

void est_init_params(float* P, unsigned long long seed, cudaStream_t s) {
  k_est_init<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(P, seed);
  count_launch();
}

}  // namespace tdb
