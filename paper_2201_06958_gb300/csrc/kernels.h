// kernels.h - host-side launchers of libtdb's kernels (internal C++ interface).
#pragma once

#include <algorithm>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace tdb {

// Bump allocator over the caller's workspace (256-byte aligned pieces); with a
// null base it only measures.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};


struct WeightView {
  int p;
  int64_t N[kMaxModes];
  const double* w[kMaxModes];
};

struct RowArgs {
  ModeDesc d;
  const void* Y[kMaxModes];      // projection tensors (Tc)
  const void* Tc;                // core in the compute type
  const double* U[kMaxModes];
  const double* w[kMaxModes];
  const double* Ginv;            // p x LD x LD
  const double* P;               // p x LD x LD
  const double* Rinv;            // p x LD x LD
  double* X[kMaxModes];
  double* Up[kMaxModes];
  double* Uout[kMaxModes];
  void* A[kMaxModes];            // weighted bases (Ta)
  double* part;                  // p x ntile x LD x LD
  int ntile;                     // tiles per mode in `part`
};

// Arguments of the fused per-step update (k_update.cu).  Tc is the compute type;
// r x r matrices are column-major with leading dimension kMaxRank.
struct UpdArgs {
  ModeDesc d;
  const void* Y[kMaxModes];      // projections Y_n (Tc)
  const void* dS;                // core increment (Tc)
  const void* ds_y2;             // Y_2 (Tc): when set, phase 1 forms dS = Y_2 x_2 A_2^T
  void* dS_out;                  // ... into this buffer (the one dS points to)
  double* T;                     // core (in: step k, out: step k+1)
  double* T2;                    // scratch core
  void* Tcore;                   // Tc copy of the core (in and out; aliases T in FP64)
  double* U[kMaxModes];          // bases (in and out)
  double* Up[kMaxModes];         // U' (scratch)
  void* X[kMaxModes];            // M G^{-1} (Tc scratch, N_n x r_n)
  const double* w[kMaxModes];    // quadrature weights
  void* A[kMaxModes];            // W U (Tc; in: step k, out: step k+1)
  void* Uc[kMaxModes];           // U (Tc; in and out)
  double* G;                     // p x LD x LD (out)
  double* Ginv;                  // p x LD x LD (out)
  float* Ginvf;                  // float copy of Ginv (in: of the core of step k; out), null in FP64
  double* R;                     // p x LD x LD (out)
  double* Rinv;                  // p x LD x LD (out)
  double* sig2;                  // p x LD, descending (out)
  float* Vprev;                  // p x LD x LD, eigenvectors of G_n (Jacobi warm start; in and out)
  void* part;                    // 2 x p x ntile x LD x LD partial sums (Tc scratch)
  void* red;                     // 2 x kMaxModes x LD x LD sums of the partials of modes over 1024 points (Tc)
  double* gpart;                 // p x gsplit x LD x LD Gram partials (scratch)
  int ntile, gsplit;
  int warm, reorth;
  int skip_finish;               // phase 7 (G, G^{-1}, sigma^2) left to launch_gram_finish
  // Heun's second stage: the right-hand side is evaluated at the predicted state held in
  // T/U, and the new state is (y_k + y_pred + increment) / 2 with y_k = (T0, U0_n) in
  // the layout of T/U.  Null for an Euler step (and for Heun's first stage).
  const double* T0;
  const double* U0[kMaxModes];
  int combine;                   // with T0: 1 = Heun's mean (T0 + T + dT) / 2, 2 = T0 + dT (midpoint)
  unsigned* bar;                 // arrival counter of the grid barriers (zeroed per launch)
  unsigned long long* stamps;    // per-phase timer stamps (profiling), or null
  unsigned* flags;
};

struct GramView {
  int p, n;
  int64_t N[kMaxModes];
  const double* w[kMaxModes];
  int64_t L, Q, Nn;
};

// A timing event on stream s: an external event-record node while s is being captured
// (so that the replayed graph records it), an ordinary record otherwise.
inline cudaError_t record_timing_event(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
  return cudaEventRecord(ev, s);
}

// Process-wide count of libtdb kernel launches (tdb_kernel_launches).
void count_launch(int n = 1);
long long launches_so_far();

// k_basic.cu
template <typename T> void launch_diff(const T* a, const T* b, T* out, int64_t n, cudaStream_t s, T scale = T(1));
template <typename T> void launch_weighted_bases(const double* U, const double* w, T* A, int64_t N, int r, cudaStream_t s);
template <typename Ts, typename Td> void launch_cast(const Ts* a, Td* b, int64_t n, cudaStream_t s);
template <typename Tb> void launch_add(const double* a, const Tb* b, double* out, int64_t n, cudaStream_t s);
template <typename T>
void launch_wnorm2(const T* x, const T* y, const WeightView& wv, double* partial, int nblocks, double* out,
                   unsigned* flags, cudaStream_t s);
void launch_sum_partials(const double* partial, int n, double* out, cudaStream_t s);
template <typename T>
void launch_recon_err(const T* V, const T* U1, const T* H, int r1, int N1, int64_t ncol, const T* w1, const T* wcol,
                      double* partial, unsigned* counter, int nblocks, double* out, unsigned* flags, cudaStream_t s,
                      const int* gate = nullptr);
template <typename T>
void launch_weights_T(const WeightView& wv, T* w1, T* wcol, cudaStream_t s);
template <typename Tin, typename Tm, typename Tacc>
void launch_modeprod(const Tin* in, Tacc* out, const Tm* M, int64_t L, int K, int J, int64_t Q, int64_t sMj,
                     int64_t sMk, cudaStream_t s, const int* gate = nullptr);

// Column slices of the Gram partials G_n = T_(n) T_(n)^T: one per 32 columns of the
// widest unfolding, at most `cap`.  The fused update and the standalone refresh use
// the same split, so both sum in the same order.
inline int gram_split(const int* r, int p, int cap) {
  int64_t Rprod = 1, maxcol = 1;
  for (int n = 0; n < p; ++n) Rprod *= r[n];
  for (int n = 0; n < p; ++n) maxcol = std::max<int64_t>(maxcol, Rprod / r[n]);
  return (int)std::min<int64_t>(cap, std::max<int64_t>(1, maxcol / 32));
}

// k_update.cu (standalone Gram refresh)
// Phase 7 of the update alone (p CTAs): G_n, G_n^{-1}, sigma^(n) from the Gram partials.
void launch_gram_finish(const ModeDesc& d, const double* Gpart, int nsplit, double* G, double* Ginv, float* Ginvf,
                        double* sig2, float* Vprev, int warm, unsigned* flags, cudaStream_t s);
void launch_gram(const ModeDesc& d, const double* T, double* Gpart, int nsplit, double* G, double* Ginv,
                 float* Ginvf, double* sig2, float* Vprev, int warm, unsigned* flags, cudaStream_t s);

// k_small.cu
template <typename Tc>
void launch_orthonormalize(RowArgs& a, double* R, double* Rinv, unsigned* flags, cudaStream_t s);

// k_update.cu
template <typename Tc>
tdb_status launch_update(UpdArgs& a, int grid_hint, cudaStream_t s);

// k_eig.cu (float compute types)
void launch_sqrt_weights(const double* w, int n, float* ws, cudaStream_t s);
void launch_weight_data(const float* V, int p, const int64_t* N, const float* const* ws, int64_t S, float* Vw,
                        cudaStream_t s);
void launch_gram_weighted(const float* Vw, int64_t L, int64_t Nn, int64_t Q, double* part, size_t part_cap,
                          double* C64, float* Cc, cudaStream_t s);
size_t eig_si_scratch_floats(int n);
// Leading k eigenpairs of the float Gram Cc (n x n) by block subspace iteration from
// hash columns (the result depends on Cc only).
tdb_status eig_si_float(const float* Cc, const double* C64, int n, int k, int iters, float* scratch, unsigned* bar,
                        unsigned* flags, double* ev, double* Q, double* trace, cudaStream_t s);

// k_hosvd.cu
template <typename Tv>
void launch_wgram(const Tv* V, const GramView& g, double* part, size_t part_cap, double* C64, void* Cc, int cc_float,
                  cudaStream_t s);
template <typename T>
tdb_status eig_leading_small(const T* Cc, const double* C64, int n, int k, T* A_ws, T* V_ws, unsigned* flags,
                             double* ev, double* Q, double* trace, double* scratch, cudaStream_t s);
template <typename T>
struct SubspaceWs {
  T* Q;        // n x 64
  T* Z;        // n x 64
  T* X;        // n x 64
  double* G;   // 64 x 64
  double* R;   // 64 x 64
  T* H;        // 64 x 64
  T* JA;       // 64 x 64
  T* JV;       // 64 x 64
};
template <typename T>
// Q0 (nullable, n x k doubles, may be Q itself): warm start from a previous solve instead
// of hash columns.
tdb_status eig_subspace(const T* Cc, const double* C64, int n, int k, int iters, const SubspaceWs<T>& ws,
                        unsigned* flags, double* ev, double* Q, double* trace, double* scratch, cudaStream_t s,
                        const double* Q0 = nullptr);
void launch_scale_basis(const double* Q, const double* w, int64_t n, int r, double* U, cudaStream_t s);
void launch_merge_weights(const WeightView& wv, int skip, int64_t M, double* wq, cudaStream_t s);
template <typename Tv>
void launch_short_map(const Tv* V, int first, int64_t Nn, int64_t M, const double* wn, const double* sqw,
                      const double* Z, const double* ev, int k, double* Q, cudaStream_t s);

}  // namespace tdb
