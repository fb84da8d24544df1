// tc_project.h - fused snapshot difference + multi-mode projection on the tensor
// cores (bf16 operands, fp32 accumulation): the projection of Eqs. 2.15/2.16.
#pragma once
#include <string>

#include "kernels.h"

namespace tdb {

struct TcPlan {
  int p = 0;
  float* z1p = nullptr;               // [tiles along i1][slices][N2][r1] partial dV x_1 A_1^T
  float* z2p = nullptr;               // [tiles along i2][slices][N1][r2] partial dV x_2 A_2^T
  double* wsl = nullptr;              // product of the weights of modes >= 3, per slice
  float* w12f = nullptr;              // float w_1, w_2, zero-padded to whole tiles
  double* npart = nullptr;            // ||dV||_W^2 per converter warp of every CTA
  float* pad[2] = {nullptr, nullptr}; // zero-padded copies of V_{k+1}, V_k (N_1 not a multiple of 4)
  float* fpart = nullptr;             // split partials of the finishing contraction
  size_t fpart_cap = 0;               // floats

  // launch shape chosen by the tuner (CTAs per tile position, finish split target), with
  // the candidates it timed (microseconds per launch)
  static constexpr int kMaxCand = 4;
  bool tuned = false;
  bool from_cache = false;
  int cstep = 0, fin_target = 0;
  int ncand = 0;
  int cand[kMaxCand] = {0};
  float cand_us[kMaxCand] = {0.f};
  int fin_cand[3] = {0};
  float fin_us[3] = {0.f};
  bool wsl_ready = false;
  bool attr_set = false;
  // profiling: device words {first CTA start, last CTA end, summed spans (ns), launches} of
  // the main kernel, accumulated by the finishing launch; null when not profiling
  unsigned long long* span = nullptr;
};

bool tc_supported(int p, const int64_t* N, const int* cap, std::string& err);
// One CTA waits on an mbarrier nothing arrives at, with the projection kernel's bounded
// wait and the given limit (clock cycles); the timeout bit lands in *flags.
tdb_status tc_selftest_mbar_wait(unsigned* flags, long long limit, cudaStream_t s);
void tc_carve(TcPlan& plan, Carver& cv, int p, const int64_t* N, const int* cap);
// Y_n of dV = dscale (Vn - Vp) (Eqs. 2.15, 2.16), dS unless defer_ds (the update kernel then forms
// dS = Y_2 x_2 A_2^T), and ||dV||_W^2 into *dv2.  A: FP32 weighted bases (N_n x r_n);
// w: mode weights; Z1 (r1 x N2 x S) and scratch (>= r1 r2 prod_{n>2} N_n) are device
// buffers of the caller; Z2 is not used.  pdl: the projection kernel is launched
// programmatically after the stream's previous kernel (which must trigger its dependents
// and leave the projection's inputs unchanged); it waits for that kernel before writing
// the status flags and before it completes.  With pdl the kernel's start event evm[0] is
// the caller's (recorded before that previous kernel).
tdb_status tc_project(TcPlan& plan, const float* Vn, const float* Vp, int p, const int64_t* N, const int* r,
                      const void* const* A, const double* const* w, float* Z1, float* Z2, float* scratch,
                      float* dS, float* const* Y, double* dv2, unsigned* flags, cudaStream_t s, cudaEvent_t* evm,
                      std::string& err, bool defer_ds = false, float dscale = 1.0f, bool pdl = false);

}  // namespace tdb
