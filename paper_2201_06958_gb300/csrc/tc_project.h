// tc_project.h - fused snapshot difference + multi-mode projection on the tensor
// cores (bf16 operands, fp32 accumulation): the projection of Eqs. 2.15/2.16.
#pragma once
#include <string>

#include "kernels.h"

namespace tdb {

struct TcPlan {
  int p = 0;
  void* Abf[2] = {nullptr, nullptr};  // BF16 operand images of A_1, A_2 (128-byte swizzled, K-major)
  float* z1p = nullptr;               // [tiles along i1][slices][N2][r1] partial dV x_1 A_1^T
  float* z2p = nullptr;               // [tiles along i2][slices][N1][r2] partial dV x_2 A_2^T
  double* wsl = nullptr;              // product of the weights of modes >= 3, per slice
  float* w12f = nullptr;              // float w_1, w_2, zero-padded to whole tiles
  double* npart = nullptr;            // per-CTA ||dV||_W^2
  bool wsl_ready = false;
  bool attr_set = false;
};

bool tc_supported(int p, const int64_t* N, const int* cap, std::string& err);
// Three modes with few slices (N_3 <= 64, r_3 <= 32): tc_project finishes with the two
// fused launches (each CTA walks all slices, so many slices would serialise them) and
// leaves dS = Y_3 x_3 A_3^T to the update kernel.
inline bool tc_defers_ds(int p, const int64_t* N, const int* r) { return p == 3 && N[2] <= 64 && r[2] <= 32; }
void tc_carve(TcPlan& plan, Carver& cv, int p, const int64_t* N, const int* cap);
// dS (unless tc_defers_ds) and Y_n of dV = Vn - Vp (Eqs. 2.15, 2.16) and ||dV||_W^2 into *dv2.  A: FP32
// weighted bases (N_n x r_n); w: mode weights; Z1 (r1 x N2 x S), Z2 (N1 x r2 x S)
// and scratch (>= the largest intermediate) are device buffers of the caller.
tdb_status tc_project(TcPlan& plan, const float* Vn, const float* Vp, int p, const int64_t* N, const int* r,
                      const void* const* A, const double* const* w, float* Z1, float* Z2, float* scratch,
                      float* dS, float* const* Y, double* dv2, unsigned* flags, cudaStream_t s, cudaEvent_t* evm,
                      std::string& err, bool defer_ds = false);

}  // namespace tdb
