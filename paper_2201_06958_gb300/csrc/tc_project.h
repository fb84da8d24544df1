// tc_project.h - fused snapshot difference + multi-mode projection on the tensor
// cores (bf16 operands, fp32 accumulation): the projection of Eqs. 2.15/2.16.
#pragma once
#include <string>

#include "kernels.h"

namespace tdb {

struct TcPlan {
  int p = 0;
  void* Abf[kMaxModes] = {nullptr};   // bf16 weighted bases, swizzled operand images
  float* zpart = nullptr;             // partial first-level contractions
  size_t zpart_elems = 0;
};

bool tc_supported(int p, const int64_t* N, const int* cap, std::string& err);
void tc_carve(TcPlan& plan, Carver& cv, int p, const int64_t* N, const int* cap);
tdb_status tc_project(TcPlan& plan, const float* Vn, const float* Vp, int p, const int64_t* N, const int* r,
                      const void* const* A, float* dS, float* const* Y, double* npart, int nblk,
                      const WeightView& wv, double* dv2, unsigned* flags, cudaStream_t s, std::string& err);

}  // namespace tdb
