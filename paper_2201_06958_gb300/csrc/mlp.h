// mlp.h - sizes of the learned error estimator and its launchers.
#pragma once
#include <cuda_runtime.h>

namespace tdb {

constexpr int MLP_F = 8;                                                  // features
constexpr int MLP_H = 64;                                                 // hidden width
constexpr int MLP_NPARAM = MLP_H * MLP_F + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;

void mlp_loss_grad(const float* P, const float* X, const float* t, int n, float* gpart, float* lpart, int max_parts,
                   float* grad, float* loss, cudaStream_t s);
void mlp_adam(float* P, const float* g, float* m, float* v, int step, float lr, cudaStream_t s);
void mlp_forward(const float* P, const float* X, int n, float* y, cudaStream_t s);

// Host-maintained counters the feature kernel needs (uploaded every step).
struct EstState {
  double last_log_eps;       // log10 of the previous step's error (exact, or the estimate when skipped)
  double prev_res_log;       // log10 of the previous step's residual ||dV||_W^2 - ||dS||^2 (square root)
  int steps_since_exact;     // steps since the last exact evaluation, this one included
  int steps_since_reinit;
  int ready;                 // estimator fitted
  int max_skip;              // force an exact evaluation after this many estimated steps
  double gate;               // exact when estimate > gate * eps_th
  double eps_th;
  double novelty_z;          // exact when a standardised feature leaves [-z, z]
};

// Features of the current step, the estimate and the gate (one CTA).
// st_dev: device copy of the estimator state for this step.
void est_features(const EstState* st_dev, const float* dS, int nds, const double* dv2, const double* sig2,
                  const int* ranks, int p, const float* P, const float* norm, float* feat, double* est, int* need,
                  double* ds2, cudaStream_t s);
void est_normalize(float* X, float* t, int n, float* norm, cudaStream_t s);
void est_init_params(float* P, unsigned long long seed, cudaStream_t s);

}  // namespace tdb
