// Host-side structures of the surrogate (device buffers and launch wrappers).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define MLP_TRAIN_BLOCKS 64
#define MLP_KSLICES 16
#define MLP_MAX_N 8

struct MlpDev {
  float *p = nullptr, *m = nullptr, *v = nullptr;          // parameters and Adam moments
  __nv_bfloat16 *w2 = nullptr, *w3 = nullptr, *w2t = nullptr, *w3t = nullptr;
};

struct MlpWork {
  __nv_bfloat16 *A1, *A2, *dZ3, *dZ2;
  float *Z1, *Z2, *Z3, *A3, *dY, *loss, *dZ1, *part2, *part3, *grad;
};

// Sampling box of the training data and the per-n envelope constants.
struct MlpDataSpec {
  double log_s_lo, log_s_hi, log_tau_lo, log_tau_hi, log_m_lo, log_m_hi;
  int n_count;
  int n_values[MLP_MAX_N];
  double alpha[MLP_MAX_N];
  double envA[MLP_MAX_N][4], envB[MLP_MAX_N][4];   // envelope (p, q, r, m) of FA and FB per n
  // 1: the screened law; tau is then q = varsigma^2 / v_c^2, the targets its quadrature (n = 0
  // normalisation) and the envelopes carry the factor 1 / (1 + q (2x + 3))^2
  int scr = 0;
};

cudaError_t mlp_refresh(MlpDev &d, cudaStream_t s);
cudaError_t mlp_infer(const MlpDev &d, const float *X, int64_t N, float *Y, cudaStream_t s);
cudaError_t mlp_make_data(const MlpDataSpec &spec, int64_t N, unsigned long long seed, float *X, float *Y,
                          cudaStream_t s);
cudaError_t mlp_train_batch(MlpDev &d, const float *X, const float *Y, const int *idx, int B, MlpWork &w, float lr,
                            int t_adam, cudaStream_t s, int64_t *launches);
cudaError_t mlp_grad(MlpDev &d, const float *X, const float *Y, const int *idx, int B, MlpWork &w, cudaStream_t s);
