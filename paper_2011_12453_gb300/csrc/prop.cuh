// Learned exchange proposal network: parameter layout and launchers (prop.cu).
#pragma once

#include "common.cuh"

namespace gna {

// 9 features -> 64 -> 64 -> 1 logit, tanh hidden units.  Flat parameters (float32):
// [W1 (9 x 64), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1)], row-major.
constexpr int kPropIn = 9;
constexpr int kPropHid = 64;
constexpr int kPropOW1 = 0;
constexpr int kPropOb1 = kPropOW1 + kPropIn * kPropHid;
constexpr int kPropOW2 = kPropOb1 + kPropHid;
constexpr int kPropOb2 = kPropOW2 + kPropHid * kPropHid;
constexpr int kPropOw3 = kPropOb2 + kPropHid;
constexpr int kPropOb3 = kPropOw3 + kPropHid;
constexpr int kPropParams = kPropOb3 + 1;

size_t prop_workspace(const gna_graph* g, int64_t B);
gna_status prop_grad_launch(const gna_graph* g, const int8_t* spins, const float* dlogpsi, int64_t B,
                            const float* params, double* grad, double* loss, void* ws, cudaStream_t st);
gna_status prop_logits_launch(const gna_graph* g, const int8_t* spins, int64_t B, const float* params, float* logits,
                              cudaStream_t st);
gna_status prop_adam_launch(float* params, float* m, float* v, const double* grad, int t, double lr,
                            cudaStream_t st);

}  // namespace gna
