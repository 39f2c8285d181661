// Tensor-core (tcgen05) plan for the dense contractions of the TF32 modes.
#pragma once

#include <cuda_runtime.h>

namespace afqmc {

struct TcShape {
  int W, M, n_up, n_dn, n_chol, taylor_order;
  bool split;   // TF32x3: hi + lo operands
};

struct TcPlan;

cudaError_t tc_plan_create(TcPlan** out, const TcShape& s, cudaStream_t st,
                           const float* L, const float* Ltil, const float* Bhalf,
                           const float* Yx_up, const float* Yx_dn);
void tc_plan_destroy(TcPlan* p);
cudaError_t tc_force_bias(TcPlan* p, cudaStream_t st, const float* Theta, float* X);
cudaError_t tc_one_body(TcPlan* p, cudaStream_t st, const float* S, float* V);
cudaError_t tc_propagate(TcPlan* p, cudaStream_t st, const float* V, float* Phi,
                         float* tmp1, float* tmp2);
cudaError_t tc_exchange(TcPlan* p, cudaStream_t st, int spin, const float* Theta,
                        float* Z);

}  // namespace afqmc
