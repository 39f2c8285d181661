// Tensor-core plan: not yet built; the TF32 modes report "not supported".
#include "tc.h"

namespace afqmc {

struct TcPlan {};

cudaError_t tc_plan_create(TcPlan** out, const TcShape&, cudaStream_t, const float*,
                           const float*, const float*, const float*, const float*) {
  *out = nullptr;
  return cudaErrorNotSupported;
}
void tc_plan_destroy(TcPlan* p) { delete p; }
cudaError_t tc_force_bias(TcPlan*, cudaStream_t, const float*, float*) {
  return cudaErrorNotSupported;
}
cudaError_t tc_one_body(TcPlan*, cudaStream_t, const float*, float*) {
  return cudaErrorNotSupported;
}
cudaError_t tc_propagate(TcPlan*, cudaStream_t, const float*, float*, float*, float*) {
  return cudaErrorNotSupported;
}
cudaError_t tc_exchange(TcPlan*, cudaStream_t, int, const float*, float*) {
  return cudaErrorNotSupported;
}

}  // namespace afqmc
