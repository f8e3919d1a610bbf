// mlp_tc.cu -- (a1) on the tcgen05 tensor cores (not yet built)
#include "rtn_internal.cuh"
namespace rtn {
cudaError_t mlp_tc_prepare(rtn_ctx*, std::string& err) {
  err = "tensor-core path not built";
  return cudaSuccess;
}
cudaError_t mlp_tc_forward(rtn_ctx*, const float*, const float*, float*, float*) {
  return cudaErrorNotSupported;
}
void mlp_tc_release(rtn_ctx*) {}
}  // namespace rtn
