// Tensor-core (tcgen05) crop network: placeholder until the kernels land.
#include "handle.cuh"

namespace locc {

int upload_tc_params(locc_handle* h, const std::vector<float>& params) {
  (void)h;
  (void)params;
  return LOCC_OK;
}

int run_network_tc(locc_handle* h, const float4* xyz, int n_pairs, const int* n_dev,
                   const PairInputs* in, const float4* centre, float* out, float* y_raw,
                   float* feat_out, cudaStream_t stream, cudaEvent_t mid) {
  (void)mid;
  (void)h, (void)xyz, (void)n_pairs, (void)n_dev, (void)in, (void)centre, (void)out, (void)y_raw;
  (void)feat_out, (void)stream;
  set_error("tensor-core precision not available in this build");
  return LOCC_ERR_INVALID_ARG;
}

}  // namespace locc
