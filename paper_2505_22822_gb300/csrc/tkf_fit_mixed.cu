// tkf_fit_mixed.cu -- instantiation of the persistent fit kernels, mixed precision.
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_mixed(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm, uint32_t* counter,
                            LaunchShape shape, cudaStream_t stream) {
  return launch_fields<true>(a, f, mode, perm, counter, shape, stream);
}

cudaError_t launch_propose_start(const FitArgs& a, const FieldDev& f, float* h0, cudaStream_t stream) {
  return propose_fields<float>(a, f, h0, stream);
}

}  // namespace tkf
