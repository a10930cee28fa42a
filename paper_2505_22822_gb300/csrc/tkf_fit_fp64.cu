// tkf_fit_fp64.cu -- instantiation of the persistent fit kernels, FP64.
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_fp64(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm, uint32_t* counter,
                            LaunchShape shape, cudaStream_t stream) {
  return launch_fields<0, 255>(a, f, mode, perm, counter, shape, stream);
}

}  // namespace tkf
