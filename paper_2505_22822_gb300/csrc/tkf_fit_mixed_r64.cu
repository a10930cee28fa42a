// tkf_fit_mixed_r64.cu -- the mixed-precision persistent fit kernels capped at 64 registers a
// thread (a translation unit of their own, so that the variants compile in parallel).
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_mixed_r64(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                   uint32_t* counter, LaunchShape shape, cudaStream_t stream) {
  return launch_fields<1, 64>(a, f, mode, perm, counter, shape, stream);
}

}  // namespace tkf
