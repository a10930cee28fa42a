// tkf_fit_fp64_r128.cu -- the FP64 persistent fit kernels capped at 128 registers a thread, with
// the smoother state in shared memory (a translation unit of their own, so that the variants
// compile in parallel).
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_fp64_r128(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                 uint32_t* counter, LaunchShape shape, cudaStream_t stream) {
  return launch_fields<0, 128>(a, f, mode, perm, counter, shape, stream);
}

}  // namespace tkf
