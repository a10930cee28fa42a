// tkf_fit_two_filter_capped_fp64.cu -- the two-filter smoother's persistent fit kernels in FP64
// capped at 128 or 64 registers a thread (a translation unit of their own, so that the variants
// compile in parallel): candidates of the launch-shape tuner.
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_two_filter_fp64_capped(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                              uint32_t* counter, LaunchShape shape, cudaStream_t stream) {
  if (shape.regs == 128) return launch_fields<0, 128, 1, 1>(a, f, mode, perm, counter, shape, stream);
  if (shape.regs == 64) return launch_fields<0, 64, 1, 1>(a, f, mode, perm, counter, shape, stream);
  return cudaErrorInvalidValue;
}

}  // namespace tkf
