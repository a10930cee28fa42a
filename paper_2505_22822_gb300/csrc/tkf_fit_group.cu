// tkf_fit_group.cu -- the group-per-track persistent fit kernels (4 lanes a track, full
// register file), FP64 and mixed precision, in a translation unit of their own so that they
// compile in parallel with the one-lane-per-track variants.
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_group(const FitArgs& a, const FieldDev& f, int precision, int mode, const uint32_t* perm,
                             uint32_t* counter, LaunchShape shape, cudaStream_t stream) {
  if (shape.regs != 255) return cudaErrorInvalidValue;
  if (precision == TKF_MIXED) return launch_fields<1, 255, 4>(a, f, mode, perm, counter, shape, stream);
  if (precision == TKF_FP64) return launch_fields<0, 255, 4>(a, f, mode, perm, counter, shape, stream);
  return cudaErrorInvalidValue;
}

}  // namespace tkf
