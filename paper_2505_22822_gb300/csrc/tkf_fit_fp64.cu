// tkf_fit_fp64.cu -- instantiation of the persistent fit kernels, FP64, full register file; the
// dispatch over register caps.
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_fp64(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm, uint32_t* counter,
                            LaunchShape shape, cudaStream_t stream) {
  if (shape.regs == 128) return launch_fit_fp64_r128(a, f, mode, perm, counter, shape, stream);
  if (shape.regs == 64) return launch_fit_fp64_r64(a, f, mode, perm, counter, shape, stream);
  return launch_fields<0, 255>(a, f, mode, perm, counter, shape, stream);
}

}  // namespace tkf
