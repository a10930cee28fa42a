// tkf_fit_mixed32.cu -- the experimental precision TKF_MIXED_FP32: the mixed path with the
// covariance algebra (Joseph update, smoother, covariance transport results) in FP32 as well,
// at the full register file and capped at 128 registers.
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_mixed32(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm, uint32_t* counter,
                               LaunchShape shape, cudaStream_t stream) {
  if (shape.regs == 128) return launch_fields<2, 128>(a, f, mode, perm, counter, shape, stream);
  if (shape.regs != 255) return cudaErrorInvalidValue;
  return launch_fields<2, 255>(a, f, mode, perm, counter, shape, stream);
}

}  // namespace tkf
