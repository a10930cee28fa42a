// tkf_fit_two_filter.cu -- the persistent fit kernels with the two-filter smoother (forward
// filter, backward filter of the reversed particle, weighted mean with the seed), one lane a
// track at the full register file; the FP64 instantiation and the dispatch over precisions.
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_two_filter(const FitArgs& a, const FieldDev& f, int precision, int mode, const uint32_t* perm,
                                  uint32_t* counter, LaunchShape shape, cudaStream_t stream) {
  if (shape.group != 1) return cudaErrorInvalidValue;
  shape.regs = 255;
  if (precision == TKF_MIXED) return launch_fit_two_filter_mixed(a, f, mode, perm, counter, shape, stream);
  if (precision == TKF_MIXED_FP32) return launch_fit_two_filter_mixed32(a, f, mode, perm, counter, shape, stream);
  if (precision != TKF_FP64) return cudaErrorInvalidValue;
  return launch_fields<0, 255, 1, 1>(a, f, mode, perm, counter, shape, stream);
}

}  // namespace tkf
