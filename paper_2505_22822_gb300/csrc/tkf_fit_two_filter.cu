// tkf_fit_two_filter.cu -- the persistent fit kernels with the two-filter smoother (forward
// filter, backward filter of the reversed particle, weighted mean with the seed), one lane a
// track; the FP64 instantiation at the full register file and the dispatch over precisions and
// register caps (128 / 64: tkf_fit_two_filter_capped_*.cu).
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_two_filter(const FitArgs& a, const FieldDev& f, int precision, int mode, const uint32_t* perm,
                                  uint32_t* counter, LaunchShape shape, cudaStream_t stream) {
  if (shape.group != 1) return cudaErrorInvalidValue;
  if (shape.regs == 128 || shape.regs == 64) {
    if (precision == TKF_MIXED) return launch_fit_two_filter_mixed_capped(a, f, mode, perm, counter, shape, stream);
    if (precision == TKF_FP64) return launch_fit_two_filter_fp64_capped(a, f, mode, perm, counter, shape, stream);
    return cudaErrorInvalidValue;
  }
  shape.regs = 255;
  if (precision == TKF_MIXED) return launch_fit_two_filter_mixed(a, f, mode, perm, counter, shape, stream);
  if (precision == TKF_MIXED_FP32) return launch_fit_two_filter_mixed32(a, f, mode, perm, counter, shape, stream);
  if (precision != TKF_FP64) return cudaErrorInvalidValue;
  return launch_fields<0, 255, 1, 1>(a, f, mode, perm, counter, shape, stream);
}

}  // namespace tkf
