// tkf_fit_two_filter_mixed32.cu -- the two-filter smoother's persistent fit kernels with the
// covariance algebra in FP32 as well (TKF_MIXED_FP32): forward and backward filters and the
// weighted mean.
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_two_filter_mixed32(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                          uint32_t* counter, LaunchShape shape, cudaStream_t stream) {
  return launch_fields<2, 255, 1, 1>(a, f, mode, perm, counter, shape, stream);
}

}  // namespace tkf
