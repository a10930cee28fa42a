// tkf_fit_two_filter_mixed.cu -- the two-filter smoother's persistent fit kernels in mixed
// precision (FP32 propagation and transport; update, backward filter and weighted mean in FP64).
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_two_filter_mixed(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm,
                                        uint32_t* counter, LaunchShape shape, cudaStream_t stream) {
  return launch_fields<1, 255, 1, 1>(a, f, mode, perm, counter, shape, stream);
}

}  // namespace tkf
