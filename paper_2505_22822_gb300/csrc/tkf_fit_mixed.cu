// tkf_fit_mixed.cu -- instantiation of the persistent fit kernels, mixed precision, full
// register file; the dispatch over register caps; the learned mode's proposal pre-pass.
#include "tkf_fit_impl.cuh"

namespace tkf {

cudaError_t launch_fit_mixed(const FitArgs& a, const FieldDev& f, int mode, const uint32_t* perm, uint32_t* counter,
                             LaunchShape shape, cudaStream_t stream) {
  if (shape.regs == 128) return launch_fit_mixed_r128(a, f, mode, perm, counter, shape, stream);
  if (shape.regs == 64) return launch_fit_mixed_r64(a, f, mode, perm, counter, shape, stream);
  return launch_fields<1, 255>(a, f, mode, perm, counter, shape, stream);
}

cudaError_t launch_propose_start(const FitArgs& a, const FieldDev& f, float* h0, cudaStream_t stream) {
  return propose_fields(a, f, h0, stream);
}

}  // namespace tkf
