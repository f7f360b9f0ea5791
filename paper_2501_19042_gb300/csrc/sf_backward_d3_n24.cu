// Adjoint kernel and the mask-writing training forward, instantiated for
// dim = 3, up to 24 robots.
#include "sf_backward_kernel.cuh"

namespace sf {
cudaError_t launch_bwd_d3_n24(const FusedArgs& a, const BwdLaunchArgs& b, const FusedLaunch& l,
                             cudaStream_t st) {
  return fused_impl::launch_bwd_from<3, 24, 256>(a, b, l, st);
}
cudaError_t prepare_bwd_d3_n24(int smem) {
  return cudaFuncSetAttribute(fused_impl::fused_bwd_kernel<3, 24, 256>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
// Forward with checkpoints (training): also writes the activity masks of
// the last checkpoint segment for this adjoint.
cudaError_t launch_fused_train_d3_n24(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  return fused_impl::launch_t<3, 24, 384, true>(a, l, st);
}
cudaError_t prepare_fused_train_d3_n24(int smem) {
  return cudaFuncSetAttribute(fused_impl::fused_fwd_kernel<3, 24, 384, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
}  // namespace sf
