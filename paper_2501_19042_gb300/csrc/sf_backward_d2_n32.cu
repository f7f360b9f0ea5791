// Adjoint kernel and the mask-writing training forward, instantiated for
// dim = 2, up to 32 robots.
#include "sf_backward_kernel.cuh"

namespace sf {
cudaError_t launch_bwd_d2_n32(const FusedArgs& a, const BwdLaunchArgs& b, const FusedLaunch& l,
                             cudaStream_t st) {
  return fused_impl::launch_bwd_from<2, 32, 256>(a, b, l, st);
}
cudaError_t prepare_bwd_d2_n32(int smem) {
  return cudaFuncSetAttribute(fused_impl::fused_bwd_kernel<2, 32, 256>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
// Forward with checkpoints (training): also writes the activity masks of
// the last checkpoint segment for this adjoint.
cudaError_t launch_fused_train_d2_n32(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  return fused_impl::launch_t<2, 32, 384, true>(a, l, st);
}
cudaError_t prepare_fused_train_d2_n32(int smem) {
  return cudaFuncSetAttribute(fused_impl::fused_fwd_kernel<2, 32, 384, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
}  // namespace sf
