// Fused forward kernel instantiated for dim = 3, up to 32 robots.
#include "sf_fused_kernel.cuh"

namespace sf {
cudaError_t launch_fused_d3_n32(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  return fused_impl::launch_t<3, 32, 384>(a, l, st);
}
cudaError_t prepare_fused_d3_n32(int smem) {
  return cudaFuncSetAttribute(fused_impl::fused_fwd_kernel<3, 32, 384>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
}  // namespace sf
