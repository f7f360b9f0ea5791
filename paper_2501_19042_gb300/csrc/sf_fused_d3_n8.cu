// Fused forward kernel instantiated for dim = 3, up to 8 robots.
#include "sf_fused_kernel.cuh"

namespace sf {
cudaError_t launch_fused_d3_n8(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  return fused_impl::launch_t<3, 8, 384>(a, l, st);
}
cudaError_t prepare_fused_d3_n8(int smem) {
  return cudaFuncSetAttribute(fused_impl::fused_fwd_kernel<3, 8, 384>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
}  // namespace sf
