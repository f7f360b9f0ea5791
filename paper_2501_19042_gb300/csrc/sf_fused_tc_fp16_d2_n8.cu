// Fused forward kernel, tensor-core form with fp16 operands, instantiated for
// dim = 2, up to 8 robots.
#include "sf_fused_kernel.cuh"

namespace sf {
cudaError_t launch_fused_tc2_d2_n8(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  return fused_impl::launch_t<2, 8, 384, 2>(a, l, st);
}
cudaError_t prepare_fused_tc2_d2_n8(int smem) {
  return cudaFuncSetAttribute(fused_impl::fused_fwd_kernel<2, 8, 384, 2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
}  // namespace sf
