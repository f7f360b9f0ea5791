// Fused forward kernel, tensor-memory form (tf32, bf16 or fp16 MMA
// operands), instantiated for dim = 2, up to 8 robots.
#include "sf_tm_kernel.cuh"

namespace sf {
cudaError_t launch_tm_d2_n8(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  if (l.prec == PREC_TM_TF32) return fused_impl::launch_tm_t<2, 8, 384, 0>(a, l, st);
  if (l.prec == PREC_TM_BF16) return fused_impl::launch_tm_t<2, 8, 384, 1>(a, l, st);
  if (l.prec == PREC_TM_FP16) return fused_impl::launch_tm_t<2, 8, 384, 2>(a, l, st);
  return cudaErrorInvalidValue;
}
// prec: the handle's sf_precision (0 float32 -> tf32 operands)
cudaError_t prepare_tm_d2_n8(int smem, int prec) {
  const int dyn = smem - (int)TM_STATIC_SMEM_RESERVE;
  if (prec == 1)
    return cudaFuncSetAttribute(fused_impl::tm_fwd_kernel<2, 8, 384, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (prec == 2)
    return cudaFuncSetAttribute(fused_impl::tm_fwd_kernel<2, 8, 384, 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  return cudaFuncSetAttribute(fused_impl::tm_fwd_kernel<2, 8, 384, 0>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
}
}  // namespace sf
