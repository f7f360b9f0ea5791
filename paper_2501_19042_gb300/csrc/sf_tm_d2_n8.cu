// Fused forward kernel, tensor-memory form (tf32, bf16 or fp16 MMA
// operands), instantiated for dim = 2, up to 8 robots.
#include "sf_tm_kernel.cuh"

namespace sf {
// a.ckpt set: the training forward (checkpoints, activity masks)
cudaError_t launch_tm_d2_n8(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  const bool train = a.ckpt != nullptr;
  if (l.prec == PREC_TM_TF32)
    return train ? fused_impl::launch_tm_t<2, 8, 384, 0, true>(a, l, st)
                 : fused_impl::launch_tm_t<2, 8, 384, 0>(a, l, st);
  if (l.prec == PREC_TM_BF16)
    return train ? fused_impl::launch_tm_t<2, 8, 384, 1, true>(a, l, st)
                 : fused_impl::launch_tm_t<2, 8, 384, 1>(a, l, st);
  if (l.prec == PREC_TM_FP16)
    return train ? fused_impl::launch_tm_t<2, 8, 384, 2, true>(a, l, st)
                 : fused_impl::launch_tm_t<2, 8, 384, 2>(a, l, st);
  return cudaErrorInvalidValue;
}
// prec: the handle's sf_precision (0 float32 -> tf32 operands)
cudaError_t prepare_tm_d2_n8(int smem, int prec) {
  const int dyn = smem - (int)TM_STATIC_SMEM_RESERVE;
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if (prec == 1) {
    e = cudaFuncSetAttribute(fused_impl::tm_fwd_kernel<2, 8, 384, 1>, at, dyn);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_impl::tm_fwd_kernel<2, 8, 384, 1, true>, at, dyn);
  } else if (prec == 2) {
    e = cudaFuncSetAttribute(fused_impl::tm_fwd_kernel<2, 8, 384, 2>, at, dyn);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_impl::tm_fwd_kernel<2, 8, 384, 2, true>, at, dyn);
  } else {
    e = cudaFuncSetAttribute(fused_impl::tm_fwd_kernel<2, 8, 384, 0>, at, dyn);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fused_impl::tm_fwd_kernel<2, 8, 384, 0, true>, at, dyn);
  }
  return e;
}
}  // namespace sf
