// Adjoint kernel and the mask-writing training forward, instantiated for
// dim = 2, up to 16 robots.
#include <cstring>

#include "sf_backward_kernel.cuh"

namespace sf {
cudaError_t launch_bwd_d2_n16(const FusedArgs& a, const BwdLaunchArgs& b, const FusedLaunch& l,
                                  cudaStream_t st) {
  fused_impl::BwdArgs x;
  std::memset(&x, 0, sizeof(x));
  x.pc = a.pc;
  x.n_scenes = a.n_scenes;
  x.basis = a.basis;
  x.ops = a.ops;
  x.start = a.start;
  x.goal = a.goal;
  x.start_va = a.start_va;
  x.goal_va = a.goal_va;
  x.xi_bar = a.xi_bar;
  x.ckpt = b.ckpt;
  x.ck_every = b.ck_every;
  x.total_coefs = b.total_coefs;
  x.ring = b.ring;
  x.tail_mask = b.tail_mask;
  x.ring_mask = b.ring_mask;
  x.mask_slot = b.mask_slot;
  x.g_xi = b.g_xi;
  x.g_lam = b.g_lam;
  x.g_fp = b.g_fp;
  x.gx0 = b.gx0;
  x.gl0 = b.gl0;
  x.gxb = b.gxb;
  x.xi0_is_xi_bar = b.xi0_is_xi_bar;
  x.tc = l.tc;
  x.nq = l.nq;
  x.total_samples = a.total_samples;
  x.status = a.status;
  std::memcpy(x.sc, a.sc, sizeof(x.sc));
  return fused_impl::launch_bwd_t<2, 16, 384>(x, l.n_ctas, l.warps, l.smem, st);
}
cudaError_t prepare_bwd_d2_n16(int smem) {
  return cudaFuncSetAttribute(fused_impl::fused_bwd_kernel<2, 16, 384>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
// Forward with checkpoints (training): also writes the activity masks of
// the last checkpoint segment for this adjoint.
cudaError_t launch_fused_train_d2_n16(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  return fused_impl::launch_t<2, 16, 384, 0, true>(a, l, st);
}
cudaError_t prepare_fused_train_d2_n16(int smem) {
  return cudaFuncSetAttribute(fused_impl::fused_fwd_kernel<2, 16, 384, 0, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
}  // namespace sf
