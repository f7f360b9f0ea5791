// Dispatch of the fused forward kernel over (dim, robot-count bucket); the
// kernel template lives in sf_fused_kernel.cuh and each instantiation is
// compiled in its own translation unit (sf_fused_d*_n*.cu).
#include "sf_internal.cuh"

namespace sf {

#define SF_DECL(D, NM) cudaError_t launch_fused_d##D##_n##NM(const FusedArgs&, const FusedLaunch&, cudaStream_t);
SF_DECL(2, 8) SF_DECL(2, 16) SF_DECL(2, 32) SF_DECL(3, 8) SF_DECL(3, 16) SF_DECL(3, 32)
#undef SF_DECL

int fused_max_warps() { return 14; }

size_t fused_smem_bytes(int dim, int nmax, int T, int gmax) {
  const int RS = dim * NP;
  const int TB = (T + 31) / 32;
  const int SB = (4 + TB) * nmax * RS + 2 * dim * NP + ((TB + 3) / 4) * 4;
  const int head = 4 * NV * NP + nmax * RS;
  return sizeof(float) * ((size_t)head + (size_t)gmax * SB);
}

cudaError_t launch_fused(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  const int dim = a.pc.dim;
  if (dim == 3) {
    if (l.nmax == 8) return launch_fused_d3_n8(a, l, st);
    if (l.nmax == 16) return launch_fused_d3_n16(a, l, st);
    if (l.nmax == 32) return launch_fused_d3_n32(a, l, st);
  } else if (dim == 2) {
    if (l.nmax == 8) return launch_fused_d2_n8(a, l, st);
    if (l.nmax == 16) return launch_fused_d2_n16(a, l, st);
    if (l.nmax == 32) return launch_fused_d2_n32(a, l, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sf
