// Debug-build checks of the fused kernels (compiled in with
// -DSF_DEBUG_CHECKS=1; the release library has none of them).
//
// No check traps or asserts. A failed index check records its site in a
// per-CTA word and the access it guards is skipped; shared-memory canary
// words (after the head of the CTA's shared memory and at the end of every
// sample block) are written once the prologue has filled the head and are
// checked after every phase of an iteration. At the end of the kernel the
// CTA's word reaches the handle's status word (ST_DEBUG, the site of the
// first failure in bits 8..15), which sf_sync_status reports as
// SF_ERR_DEBUG_CHECK.
#pragma once
#include "sf_internal.cuh"

#ifndef SF_DEBUG_CHECKS
#define SF_DEBUG_CHECKS 0
#endif

namespace sf {

// sites of the checks (also the values sf_last_error names)
enum DebugSite : int {
  DS_PAIR_DECODE = 1,   // pair (i, j) decoded from a candidate bit outside 0 <= i < j < N
  DS_CHUNK_ROW = 2,     // chunk-buffer row beyond the chunk buffer
  DS_TMEM_COL = 3,      // TMEM column beyond the CTA's allocation
  DS_TABLE = 4,         // MMA B-table word beyond its table
  DS_MASK = 5,          // activity-mask word beyond the sample's slot
  DS_OUT = 6,           // global output index beyond the batch
  DS_CANARY_HEAD = 7,   // canary after the shared-memory head overwritten
  DS_CANARY_BLOCK = 8,  // canary at the end of a sample block overwritten
};

constexpr unsigned kCanary = 0x5AFEC0DEu;
constexpr int kCanaryWords = SF_DEBUG_CHECKS ? 4 : 0;   // words added to the head and to every sample block

#if SF_DEBUG_CHECKS
__device__ __forceinline__ int& dbg_word() {
  __shared__ int w;
  return w;
}
#endif

// true when the check passes (always in a release build); a failure records
// the site (first failure of the CTA wins)
__device__ __forceinline__ bool dcheck(bool ok, int site) {
#if SF_DEBUG_CHECKS
  if (!ok) atomicCAS(&dbg_word(), 0, site);
  return ok;
#else
  (void)site;
  return true;
#endif
}

// before the kernel's first barrier
__device__ __forceinline__ void dbg_begin() {
#if SF_DEBUG_CHECKS
  if (threadIdx.x == 0) dbg_word() = 0;
#endif
}

// after the kernel's last barrier
__device__ __forceinline__ void dbg_end(int* status) {
#if SF_DEBUG_CHECKS
  __syncthreads();
  if (threadIdx.x == 0 && dbg_word() != 0) atomicOr(status, ST_DEBUG | ((dbg_word() & 0xFF) << 8));
#else
  (void)status;
#endif
}

// Canary words: 4 words before samp (the end of the head) and the last 4
// words of each of the G sample blocks of `sb` floats. plant > 0 (the test
// of the checks) writes a wrong value into the last block's canary.
__device__ __forceinline__ void canary_set(float* samp, int sb, int G, int plant) {
#if SF_DEBUG_CHECKS
  unsigned* h = reinterpret_cast<unsigned*>(samp) - 4;
  for (int v = threadIdx.x; v < 4 * (G + 1); v += blockDim.x) {
    const int b = v >> 2, w = v & 3;
    unsigned* p = b == 0 ? h + w : reinterpret_cast<unsigned*>(samp + (size_t)b * sb) - 4 + w;
    *p = kCanary ^ (unsigned)v;
    if (plant && b == G && w == 3) *p = ~(kCanary ^ (unsigned)v);
  }
#else
  (void)samp; (void)sb; (void)G; (void)plant;
#endif
}

__device__ __forceinline__ void canary_check(const float* samp, int sb, int G) {
#if SF_DEBUG_CHECKS
  const unsigned* h = reinterpret_cast<const unsigned*>(samp) - 4;
  for (int v = threadIdx.x; v < 4 * (G + 1); v += blockDim.x) {
    const int b = v >> 2, w = v & 3;
    const unsigned* p = b == 0 ? h + w : reinterpret_cast<const unsigned*>(samp + (size_t)b * sb) - 4 + w;
    dcheck(*p == (kCanary ^ (unsigned)v), b == 0 ? DS_CANARY_HEAD : DS_CANARY_BLOCK);
  }
#else
  (void)samp; (void)sb; (void)G;
#endif
}

}  // namespace sf
