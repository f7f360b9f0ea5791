// Dispatch of the fused forward kernel over (dim, robot-count bucket); the
// kernel template lives in sf_fused_kernel.cuh and each instantiation is
// compiled in its own translation unit (sf_fused_d*_n*.cu).
#include <algorithm>
#include <cmath>

#include "sf_tm_kernel.cuh"

namespace sf {

#define SF_DECL(D, NM)                                                                                   \
  cudaError_t launch_fused_d##D##_n##NM(const FusedArgs&, const FusedLaunch&, cudaStream_t);           \
  cudaError_t launch_fused_train_d##D##_n##NM(const FusedArgs&, const FusedLaunch&, cudaStream_t);     \
  cudaError_t launch_bwd_d##D##_n##NM(const FusedArgs&, const BwdLaunchArgs&, const FusedLaunch&,      \
                                      cudaStream_t);
SF_DECL(2, 8) SF_DECL(2, 16) SF_DECL(2, 24) SF_DECL(2, 32) SF_DECL(3, 8) SF_DECL(3, 16) SF_DECL(3, 24) SF_DECL(3, 32)
#define SF_DECL_TM(D, NM) \
  cudaError_t launch_tm_d##D##_n##NM(const FusedArgs&, const FusedLaunch&, cudaStream_t); \
  cudaError_t prepare_tm_d##D##_n##NM(int, int);
SF_DECL_TM(2, 8) SF_DECL_TM(2, 16) SF_DECL_TM(2, 24) SF_DECL_TM(2, 32)
SF_DECL_TM(3, 8) SF_DECL_TM(3, 16) SF_DECL_TM(3, 24) SF_DECL_TM(3, 32)
#undef SF_DECL
#undef SF_DECL_TM
#define SF_PREP(D, NM) cudaError_t prepare_fused_d##D##_n##NM(int); cudaError_t prepare_bwd_d##D##_n##NM(int); \
  cudaError_t prepare_fused_train_d##D##_n##NM(int);
SF_PREP(2, 8) SF_PREP(2, 16) SF_PREP(2, 24) SF_PREP(2, 32) SF_PREP(3, 8) SF_PREP(3, 16) SF_PREP(3, 24) SF_PREP(3, 32)
#undef SF_PREP

// Raises the dynamic shared-memory limit of every fused / adjoint kernel of
// this dimension (the tensor-memory kernels with the handle's operand
// format) once, at handle creation, so that no launch (and no stream capture)
// has to configure a kernel.
cudaError_t prepare_kernels(int dim, int smem, int prec) {
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  // tensor-memory form with the handle's operand format (tf32 for float32)
  if (dim == 3) {
    chk(prepare_tm_d3_n8(smem, prec)); chk(prepare_tm_d3_n16(smem, prec)); chk(prepare_tm_d3_n24(smem, prec));
    chk(prepare_tm_d3_n32(smem, prec));
  } else {
    chk(prepare_tm_d2_n8(smem, prec)); chk(prepare_tm_d2_n16(smem, prec)); chk(prepare_tm_d2_n24(smem, prec));
    chk(prepare_tm_d2_n32(smem, prec));
  }
  if (dim == 3) {
    chk(prepare_fused_d3_n8(smem)); chk(prepare_fused_d3_n16(smem)); chk(prepare_fused_d3_n24(smem));
    chk(prepare_fused_d3_n32(smem));
    chk(prepare_fused_train_d3_n8(smem)); chk(prepare_fused_train_d3_n16(smem));
    chk(prepare_fused_train_d3_n24(smem)); chk(prepare_fused_train_d3_n32(smem));
    chk(prepare_bwd_d3_n8(smem)); chk(prepare_bwd_d3_n16(smem)); chk(prepare_bwd_d3_n24(smem));
    chk(prepare_bwd_d3_n32(smem));
  } else {
    chk(prepare_fused_d2_n8(smem)); chk(prepare_fused_d2_n16(smem)); chk(prepare_fused_d2_n24(smem));
    chk(prepare_fused_d2_n32(smem));
    chk(prepare_fused_train_d2_n8(smem)); chk(prepare_fused_train_d2_n16(smem));
    chk(prepare_fused_train_d2_n24(smem)); chk(prepare_fused_train_d2_n32(smem));
    chk(prepare_bwd_d2_n8(smem)); chk(prepare_bwd_d2_n16(smem)); chk(prepare_bwd_d2_n24(smem));
    chk(prepare_bwd_d2_n32(smem));
  }
  return e;
}

int fused_max_warps(int nmax, bool bwd) { return (bwd && nmax > 16) ? 8 : 12; }

size_t fused_smem_bytes(int dim, int nmax, int T, int gmax, int tc, int nq, bool bwd, int prec) {
  const bool tm = prec >= PREC_TM_TF32;
  const fused_impl::Lay L(dim, nmax, T, tc, nq, bwd, !bwd, tm ? prec - PREC_TM_TF32 : -1);
  return sizeof(float) * ((size_t)L.head + (size_t)gmax * L.SB);
}

// Cost model: instruction slots of the pair phase (per (sample, t) lane) and
// of the contraction phase (per (sample, robot, t)), padded to whole rounds
// of the CTA's threads, over an issue rate that saturates at 4 warp
// instructions per cycle; plus a charge per block-wide barrier. The CTA count
// over the SM count gives the number of waves. The tensor-memory form (prec
// >= PREC_TM_TF32) charges its TMEM pass per 8-step block of a warp group
// instead of the contraction phase.
FusedPlan plan_fused(int dim, int nmax, int T, const int* nr, const int* ns, int n_scenes, int num_sms,
                     size_t smem_cap, int force_G, int force_warps, int force_tc, bool bwd, FusedPlan* top,
                     int n_top, int prec) {
  FusedPlan best;
  best.G = 0;
  best.cost = INFINITY;
  for (int q = 0; q < n_top; ++q) top[q] = FusedPlan{0, 0, 0, 0, 0, INFINITY};
  long long tot = 0;
  int Nbig = 1;
  for (int q = 0; q < n_scenes; ++q) {
    tot += ns[q];
    Nbig = std::max(Nbig, nr[q]);
  }
  const int maxw = fused_max_warps(nmax, bwd);
  const double cA = 0.5 * Nbig * (Nbig - 1) * 14.0 + 45.0 * Nbig;
  const double cB = 200.0;
  auto add_top = [&](const FusedPlan& cand) {
    if (cand.cost < best.cost) best = cand;
    if (top && n_top > 0) {
      // keep the n_top cheapest candidates, sorted by model cost
      int pos = n_top;
      while (pos > 0 && (top[pos - 1].G == 0 || cand.cost < top[pos - 1].cost)) --pos;
      if (pos < n_top) {
        for (int q = n_top - 1; q > pos; --q) top[q] = top[q - 1];
        top[pos] = cand;
      }
    }
  };
  const int gmax_try = (int)std::min<long long>(64, std::max<long long>(1, tot));
  for (int G = 1; G <= gmax_try; ++G) {
    if (force_G > 0 && G != force_G) continue;
    long long ctas = 0;
    for (int q = 0; q < n_scenes; ++q) ctas += (ns[q] + std::min(G, std::max(ns[q], 1)) - 1) / std::min(G, std::max(ns[q], 1));
    const double waves = std::ceil((double)ctas / num_sms);
    if (prec >= PREC_TM_TF32) {
      // tensor-memory form: G (sample, robot) rows in the 128 TMEM lanes,
      // warps in groups of four (one per lane quarter), one partial of F^T q
      // per group; a chunk of the pair phase is split into TMEM sub-chunks of
      // at most 64 steps (the velocity and acceleration states of a
      // sub-chunk beside the coefficient operand)
      if (G * nmax > 128) continue;
      const int fmt = prec - PREC_TM_TF32;
      int prev_tc = 0;
      for (int nch = 1; nch <= 8; ++nch) {
        const int tc = (T + nch - 1) / nch;
        if (tc == prev_tc) continue;
        prev_tc = tc;
        if (fused_impl::tm_cols(dim, tc, fmt) > 512) continue;
        if (force_tc > 0 && tc != force_tc) continue;
        const int real_nch = (T + tc - 1) / tc;
        const int nsub = fused_impl::tm_nsub(tc);
        const int nb = (fused_impl::tm_ts(tc) + 7) / 8;
        // warps of lane quarters with none of the CTA's rows skip the pass
        const int quarters = std::min(4, (G * nmax + 31) / 32);
        for (int w = 8; w <= maxw; w += 4) {
          if (force_warps > 0 && w != force_warps) continue;
          const int ncg = w / 4;
          // the groups' partials of F^T q pass through the allocated columns
          if (ncg * dim * 16 > fused_impl::tm_alloc_cols(fused_impl::tm_cols(dim, tc, fmt))) continue;
          const size_t smem = fused_smem_bytes(dim, nmax, T, G, tc, ncg, bwd, prec);
          if (smem + TM_STATIC_SMEM_RESERVE > smem_cap) continue;
          const double rate = std::min(4.0, w / 2.0);
          // TMEM pass: every warp walks its 8-step blocks (about 22 issue
          // slots per step: two ball tests, the E flag, votes), issue-bound
          // over the CTA or latency-bound per warp
          const double rounds = std::ceil((double)nb / ncg);
          const double tPass =
              std::max(quarters * ncg * rounds * 8.0 * 22.0 / rate, rounds * 8.0 * 22.0 * 2.0) * nsub;
          const double a_rounds = std::ceil((double)G * tc / (32.0 * w));
          const double tPair = a_rounds * w * cA / rate;
          const double per_iter = real_nch * (tPass + tPair) + ((1.0 + nsub) * real_nch + 3.0) * 400.0 +
                                  24.0 * G * Nbig * dim * 4.0 / rate;
          add_top(FusedPlan{G, w, tc, ncg, smem, waves * per_iter});
        }
      }
      continue;
    }
    for (int nch = 1; nch <= 6; ++nch) {
      const int tc = (T + nch - 1) / nch;
      if (force_tc > 0 && tc != force_tc) continue;
      for (int w = 4; w <= maxw; ++w) {
        if (force_warps > 0 && w != force_warps) continue;
        const int nthr = 32 * w;
        // a forced shape fixes the reduction order of F^T q for every batch
        // of the bucket: the time ranges follow from the bucket size then,
        // not from the batch's largest swarm
        const int nbase = (force_G > 0 || force_warps > 0 || force_tc > 0) ? nmax : Nbig;
        const int nq = std::max(1, std::min(tc, nthr / std::max(1, G * nbase)));
        const size_t smem = fused_smem_bytes(dim, nmax, T, G, tc, nq, bwd);
        if (smem > smem_cap) continue;
        const int real_nch = (T + tc - 1) / tc;
        const double rate = std::min(4.0, w / 2.0);
        const double a_rounds = std::ceil((double)G * tc / nthr);
        const double b_rounds = std::ceil((double)nq * G * Nbig / nthr);
        const double tq = std::ceil((double)tc / nq);
        const double per_iter = real_nch * (a_rounds * w * cA + b_rounds * w * tq * cB) / rate +
                                (2.0 * real_nch + 2.0) * 400.0 + 24.0 * G * Nbig * dim * 4.0 / rate;
        add_top(FusedPlan{G, w, tc, nq, smem, waves * per_iter});
      }
    }
  }
  return best;
}

cudaError_t launch_backward(const FusedArgs& a, const BwdLaunchArgs& b, const FusedLaunch& l, cudaStream_t st) {
  const int dim = a.pc.dim;
  if (dim == 3) {
    if (l.nmax == 8) return launch_bwd_d3_n8(a, b, l, st);
    if (l.nmax == 16) return launch_bwd_d3_n16(a, b, l, st);
    if (l.nmax == 24) return launch_bwd_d3_n24(a, b, l, st);
    if (l.nmax == 32) return launch_bwd_d3_n32(a, b, l, st);
  } else if (dim == 2) {
    if (l.nmax == 8) return launch_bwd_d2_n8(a, b, l, st);
    if (l.nmax == 16) return launch_bwd_d2_n16(a, b, l, st);
    if (l.nmax == 24) return launch_bwd_d2_n24(a, b, l, st);
    if (l.nmax == 32) return launch_bwd_d2_n32(a, b, l, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  const int dim = a.pc.dim;
  if (l.prec >= PREC_TM_TF32) {
#define SF_TM(D, NM) \
  if (dim == D && l.nmax == NM) return launch_tm_d##D##_n##NM(a, l, st);
    SF_TM(3, 8) SF_TM(3, 16) SF_TM(3, 24) SF_TM(3, 32) SF_TM(2, 8) SF_TM(2, 16) SF_TM(2, 24) SF_TM(2, 32)
#undef SF_TM
    return cudaErrorInvalidValue;
  }
  if (a.amask) {
    if (dim == 3) {
      if (l.nmax == 8) return launch_fused_train_d3_n8(a, l, st);
      if (l.nmax == 16) return launch_fused_train_d3_n16(a, l, st);
      if (l.nmax == 24) return launch_fused_train_d3_n24(a, l, st);
      if (l.nmax == 32) return launch_fused_train_d3_n32(a, l, st);
    } else if (dim == 2) {
      if (l.nmax == 8) return launch_fused_train_d2_n8(a, l, st);
      if (l.nmax == 16) return launch_fused_train_d2_n16(a, l, st);
      if (l.nmax == 24) return launch_fused_train_d2_n24(a, l, st);
      if (l.nmax == 32) return launch_fused_train_d2_n32(a, l, st);
    }
    return cudaErrorInvalidValue;
  }
  if (dim == 3) {
    if (l.nmax == 8) return launch_fused_d3_n8(a, l, st);
    if (l.nmax == 16) return launch_fused_d3_n16(a, l, st);
    if (l.nmax == 24) return launch_fused_d3_n24(a, l, st);
    if (l.nmax == 32) return launch_fused_d3_n32(a, l, st);
  } else if (dim == 2) {
    if (l.nmax == 8) return launch_fused_d2_n8(a, l, st);
    if (l.nmax == 16) return launch_fused_d2_n16(a, l, st);
    if (l.nmax == 24) return launch_fused_d2_n24(a, l, st);
    if (l.nmax == 32) return launch_fused_d2_n32(a, l, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sf
