// Fused forward of the safety filter: one launch runs all K iterations of
// f_FP (Appendix, AM steps) for many samples, with every sample's
// coefficient-space state (xi, lambda) resident in shared memory.
//
// CTA = G samples of one scene. The time axis is processed in chunks of TC
// steps. Per iteration and chunk:
//  * pair phase — one thread per (sample, t), the (sample, t) pairs of the
//    chunk laid out flat over the CTA's lanes: positions p_i(t) = P[t] c_i of
//    all robots, then every pair (i < j) by the alpha / beta / d closed forms,
//    q = e - delta accumulated per robot in registers (E_i += q, E_j -= q).
//    A pair that is inactive on all 32 lanes of a warp is skipped after its
//    distance test. E_i(t) goes to a shared-memory chunk buffer. With pair
//    pruning, only the rows recorded as candidates at the last full test
//    are retested while a drift bound shows the others still inactive.
//  * contraction phase — one thread per (sample, robot, range of t): the
//    robot's coefficients in registers, velocity / acceleration and their
//    ball projections, and the transposed contraction
//      g_i += P[t] E_i(t) + Pd[t] qv_i(t) + Pdd[t] qa_i(t)
//    (F^T of the residual, Eq. lambda_step) kept in registers and added to a
//    per-range partial.
// Then the solve phase: lambda' = lambda + rho g (minus-sign reading),
// r = rho g + lambda' + xi_bar, robot means, and the xi step
//   c_i' = W1 c_i + S1 r_i + DW cbar + DS rbar + beta_i
// with the operators pre-stored from the KKT system; DW cbar + DS rbar is
// the same for every robot of a (sample, axis) and formed once for it.
// After the last iteration one more pass evaluates
//   ||r_p|| = ||F xi^K - e(xi^{K-1})||  (Eq. primal_residual)
// row by row as F(xi^K - xi^{K-1}) - q(xi^{K-1}).
// Every reduction is done in a fixed order: results are bit-reproducible.
#pragma once
#include "sf_debug.cuh"
#include "sf_internal.cuh"
#include "sf_pack16.cuh"

namespace sf {
namespace fused_impl {

constexpr unsigned FULL = 0xffffffffu;

// Pair pruning (float32 forward). A full pair test of a sample records as
// candidates the pair rows with scaled distance < 1 + kPruneMargin; while the
// sample's coefficients stay within kPruneMargin / 2 (minus a rounding slack)
// of the coefficients of that test, in the bound below, only candidates are
// tested. Bound: with Bernstein weights P[t][k] >= 0 summing to 1,
// |M^-1 (p_i(t) - p_i^ref(t))| <= max_k |M^-1 (c_ik - c_ik^ref)|
// <= sqrt(dim) max_{k,x} |c_ikx - c_ikx^ref| / a_x, so a pair that was not a
// candidate is still at scaled distance > 1 and inactive.
constexpr float kPruneMargin = 0.5f;
constexpr float kPruneCandS2 = (1.0f + kPruneMargin) * (1.0f + kPruneMargin);
constexpr float kPruneDriftLimit = 0.5f * kPruneMargin - 1e-3f;
// Workspace rows: a full test records the robots with workspace-scaled
// offset > 1 - kWsMargin; the others stay inside while the workspace-scaled
// drift sqrt(dim) max_x (a_x / w_x) max |c - c_ref| / a_x stays below it.
constexpr float kWsMargin = 0.1f;
constexpr float kWsCandS2 = (1.0f - kWsMargin) * (1.0f - kWsMargin);
constexpr float kWsDriftLimit = kWsMargin - 1e-3f;

// ---- tensor-memory form: sizes ------------------------------------------
// Per time chunk the velocity / acceleration products run as M = 128 MMAs
// (rows = (sample, robot) of the CTA, columns = time steps of the chunk,
// padded to TCW = a multiple of 16) for Pd, Pdd and every axis, A = the
// coefficient rows in TMEM (rounded and remainder copies of 16 k), B =
// per-chunk basis tables in shared memory. Operand format 0: tf32 (K = 8
// per instruction, tables of 12 k per row, three 128-byte core matrices per
// 8 rows); 1 / 2: bf16 / fp16 (K = 16, two core matrices per 8 rows).
constexpr int TM_TABLES = 4;   // Pd, Pdd; rounded and remainder
// A pair-phase chunk of tc steps is split into tm_nsub(tc) TMEM sub-chunks of
// at most 64 steps (tm_ts(tc) steps, the last one shorter), whose states
// occupy TCW = tm_tcw(tc) columns per (state, axis).
__host__ __device__ constexpr int tm_nsub(int tc) { return (tc + 63) / 64; }
__host__ __device__ constexpr int tm_ts(int tc) { return (tc + tm_nsub(tc) - 1) / tm_nsub(tc); }
__host__ __device__ constexpr int tm_tcw(int tc) { return (tm_ts(tc) + 15) / 16 * 16; }
__host__ __device__ constexpr int tm_ka(int fmt) { return fmt == 0 ? 16 : 8; }
__host__ __device__ constexpr int tm_sbo(int fmt) { return fmt == 0 ? 384 : 256; }
// TMEM columns: the states of one sub-chunk [2][dim][TCW], then A [dim][2][KA]
__host__ __device__ constexpr int tm_cols(int dim, int tc, int fmt) { return 2 * dim * tm_tcw(tc) + 2 * dim * tm_ka(fmt); }
__host__ __device__ constexpr int tm_alloc_cols(int cols) {
  return cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
}
// Bytes of one B table: sub-chunk j of chunk c (global sub-chunk c nsub + j)
// at rows (c nsub + j) TCW, plus one zero 8-row group (the tf32 form's
// second K step reads one core matrix past a group; the coefficients'
// k >= 11 are zero, so any finite value there adds nothing).
__host__ __device__ constexpr int tm_tab_bytes(int T, int tc, int fmt) {
  return ((T + tc - 1) / tc * tm_nsub(tc) * tm_tcw(tc) / 8 + 1) * tm_sbo(fmt);
}

// Shared-memory layout (floats). Head: (tensor-memory form) the MMA B
// tables, then the float32 basis [T][36], operators, beta.
// Per sample: C, LAM, XIB [NMAX][DIM][12]; PG [NPG][NMAX][DIM][12] (partials
// of F^T q, later r; one in the tensor-memory form); MC, MR
// [DIM][12] (forward: MR holds the xi step's mean term DW mean(c) + DS
// mean(r); adjoint: DS^T mean(xb) and DW^T mean(xb)); EB [TC][EP] (E of the
// chunk, EP = NMAX*DIM + 1, or NMAX*DIM + 4 in the tensor-memory form, whose
// element NMAX*DIM flags an active pair; also holds xi^{K-1} after the last
// iteration); RS2 [T] (pair residual per t); RSB [NQ][NMAX] (ball residual
// partials); with pair pruning: CR [NMAX][DIM][12] (coefficients at the last
// full pair test), CM [T][CMW] (candidate pair rows of that test), WC [T]
// (candidate workspace rows: robots near or outside the workspace), RF (in the
// first sample's block: the largest drift of the CTA's coefficients since
// then, as the bit pattern of a non-negative float).
struct Lay {
  int RS, EP, TC, NQ, NPG, PQ1, T, nmax, dim;
  int C, LAM, XIB, PG, MC, MR, EB, RS2, RSB, FPP, FPR, XB, LB, GXB, U, CW, CR, CM, WC, RF, CMW, SB;
  int head, basis, opso, betao;
  __host__ __device__ Lay(int dim_, int nmax_, int T_, int TC_, int NQ_, bool bwd = false, bool cand = false,
                          int tmp = -1) {
    dim = dim_; nmax = nmax_; T = T_; TC = TC_; NQ = NQ_;
    // partials of F^T q in shared memory: one per time range (NPG = NQ),
    // partial 0 at PG and partial q >= 1 at PQ1 + (q - 1) nmax RS; one in
    // the tensor-memory form (its warp groups sum theirs through TMEM)
    NPG = tmp >= 0 ? 1 : NQ;
    const int npg_smem = NPG;
    RS = dim * NP;
    // tmp >= 0: tensor-memory form with operand format tmp (0 tf32, 1 bf16,
    // 2 fp16): chunk-buffer rows 16-byte aligned with the active-pair flag
    // at NMAX * DIM
    EP = nmax * dim + (tmp >= 0 ? 4 : 1);
    C = 0;
    LAM = C + nmax * RS;
    XIB = LAM + nmax * RS;
    PG = XIB + nmax * RS;
    MC = PG + npg_smem * nmax * RS;
    MR = MC + dim * NP;
    EB = MR + dim * NP;
    int eb = TC * EP;
    if (eb < nmax * RS) eb = nmax * RS;
    PQ1 = PG + nmax * RS;
    RS2 = EB + ((eb + 3) / 4) * 4;
    RSB = RS2 + T;
    FPP = RSB + NQ * nmax;
    FPR = FPP + dim * NV + nmax * dim;
    XB = ((FPR + 1 + 3) / 4) * 4;
    LB = XB + (bwd ? nmax * RS : 0);
    GXB = LB + (bwd ? nmax * RS : 0);
    U = GXB + (bwd ? nmax * RS : 0);
    CW = U + (bwd ? nmax * RS : 0);
    // pair pruning (float32 forward): reference coefficients, candidate
    // pair masks per (t) of mask_pair_words rounded to 4 words, workspace
    // candidate robots per (t), drift word
    CMW = cand ? (mask_pair_words(nmax) + 3) / 4 * 4 : 0;
    CR = CW + (bwd ? nmax * RS : 0);
    CM = CR + (cand ? nmax * RS : 0);
    WC = CM + T * CMW;
    RF = WC + (cand ? ((T + 3) / 4) * 4 : 0);
    SB = RF + (cand ? 4 : 0) + kCanaryWords;   // (debug builds: canary words at the end)
    // head: (tensor-memory form) the MMA B tables (Pd, Pdd; rounded and
    // remainder), then the float32 basis [T][36], the operators and beta
    basis = tmp >= 0 ? TM_TABLES * tm_tab_bytes(T, TC, tmp) / 4 : 0;
    opso = basis + T * BASIS_ROW;
    betao = opso + 4 * NV * NP;
    head = betao + nmax * RS + kCanaryWords;
  }
};

__device__ __forceinline__ void row_from(const float* __restrict__ src, float (&r)[NV]) {
  const float4* p = reinterpret_cast<const float4*>(src);
  const float4 a = p[0], b = p[1], c = p[2];
  r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
  r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
  r[8] = c.x; r[9] = c.y; r[10] = c.z;
}

__device__ __forceinline__ float dot_row(const float (&r)[NV], const float* crow) {
  const float4* c4 = reinterpret_cast<const float4*>(crow);
  const float4 a = c4[0], b = c4[1], c = c4[2];
  float s = r[0] * a.x;
  s = fmaf(r[1], a.y, s); s = fmaf(r[2], a.z, s); s = fmaf(r[3], a.w, s);
  s = fmaf(r[4], b.x, s); s = fmaf(r[5], b.y, s); s = fmaf(r[6], b.z, s);
  s = fmaf(r[7], b.w, s); s = fmaf(r[8], c.x, s); s = fmaf(r[9], c.y, s);
  s = fmaf(r[10], c.z, s);
  return s;
}

__device__ __forceinline__ float dot_reg(const float (&r)[NV], const float (&c)[NV]) {
  float s = r[0] * c[0];
#pragma unroll
  for (int k = 1; k < NV; ++k) s = fmaf(r[k], c[k], s);
  return s;
}

template <int DIM>
__device__ __forceinline__ void state(const float (&r)[NV], const float* Crow, float (&p)[DIM]) {
#pragma unroll
  for (int x = 0; x < DIM; ++x) p[x] = dot_row(r, Crow + x * NP);
}

// One pair row (i < j): q = e(delta) - delta with delta = p_i - p_j, added to
// E_i and subtracted from E_j. The scaled distance s2 >= 1 means the row is
// inactive (e = delta); a warp skips the rest when no lane is active.
template <int DIM>
__device__ __forceinline__ void pair_update(const float (&pi)[DIM], const float (&pj)[DIM], float (&Ei)[DIM],
                                            float (&Ej)[DIM], bool valid, const ProblemConsts& pc,
                                            float& res2) {
  float d[DIM];
#pragma unroll
  for (int x = 0; x < DIM; ++x) d[x] = pi[x] - pj[x];
  float s2;
  if (DIM == 3)
    s2 = fmaf(d[2] * d[2], pc.inv_b2, (d[0] * d[0] + d[1] * d[1]) * pc.inv_a2);
  else
    s2 = (d[0] * d[0] + d[1] * d[1]) * pc.inv_a2;
  s2 = valid ? s2 : 2.0f;
  if (__any_sync(FULL, s2 < 1.0f)) {
    const bool zero = (s2 == 0.0f);
    float f = fmaxf(rsqrtf(s2) - 1.0f, 0.0f);
    f = zero ? 0.0f : f;
    float q[DIM];
#pragma unroll
    for (int x = 0; x < DIM; ++x) q[x] = f * d[x];
    if (zero) q[DIM == 3 ? 2 : 0] = pc.tie;
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      Ei[x] += q[x];
      Ej[x] -= q[x];
      res2 = fmaf(q[x], q[x], res2);
    }
  }
}

// Pair row (i < j) of bit idx of an activity / candidate mask (row-major
// upper triangle of NMAX x NMAX, the inverse of pair_bit): row i is the
// largest with start s_i = i (2 NMAX - i - 1) / 2 <= idx, from the root of
// the quadratic, corrected by one where the float root rounds across an
// integer.
template <int NMAX>
__device__ __forceinline__ void pair_of_bit(int idx, int& i, int& j) {
  constexpr float b = 2.0f * NMAX - 1.0f;
  int r = (int)((b - sqrtf(b * b - 8.0f * (float)idx)) * 0.5f);
  r = max(0, min(r, NMAX - 2));
  if ((r + 1) * (2 * NMAX - r - 2) / 2 <= idx) ++r;
  else if (r * (2 * NMAX - r - 1) / 2 > idx) --r;
  i = r;
  j = idx - r * (2 * NMAX - r - 1) / 2 + r + 1;
}

// Positions in the pair phase are kept scaled by M_a^-1 = diag(1/a, 1/a, 1/b),
// so the distance test of a pair row is |ps_i - ps_j|^2 < 1.
template <int DIM>
__device__ __forceinline__ float scaled_d2(const float (&pi)[DIM], const float (&pj)[DIM]) {
  float s2 = 0.0f;
#pragma unroll
  for (int x = 0; x < DIM; ++x) {
    const float d = pi[x] - pj[x];
    s2 = fmaf(d, d, s2);
  }
  return s2;
}

// q = e - delta of one pair row from scaled positions: delta = M (ps_i - ps_j);
// e = delta / sqrt(s2) inside the spheroid, delta outside, (0, 0, b) / (a, 0)
// at delta = 0. Added to E_i, subtracted from E_j.
template <int DIM>
__device__ __forceinline__ void pair_apply_scaled(const float (&pi)[DIM], const float (&pj)[DIM], float (&Ei)[DIM],
                                                  float (&Ej)[DIM], const ProblemConsts& pc, float& res2) {
  float ds[DIM];
#pragma unroll
  for (int x = 0; x < DIM; ++x) ds[x] = pi[x] - pj[x];
  float s2 = 0.0f;
#pragma unroll
  for (int x = 0; x < DIM; ++x) s2 = fmaf(ds[x], ds[x], s2);
  const bool zero = (s2 == 0.0f);
  float f = fmaxf(rsqrtf(s2) - 1.0f, 0.0f);
  f = zero ? 0.0f : f;
  float q[DIM];
#pragma unroll
  for (int x = 0; x < DIM; ++x) q[x] = f * ds[x] * (x == 2 ? pc.coll_b : pc.coll_a);
  if (zero) q[DIM == 3 ? 2 : 0] = pc.tie;
#pragma unroll
  for (int x = 0; x < DIM; ++x) {
    Ei[x] += q[x];
    Ej[x] -= q[x];
    res2 = fmaf(q[x], q[x], res2);
  }
}

// Update of one pair row known to be active on some lane of the warp.
template <int DIM>
__device__ __forceinline__ void pair_apply(const float (&pi)[DIM], const float (&pj)[DIM], float (&Ei)[DIM],
                                           float (&Ej)[DIM], bool valid, const ProblemConsts& pc,
                                           float& res2) {
  float d[DIM];
#pragma unroll
  for (int x = 0; x < DIM; ++x) d[x] = pi[x] - pj[x];
  float s2;
  if (DIM == 3)
    s2 = fmaf(d[2] * d[2], pc.inv_b2, (d[0] * d[0] + d[1] * d[1]) * pc.inv_a2);
  else
    s2 = (d[0] * d[0] + d[1] * d[1]) * pc.inv_a2;
  s2 = valid ? s2 : 2.0f;
  const bool zero = (s2 == 0.0f);
  float f = fmaxf(rsqrtf(s2) - 1.0f, 0.0f);
  f = zero ? 0.0f : f;
  float q[DIM];
#pragma unroll
  for (int x = 0; x < DIM; ++x) q[x] = f * d[x];
  if (zero) q[DIM == 3 ? 2 : 0] = pc.tie;
#pragma unroll
  for (int x = 0; x < DIM; ++x) {
    Ei[x] += q[x];
    Ej[x] -= q[x];
    res2 = fmaf(q[x], q[x], res2);
  }
}

// Workspace row of one robot from its collision-scaled position ps: when
// outside the workspace spheroid, q = e - p = (p - p_w) (1 / sqrt(s2) - 1) is
// added to the robot's E (the row is P c_i, like a pair row's), its square to
// res2, and (MASKS) the row's activity bit is set.
template <int DIM, int NMAX, bool MASKS>
__device__ __forceinline__ void ws_row(const float (&ps)[DIM], float (&Ei)[DIM], bool valid, int i,
                                       const ProblemConsts& pc, float& res2, unsigned* mrow) {
  float w[DIM], s2 = 0.0f;
#pragma unroll
  for (int x = 0; x < DIM; ++x) {
    w[x] = fmaf(ps[x], pc.wk[x], -pc.wo[x]);
    s2 = fmaf(w[x], w[x], s2);
  }
  if (valid && s2 > 1.0f) {
    const float f = rsqrtf(s2) - 1.0f;
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      const float q = f * (w[x] * pc.wa[x]);
      Ei[x] += q;
      res2 = fmaf(q, q, res2);
    }
    if (MASKS) {
      const int b = 2 * NMAX + i;
      atomicOr(mrow + mask_pair_words(NMAX) + (b >> 5), 1u << (b & 31));
    }
  }
}

// Pair phase of one chunk [t0, t0 + TCc). With MASKS the lane's
// activity-mask row (mk + (s T + t) mask_words) is cleared and the bit of
// every active pair row is set.
// With CAND (pair pruning on) each sample is tested in full (recording its
// candidates and, in the first chunk, copying C to the reference
// coefficients) when its drift word requires it, otherwise only its recorded
// candidate rows are tested, the robots' positions computed on demand and E
// accumulated in the row.
// FLAG (tensor-memory form) writes the row's active-pair flag and stores the
// row in 16-byte pieces (rows of NMAX*DIM + 4 floats); a row whose flag is
// clear is left as it is (never read).
template <int DIM, int NMAX, bool MASKS = false, bool CAND = false, bool FLAG = false>
__device__ void pair_phase(float* SAMP, const Lay& L, const float* BASIS, int G, int N, int t0, int TCc,
                           const ProblemConsts& pc, bool want_res, int warp, int nwarps, int lane,
                           unsigned* mk = nullptr, bool prune = false) {
  constexpr int MW = mask_words(NMAX);
  constexpr int RS = DIM * NP;
  constexpr int PW = mask_pair_words(NMAX);
  const int nA = G * TCc;
  for (int base = warp * 32; base < nA; base += nwarps * 32) {
    const int u = base + lane;
    const bool valid = u < nA;
    const int s = valid ? u / TCc : 0;
    const int tl = valid ? u - s * TCc : 0;
    const int t = t0 + tl;
    float* blk = SAMP + (size_t)s * L.SB;
    const float* Cs = blk + L.C;
    float Pr[NV];
    row_from(BASIS + (size_t)t * BASIS_ROW, Pr);
    float res2 = 0.0f;
    // this lane's row of the chunk buffer (a row past the buffer, which a
    // debug build reports, is redirected to row 0)
    float* ebw = blk + L.EB + (dcheck(L.EB + (tl + 1) * L.EP <= L.RS2, DS_CHUNK_ROW) ? tl : 0) * L.EP;
    unsigned* mrow = MASKS ? mk + ((size_t)s * L.T + t) * MW : nullptr;
    if (MASKS && valid) {
#pragma unroll
      for (int q = 0; q < MW / 4; ++q) reinterpret_cast<uint4*>(mrow)[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    // records pair row (i, j) of this lane as active
    auto mark = [&](int i, int j, bool act) {
      if (MASKS && valid && act) {
        const int b = pair_bit(NMAX, i, j);
        atomicOr(mrow + (b >> 5), 1u << (b & 31));
      }
    };
    // pair pruning: full test (and record candidates) or candidates only.
    // The decision is taken for the whole CTA (a full test of every sample as
    // soon as one sample needs it): a full test of one sample resets the
    // drift of all, so the CTA runs fewer full-test iterations than with a
    // decision per sample (measured: 22 against 38 of 200 on the bench
    // workload), and the warps of a phase do the same kind of work.
    bool refresh = true;
    unsigned* cmrow = nullptr;
    if (CAND) {
      refresh = !prune;
      float wkmax = 0.0f;
#pragma unroll
      for (int x = 0; x < DIM; ++x) wkmax = fmaxf(wkmax, pc.wk[x]);
      if (!refresh) {
        // the CTA's drift word (in the first sample's block): the largest
        // drift of any of its samples
        const float drift = sqrtf((float)DIM) * __int_as_float(*reinterpret_cast<const int*>(SAMP + L.RF));
        refresh = !(drift < kPruneDriftLimit) || (pc.use_w && !(drift * wkmax < kWsDriftLimit));  // NaN: full
      }
      cmrow = reinterpret_cast<unsigned*>(blk + L.CM) + (size_t)t * L.CMW;
    }
    const bool rec = CAND && refresh && valid;
    auto cand = [&](int i, int j, float s2) {
      if (CAND && rec && s2 < kPruneCandS2) {
        const int b = pair_bit(NMAX, i, j);
        cmrow[b >> 5] |= 1u << (b & 31);
      }
    };
    if (rec) {
      for (int q = 0; q < L.CMW / 4; ++q) reinterpret_cast<uint4*>(cmrow)[q] = make_uint4(0u, 0u, 0u, 0u);
      if (t0 == 0)
        for (int v = tl; v < NMAX * RS; v += TCc) blk[L.CR + v] = Cs[v];
    }
    // pair rows (bits in pair_bit order) and workspace robots (bits) whose
    // projection is applied into the lane's row of the chunk buffer: the
    // recorded candidates, or the active rows that a full test found (N <= 16)
    unsigned wsel[(PW + 3) / 4 * 4];
    unsigned wsm = 0u;
    bool apply = false;
    if (CAND && !__any_sync(FULL, refresh)) {
      // candidate path: no warp-wide votes below, lanes run their own lists
      apply = true;
      const uint4* c4 = reinterpret_cast<const uint4*>(cmrow);
#pragma unroll
      for (int q = 0; q < (PW + 3) / 4; ++q) {
        const uint4 v = c4[q];
        wsel[4 * q] = v.x; wsel[4 * q + 1] = v.y; wsel[4 * q + 2] = v.z; wsel[4 * q + 3] = v.w;
      }
      if (pc.use_w) wsm = reinterpret_cast<const unsigned*>(blk + L.WC)[t];
    } else if (NMAX <= 16) {
      // full test: scaled positions of all robots in registers, every pair
      // row and workspace row tested branch-free; the active ones are then
      // applied by the same loop as the candidates (one copy of the
      // projection code). Lanes past the chunk get far-apart dummies so that
      // none of their rows tests active.
      apply = true;
      float p[NMAX][DIM];
#pragma unroll
      for (int i = 0; i < NMAX; ++i) {
        if (i < N) {
          state<DIM>(Pr, Cs + i * RS, p[i]);
#pragma unroll
          for (int x = 0; x < DIM; ++x) p[i][x] *= (x == 2 ? pc.inv_b : pc.inv_a);
        } else {
#pragma unroll
          for (int x = 0; x < DIM; ++x) p[i][x] = 0.0f;
        }
        if (!valid) p[i][0] = 4096.0f * (float)i;
      }
      unsigned cmr[PW];
#pragma unroll
      for (int q = 0; q < PW; ++q) {
        cmr[q] = 0u;
        wsel[q] = 0u;
      }
#pragma unroll
      for (int i = 0; i < NMAX; ++i)
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
          if (j > i && j < N) {
            const float s2 = scaled_d2<DIM>(p[i], p[j]);
            const int b = pair_bit(NMAX, i, j);
            wsel[b >> 5] |= (s2 < 1.0f) ? (1u << (b & 31)) : 0u;
            if (CAND) cmr[b >> 5] |= (s2 < kPruneCandS2) ? (1u << (b & 31)) : 0u;
          }
      if (CAND && rec) {
#pragma unroll
        for (int q = 0; q < PW; ++q) cmrow[q] = cmr[q];
      }
      // workspace rows of every robot (Eq. workspace_con)
      if (pc.use_w) {
        unsigned wsc = 0u;
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
          if (i < N) {
            float s2 = 0.0f;
#pragma unroll
            for (int x = 0; x < DIM; ++x) {
              const float w = fmaf(p[i][x], pc.wk[x], -pc.wo[x]);
              s2 = fmaf(w, w, s2);
            }
            wsm |= (s2 > 1.0f) ? (1u << i) : 0u;
            if (CAND) wsc |= (s2 > kWsCandS2) ? (1u << i) : 0u;
          }
        if (CAND && rec) reinterpret_cast<unsigned*>(blk + L.WC)[t] = wsc;
      }
    } else {
      // full test, N > 16: scaled positions staged once in the lane's own
      // row of the chunk buffer (overwritten by E when the active rows are
      // applied below), robots in blocks of 8 reloaded from there, each
      // later robot tested against a block in one group; active rows as bits
      apply = true;
#pragma unroll
      for (int q = 0; q < PW; ++q) wsel[q] = 0u;
#pragma unroll
      for (int i = 0; i < NMAX; ++i) {
        if (i < N) {
          float pi[DIM];
          state<DIM>(Pr, Cs + i * RS, pi);
          if (valid)
#pragma unroll
            for (int x = 0; x < DIM; ++x) ebw[i * DIM + x] = pi[x] * (x == 2 ? pc.inv_b : pc.inv_a);
        }
      }
      auto sel = [&](int i, int j, float s2) {
        const int b = pair_bit(NMAX, i, j);
        wsel[b >> 5] |= (s2 < 1.0f) ? (1u << (b & 31)) : 0u;
        cand(i, j, s2);
      };
#pragma unroll
      for (int I0 = 0; I0 < NMAX; I0 += 8) {
        if (I0 < N) {
          float pI[8][DIM];
#pragma unroll
          for (int a = 0; a < 8; ++a) {
#pragma unroll
            for (int x = 0; x < DIM; ++x) pI[a][x] = (valid && I0 + a < N) ? ebw[(I0 + a) * DIM + x] : 0.0f;
            if (!valid) pI[a][0] = 4096.0f * (float)(I0 + a);
          }
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b)
              if (b > a && I0 + b < N) sel(I0 + a, I0 + b, scaled_d2<DIM>(pI[a], pI[b]));
#pragma unroll
          for (int j = 0; j < NMAX; ++j) {
            if (j >= I0 + 8 && j < N) {
              float pj[DIM];
#pragma unroll
              for (int x = 0; x < DIM; ++x) pj[x] = valid ? ebw[j * DIM + x] : 0.0f;
              if (!valid) pj[0] = 4096.0f * (float)j;
#pragma unroll
              for (int a = 0; a < 8; ++a) sel(I0 + a, j, scaled_d2<DIM>(pI[a], pj));
            }
          }
        }
      }
      if (pc.use_w) {
        unsigned wsc = 0u;
        for (int i = 0; i < N; ++i) {
          float s2 = 0.0f;
#pragma unroll
          for (int x = 0; x < DIM; ++x) {
            const float w = fmaf(valid ? ebw[i * DIM + x] : 0.0f, pc.wk[x], -pc.wo[x]);
            s2 = fmaf(w, w, s2);
          }
          if (valid && s2 > 1.0f) wsm |= 1u << i;
          if (CAND && s2 > kWsCandS2) wsc |= 1u << i;
        }
        if (CAND && rec) reinterpret_cast<unsigned*>(blk + L.WC)[t] = wsc;
      }
    }
    if (apply) {
      // FLAG: the row is cleared (16-byte stores) only when the lane meets
      // its first active row; a row whose flag stays clear is never read
      bool zeroed = !FLAG;
      auto ensure_zero = [&]() {
        if (FLAG && !zeroed) {
#pragma unroll
          for (int q = 0; q < NMAX * DIM / 4; ++q)
            reinterpret_cast<float4*>(ebw)[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          zeroed = true;
        }
      };
      if (valid) {
        if (!FLAG)
          for (int q = 0; q < N * DIM; ++q) ebw[q] = 0.0f;
#pragma unroll
        for (int q = 0; q < PW; ++q) {
          unsigned m = wsel[q];
          while (m) {
            const int idx = q * 32 + __ffs(m) - 1;
            m &= m - 1;
            int i, j;
            pair_of_bit<NMAX>(idx, i, j);
            if (!dcheck(i >= 0 && i < j && j < N, DS_PAIR_DECODE)) continue;
            float pi[DIM], pj[DIM];
            state<DIM>(Pr, Cs + i * RS, pi);
            state<DIM>(Pr, Cs + j * RS, pj);
#pragma unroll
            for (int x = 0; x < DIM; ++x) {
              pi[x] *= (x == 2 ? pc.inv_b : pc.inv_a);
              pj[x] *= (x == 2 ? pc.inv_b : pc.inv_a);
            }
            if (scaled_d2<DIM>(pi, pj) < 1.0f) {
              float Ei[DIM], Ej[DIM];
#pragma unroll
              for (int x = 0; x < DIM; ++x) Ei[x] = Ej[x] = 0.0f;
              mark(i, j, true);
              pair_apply_scaled<DIM>(pi, pj, Ei, Ej, pc, res2);
              ensure_zero();
#pragma unroll
              for (int x = 0; x < DIM; ++x) {
                ebw[i * DIM + x] += Ei[x];
                ebw[j * DIM + x] += Ej[x];
              }
            }
          }
        }
        if (pc.use_w) {   // workspace rows of the selected robots
          unsigned m = wsm;
          while (m) {
            const int i = __ffs(m) - 1;
            m &= m - 1;
            float pi[DIM], Ei[DIM];
            state<DIM>(Pr, Cs + i * RS, pi);
#pragma unroll
            for (int x = 0; x < DIM; ++x) {
              pi[x] *= (x == 2 ? pc.inv_b : pc.inv_a);
              Ei[x] = 0.0f;
            }
            ws_row<DIM, NMAX, MASKS>(pi, Ei, true, i, pc, res2, mrow);
            bool act = false;
#pragma unroll
            for (int x = 0; x < DIM; ++x) act |= Ei[x] != 0.0f;
            if (act || !FLAG) {
              ensure_zero();
#pragma unroll
              for (int x = 0; x < DIM; ++x) ebw[i * DIM + x] += Ei[x];
            }
          }
        }
        if (FLAG) ebw[NMAX * DIM] = zeroed ? 1.0f : 0.0f;
      }
    }
    if (valid && want_res) blk[L.RS2 + t] = res2;
  }
}

// Contraction phase of one chunk: F^T of the residual per (sample, robot).
// Each 11-term group P[t] E, Pd[t] qv, Pdd[t] qa is skipped when it is zero
// on every lane of the warp (inactive rows contribute exactly 0). With MASKS
// the ball rows outside their ball set their bits in the activity masks.
template <int DIM, int NMAX = 0, bool MASKS = false>
__device__ void contract_phase(float* SAMP, const Lay& L, const float* BASIS, int G, int N, int t0, int TCc,
                               bool first_chunk, const ProblemConsts& pc, bool want_res, int tid, int nthr,
                               unsigned* mk = nullptr) {
  const int RS = DIM * NP;
  const int NQ = L.NQ;
  const int nB = NQ * G * N;
  const int TQ = (TCc + NQ - 1) / NQ;
  const int lane = tid & 31;
  for (int base = tid - lane; base < nB; base += nthr) {
    const int u = base + lane;
    const bool uvalid = u < nB;
    const int uu = uvalid ? u : 0;
    const int i = uu % N;
    const int s = (uu / N) % G;
    const int tq = uu / (N * G);
    const int ta = tq * TQ;
    const int trip = uvalid ? max(0, min(ta + TQ, TCc) - ta) : 0;
    int wtrip = trip;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) wtrip = max(wtrip, __shfl_xor_sync(FULL, wtrip, o));
    float* blk = SAMP + (size_t)s * L.SB;
    float c[DIM][NV], g[DIM][NV];
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      row_from(blk + L.C + i * RS + x * NP, c[x]);
#pragma unroll
      for (int k = 0; k < NV; ++k) g[x][k] = 0.0f;
    }
    float rb = 0.0f;
    for (int step = 0; step < wtrip; ++step) {
      const bool live = step < trip;
      const int tl = live ? ta + step : ta;
      const float* brow = BASIS + (size_t)(t0 + tl) * BASIS_ROW;
      float Pd[NV], Pdd[NV];
      row_from(brow + NP, Pd);
      row_from(brow + 2 * NP, Pdd);
      const float* eb = blk + L.EB + tl * L.EP + i * DIM;
      float e[DIM], qv[DIM], qa[DIM];
      bool ne = false;
#pragma unroll
      for (int x = 0; x < DIM; ++x) {
        e[x] = live ? eb[x] : 0.0f;
        ne |= e[x] != 0.0f;
        qv[x] = 0.0f;
        qa[x] = 0.0f;
      }
      float rl = 0.0f;
      unsigned* mball = nullptr;
      if (MASKS)
        mball = mk + ((size_t)s * L.T + t0 + tl) * mask_words(NMAX) + mask_pair_words(NMAX);
      // ball rows: the projection (rsqrt, residual, its square) only runs when
      // some lane of the warp is outside its ball; inside, q = 0 exactly
      if (pc.use_v) {
        float v[DIM], n2 = 0.0f;
#pragma unroll
        for (int x = 0; x < DIM; ++x) {
          v[x] = dot_reg(Pd, c[x]);
          n2 = fmaf(v[x], v[x], n2);
        }
        const bool out = n2 > pc.v_max * pc.v_max;
        if (__any_sync(FULL, out)) {
          ball_residual<DIM>(v, pc.v_max, qv, rl);
          if (MASKS && live && out) atomicOr(mball + (i >> 5), 1u << (i & 31));
        }
      }
      if (pc.use_a) {
        float a[DIM], n2 = 0.0f;
#pragma unroll
        for (int x = 0; x < DIM; ++x) {
          a[x] = dot_reg(Pdd, c[x]);
          n2 = fmaf(a[x], a[x], n2);
        }
        const bool out = n2 > pc.a_max * pc.a_max;
        if (__any_sync(FULL, out)) {
          ball_residual<DIM>(a, pc.a_max, qa, rl);
          if (MASKS && live && out) {
            const int b = NMAX + i;
            atomicOr(mball + (b >> 5), 1u << (b & 31));
          }
        }
      }
      if (live) rb += rl;
      if (__any_sync(FULL, ne)) {
        float P[NV];
        row_from(brow, P);
#pragma unroll
        for (int x = 0; x < DIM; ++x)
#pragma unroll
          for (int k = 0; k < NV; ++k) g[x][k] = fmaf(P[k], e[x], g[x][k]);
      }
      if (__any_sync(FULL, live && rl > 0.0f)) {
#pragma unroll
        for (int x = 0; x < DIM; ++x)
#pragma unroll
          for (int k = 0; k < NV; ++k) {
            float acc = g[x][k];
            if (pc.use_v) acc = fmaf(Pd[k], live ? qv[x] : 0.0f, acc);
            if (pc.use_a) acc = fmaf(Pdd[k], live ? qa[x] : 0.0f, acc);
            g[x][k] = acc;
          }
      }
    }
    if (uvalid) {
      float* pg = blk + L.PG + tq * L.nmax * RS + i * RS;
#pragma unroll
      for (int x = 0; x < DIM; ++x)
#pragma unroll
        for (int k = 0; k < NV; ++k) pg[x * NP + k] = first_chunk ? g[x][k] : pg[x * NP + k] + g[x][k];
      if (want_res) {
        float* r = blk + L.RSB + tq * L.nmax + i;
        *r = first_chunk ? rb : *r + rb;
      }
    }
  }
}

// Final residual of one (sample, t): ||F xi^K - e(xi^{K-1})||^2 over the rows
// at t, written to RS2[t]. Cp holds xi^{K-1}, C holds xi^K.
template <int DIM, int NMAX>
__device__ void residual_phase(float* SAMP, const Lay& L, const float* BASIS, int G, int N, int T,
                               const ProblemConsts& pc, int warp, int nwarps, int lane) {
  constexpr int RS = DIM * NP;
  const int nA = G * T;
  for (int base = warp * 32; base < nA; base += nwarps * 32) {
    const int u = base + lane;
    const bool valid = u < nA;
    const int s = valid ? u / T : 0;
    const int t = valid ? u - s * T : 0;
    float* blk = SAMP + (size_t)s * L.SB;
    const float* C = blk + L.C;
    const float* Cp = blk + L.EB;
    float Pr[NV];
    row_from(BASIS + (size_t)t * BASIS_ROW, Pr);
    float r2 = 0.0f, dummy = 0.0f;
#pragma unroll
    for (int I0 = 0; I0 < NMAX; I0 += 8) {
      if (I0 < N) {
        float pI[8][DIM], dI[8][DIM];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          state<DIM>(Pr, Cp + (I0 + a) * RS, pI[a]);
          float pn[DIM];
          state<DIM>(Pr, C + (I0 + a) * RS, pn);
#pragma unroll
          for (int x = 0; x < DIM; ++x) dI[a][x] = pn[x] - pI[a][x];
        }
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = a + 1; b < 8; ++b) {
            if (I0 + b < N) {
              float q[DIM];
              pair_residual<DIM>(pI[a], pI[b], q, pc, dummy);
#pragma unroll
              for (int x = 0; x < DIM; ++x) {
                const float r = (dI[a][x] - dI[b][x]) - q[x];
                r2 = fmaf(r, r, r2);
              }
            }
          }
        for (int j = I0 + 8; j < N; ++j) {
          float pj[DIM], pn[DIM], dj[DIM];
          state<DIM>(Pr, Cp + j * RS, pj);
          state<DIM>(Pr, C + j * RS, pn);
#pragma unroll
          for (int x = 0; x < DIM; ++x) dj[x] = pn[x] - pj[x];
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            float q[DIM];
            pair_residual<DIM>(pI[a], pj, q, pc, dummy);
#pragma unroll
            for (int x = 0; x < DIM; ++x) {
              const float r = (dI[a][x] - dj[x]) - q[x];
              r2 = fmaf(r, r, r2);
            }
          }
        }
      }
    }
    float Pd[NV], Pdd[NV];
    row_from(BASIS + (size_t)t * BASIS_ROW + NP, Pd);
    row_from(BASIS + (size_t)t * BASIS_ROW + 2 * NP, Pdd);
    for (int i = 0; i < N; ++i) {
      if (pc.use_v) {
        float vo[DIM], vn[DIM], q[DIM];
        state<DIM>(Pd, Cp + i * RS, vo);
        state<DIM>(Pd, C + i * RS, vn);
        ball_residual<DIM>(vo, pc.v_max, q, dummy);
#pragma unroll
        for (int x = 0; x < DIM; ++x) {
          const float r = (vn[x] - vo[x]) - q[x];
          r2 = fmaf(r, r, r2);
        }
      }
      if (pc.use_a) {
        float ao[DIM], an[DIM], q[DIM];
        state<DIM>(Pdd, Cp + i * RS, ao);
        state<DIM>(Pdd, C + i * RS, an);
        ball_residual<DIM>(ao, pc.a_max, q, dummy);
#pragma unroll
        for (int x = 0; x < DIM; ++x) {
          const float r = (an[x] - ao[x]) - q[x];
          r2 = fmaf(r, r, r2);
        }
      }
      if (pc.use_w) {
        float po[DIM], pn[DIM], q[DIM];
        state<DIM>(Pr, Cp + i * RS, po);
        state<DIM>(Pr, C + i * RS, pn);
        ws_residual<DIM>(po, pc, q, dummy);
#pragma unroll
        for (int x = 0; x < DIM; ++x) {
          const float r = (pn[x] - po[x]) - q[x];
          r2 = fmaf(r, r, r2);
        }
      }
    }
    if (valid) blk[L.RS2 + t] = r2;
  }
}

// Per-CTA context: which scene and samples the CTA owns and where things
// live in shared memory.
template <int DIM, int NMAX>
struct Cta {
  Lay L;
  int N, G, robot_off, gsample0;
  long long per_sample, coef0, mask0;
  float *BASIS, *OPS, *BETA, *SAMP;
  int tid, nthr, warp, lane, nwarps;
  __device__ Cta(const SceneDesc* sc, int n_scenes, int T, int tc, int nq, bool bwd, float* sm, bool cand = false,
                 int tmp = -1)
      : L(DIM, NMAX, T, tc, nq, bwd, cand, tmp) {
    int sidx = 0;
    for (int q = 1; q < n_scenes; ++q) {
      if (sc[q].cta_begin <= (int)blockIdx.x) sidx = q;
      else break;
    }
    N = sc[sidx].N;
    const int Gs = sc[sidx].G;
    const int s_first = ((int)blockIdx.x - sc[sidx].cta_begin) * Gs;
    G = min(Gs, sc[sidx].S - s_first);
    robot_off = sc[sidx].robot_off;
    gsample0 = sc[sidx].sample_off + s_first;
    per_sample = (long long)DIM * N * NV;
    coef0 = sc[sidx].coef_off + (long long)s_first * per_sample;
    mask0 = sc[sidx].mask_off + (long long)s_first * T * mask_words(NMAX);
    BASIS = sm + L.basis;
    OPS = sm + L.opso;
    BETA = sm + L.betao;
    SAMP = sm + L.head;
    tid = threadIdx.x;
    nthr = blockDim.x;
    warp = tid >> 5;
    lane = tid & 31;
    nwarps = nthr >> 5;
  }
  // global index of coefficient (s, x, i, k) and shared offset of its row
  __device__ long long gidx(int s, int x, int i, int k) const {
    return coef0 + s * per_sample + ((long long)x * N + i) * NV + k;
  }
  __device__ float* blk(int s) const { return SAMP + (size_t)s * L.SB; }
};

// Basis table (float32 copy), operators of this N and
// beta_i = R1 b_i + (R0 - R1) bbar.
template <int DIM, int NMAX>
__device__ void prologue(const Cta<DIM, NMAX>& c, int T, const float4* basis, const float* ops,
                         const float* start, const float* goal, const float* start_va, const float* goal_va) {
  constexpr int RS = DIM * NP;
  {
    const float4* b4 = basis;
    float4* s4 = reinterpret_cast<float4*>(c.BASIS);
    for (int v = c.tid; v < T * 9; v += c.nthr) s4[v] = b4[v];
  }
  const float* gops = ops + (size_t)c.N * OPS_STRIDE;
  for (int v = c.tid; v < 4 * NV * NP; v += c.nthr) c.OPS[v] = gops[v];
  const int N = c.N;
  for (int v = c.tid; v < NMAX * RS; v += c.nthr) {
    const int i = v / RS, x = (v / NP) % DIM, k = v % NP;
    float beta = 0.0f;
    if (i < N && k < NV) {
      float bi[6] = {0, 0, 0, 0, 0, 0}, bm[6] = {0, 0, 0, 0, 0, 0};
      for (int j = 0; j < N; ++j) {
        const int rr = c.robot_off + j;
        float bj[6];
        bj[0] = start[rr * DIM + x];
        bj[1] = start_va ? start_va[(rr * 2 + 0) * DIM + x] : 0.0f;
        bj[2] = start_va ? start_va[(rr * 2 + 1) * DIM + x] : 0.0f;
        bj[3] = goal[rr * DIM + x];
        bj[4] = goal_va ? goal_va[(rr * 2 + 0) * DIM + x] : 0.0f;
        bj[5] = goal_va ? goal_va[(rr * 2 + 1) * DIM + x] : 0.0f;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          bm[q] += bj[q];
          if (j == i) bi[q] = bj[q];
        }
      }
      const float invN = 1.0f / (float)N;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float r0 = gops[OPS_R0 + k * 8 + q], r1 = gops[OPS_R1 + k * 8 + q];
        beta = fmaf(r1, bi[q], fmaf(r0 - r1, bm[q] * invN, beta));
      }
    }
    c.BETA[v] = beta;
  }
}

// Loads (xi, lambda) of every sample into C, LAM (rows beyond N and the
// padding column are zero) and clears the partials.
template <int DIM, int NMAX>
__device__ void load_state(const Cta<DIM, NMAX>& c, const float* xi, const float* lam, const float* fallback_xi,
                           const float* xi_bar_src) {
  constexpr int RS = DIM * NP;
  for (int v = c.tid; v < c.G * NMAX * RS; v += c.nthr) {
    const int s = v / (NMAX * RS), rem = v % (NMAX * RS);
    const int i = rem / RS, x = (rem / NP) % DIM, k = rem % NP;
    float* b = c.blk(s);
    float cv = 0.0f, l = 0.0f;
    if (i < c.N && k < NV) {
      const long long g = c.gidx(s, x, i, k);
      cv = xi ? xi[g] : fallback_xi[g];
      l = lam ? lam[g] : 0.0f;
    }
    b[c.L.C + rem] = cv;
    b[c.L.LAM + rem] = l;
    b[c.L.XIB + rem] = (i < c.N && k < NV) ? xi_bar_src[c.gidx(s, x, i, k)] : 0.0f;
    for (int q = 0; q < c.L.NPG; ++q) b[c.L.PG + q * NMAX * RS + rem] = 0.0f;
  }
}

// Copies C, LAM of every sample to global memory in the [dim][N][nvar] layout.
template <int DIM, int NMAX>
__device__ void store_state(const Cta<DIM, NMAX>& c, float* xi_dst, float* lam_dst, long long base) {
  constexpr int RS = DIM * NP;
  const int N = c.N;
  for (int v = c.tid; v < c.G * DIM * N * NV; v += c.nthr) {
    const int s = v / (DIM * N * NV), rem = v % (DIM * N * NV);
    const int x = rem / (N * NV), i = (rem / NV) % N, k = rem % NV;
    const float* b = c.blk(s);
    const int o = i * RS + x * NP + k;
    const long long g = base + c.coef0 + (long long)s * c.per_sample + rem;
    xi_dst[g] = b[c.L.C + o];
    lam_dst[g] = b[c.L.LAM + o];
  }
}

// The CTA-wide pruning decision of the pair phase: a full pair test when
// pruning is off or some sample's drift (or workspace drift) bound is
// reached.
template <int DIM, int NMAX>
__device__ __forceinline__ bool cta_refresh(const Cta<DIM, NMAX>& c, const Lay& L, const ProblemConsts& pc,
                                            bool prune) {
  if (!prune) return true;
  float wkmax = 0.0f;
#pragma unroll
  for (int x = 0; x < DIM; ++x) wkmax = fmaxf(wkmax, pc.wk[x]);
  const float drift = sqrtf((float)DIM) * __int_as_float(*reinterpret_cast<const int*>(c.SAMP + L.RF));
  return !(drift < kPruneDriftLimit) || (pc.use_w && !(drift * wkmax < kWsDriftLimit));
}

// Solve phase 1 of one iteration on every sample of the CTA: the lambda step
// lambda' = lambda + rho g (minus-sign reading of Eq. lambda_step), r = rho g +
// lambda' + xi_bar (kept in PG, partial 0), the robot means and the xi step's
// mean term DW mean(c) + DS mean(r) per (sample, axis) in MR, the history
// entry and (fp) the lambda part of ||z^{k+1} - z^k||^2.
template <int DIM, int NMAX, bool CAND>
__device__ void solve_lambda_means(const Cta<DIM, NMAX>& c, const ProblemConsts& pc, int it, float* hist,
                                   int total_samples, bool fp) {
  constexpr int RS = DIM * NP;
  const Lay& L = c.L;
  const int T = pc.T, N = c.N, G = c.G;
  const bool want_res = hist != nullptr;
  const float rho = pc.rho;
  const float invN = 1.0f / (float)N;
  // ---- solve phase 1: lambda step, r, robot means, and the mean term of
  // the xi step (and the history entry). Lanes (s, x, k) with k padded to 16,
  // so that the 11 k of one (s, x) share a half-warp: after the robot loop
  // each lane forms its k of DW mean(c) + DS mean(r) from its neighbours'
  // means by shuffles, and stores it in MR (phase 2 reads only that).
  {
    const int nB1 = G * DIM * 16;
    const int lane = c.lane;
    for (int base = c.tid - lane; base < nB1; base += c.nthr) {
      const int v = base + lane;
      const int vq = v < nB1 ? v : 0;
      const int s = vq / (DIM * 16), x = (vq >> 4) % DIM, k = vq & 15;
      const bool act = v < nB1 && k < NV;
      float* blk = c.blk(s);
      float sr = 0.0f, sc = 0.0f, dl2 = 0.0f;
      if (act) {
        const int o0 = x * NP + k;
        int i = 0;
        // four robots' loads first (no store in between), then their updates
        for (; i + 4 <= N; i += 4) {
          float gq[4], lq[4], xq[4], cq[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int o = (i + u) * RS + o0;
            float g = blk[L.PG + o];
            for (int q = 1; q < L.NPG; ++q) g += blk[L.PQ1 + (q - 1) * NMAX * RS + o];
            gq[u] = g;
            lq[u] = blk[L.LAM + o];
            xq[u] = blk[L.XIB + o];
            cq[u] = blk[L.C + o];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int o = (i + u) * RS + o0;
            const float lam = fmaf(rho, gq[u], lq[u]);
            dl2 = fmaf(lam - lq[u], lam - lq[u], dl2);
            blk[L.LAM + o] = lam;
            const float r = fmaf(rho, gq[u], lam) + xq[u];
            blk[L.PG + o] = r;
            sr += r;
            sc += cq[u];
          }
        }
        for (; i < N; ++i) {
          const int o = i * RS + o0;
          float g = blk[L.PG + o];
          for (int q = 1; q < L.NPG; ++q) g += blk[L.PQ1 + (q - 1) * NMAX * RS + o];
          const float lold = blk[L.LAM + o];
          const float lam = fmaf(rho, g, lold);
          dl2 = fmaf(lam - lold, lam - lold, dl2);
          blk[L.LAM + o] = lam;
          const float r = fmaf(rho, g, lam) + blk[L.XIB + o];
          blk[L.PG + o] = r;
          sr += r;
          sc += blk[L.C + o];
        }
      }
      const float mr = sr * invN, mc = sc * invN;
      float dw[NV], ds[NV];
      row_from(c.OPS + OPS_DW + (k < NV ? k : 0) * NP, dw);
      row_from(c.OPS + OPS_DS + (k < NV ? k : 0) * NP, ds);
      float m0 = 0.0f, m1 = 0.0f;
#pragma unroll
      for (int m = 0; m < NV; ++m) {
        m0 = fmaf(dw[m], __shfl_sync(FULL, mc, (lane & 16) + m), m0);
        m1 = fmaf(ds[m], __shfl_sync(FULL, mr, (lane & 16) + m), m1);
      }
      if (act) blk[L.MR + x * NP + k] = m0 + m1;
      if (CAND && act && s == 0 && x == 0 && k == 0)   // the CTA's drift since the reference
        *reinterpret_cast<int*>(c.SAMP + L.RF) = 0;
      if (fp && act) blk[L.FPP + x * NV + k] = dl2;
      if (want_res && act && x == 0 && k == 0) {
        float r2 = 0.0f;
        for (int t = 0; t < T; ++t) r2 += blk[L.RS2 + t];
        for (int q = 0; q < L.NQ; ++q)
          for (int i = 0; i < N; ++i) r2 += blk[L.RSB + q * NMAX + i];
        hist[(size_t)it * total_samples + c.gsample0 + s] = sqrtf(r2);
      }
    }
  }
}

// Solve phase 2 for one coefficient row (sample s, robot i, axis x): the xi
// step xi_i = W1 c_i + S1 r_i + (DW mean(c) + DS mean(r)) + beta_i with the
// operators pre-stored from the KKT system (Eq. xi_step). Writes the new row
// to C (and the old one to the EB region when keep_prev), raises the
// sample's drift word (pair pruning; with ATOMIC_DRIFT false the row's drift
// goes to *drift_bits instead, as the bit pattern of a non-negative float)
// and (fp) records ||xi' - xi||^2 of the row; out receives the new row
// (entry NV zero).
// The xi step of one row from its operands in registers: cc the row's
// coefficients, r its right-hand side rho g + lambda' + xi_bar, mt the mean
// term of its (sample, axis).
template <int DIM, int NMAX, bool CAND, bool ATOMIC_DRIFT = true>
__device__ __forceinline__ void xi_step_core(const Cta<DIM, NMAX>& c, const ProblemConsts& pc, int s, int i, int x,
                                             bool keep_prev, bool fp, const float (&cc)[NP], const float (&r)[NP],
                                             const float (&mt)[NP], float (&out)[NP], int* drift_bits) {
  constexpr int RS = DIM * NP;
  const Lay& L = c.L;
  float* blk = c.blk(s);
  const int o = i * RS + x * NP;
  float dx2 = 0.0f;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float w1[NV], s1[NV];
    row_from(c.OPS + OPS_W1 + k * NP, w1);
    row_from(c.OPS + OPS_S1 + k * NP, s1);
    float a0 = c.BETA[o + k] + mt[k], a1 = 0.0f;
#pragma unroll
    for (int m = 0; m < NV; ++m) {
      a0 = fmaf(w1[m], cc[m], a0);
      a1 = fmaf(s1[m], r[m], a1);
    }
    const float acc = a0 + a1;
    out[k] = acc;
    dx2 = fmaf(acc - cc[k], acc - cc[k], dx2);
  }
  out[NV] = 0.0f;
  if constexpr (CAND) {
    // drift of this coefficient row from the reference, in scaled units
    const float inv = x == 2 ? pc.inv_b : pc.inv_a;
    float d = 0.0f;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float e = fabsf(out[k] - blk[L.CR + o + k]) * inv;
      d = fmaxf(d, e);
      bad |= !(e == e);
    }
    if (ATOMIC_DRIFT)
      atomicMax(reinterpret_cast<int*>(c.SAMP + L.RF), __float_as_int(bad ? INFINITY : d));
    else
      *drift_bits = __float_as_int(bad ? INFINITY : d);
  }
  float4* o4 = reinterpret_cast<float4*>(blk + L.C + o);
  float4* p4 = reinterpret_cast<float4*>(blk + L.EB + o);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (keep_prev) p4[q] = make_float4(cc[4 * q], cc[4 * q + 1], cc[4 * q + 2], cc[4 * q + 3]);
    o4[q] = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
  }
  if (fp) blk[L.FPP + DIM * NV + i * DIM + x] = dx2;
}

template <int DIM, int NMAX, bool CAND, bool ATOMIC_DRIFT = true>
__device__ __forceinline__ void xi_step_row(const Cta<DIM, NMAX>& c, const ProblemConsts& pc, int s, int i, int x,
                                            bool keep_prev, bool fp, float (&out)[NP], int* drift_bits = nullptr) {
  constexpr int RS = DIM * NP;
  const Lay& L = c.L;
  float* blk = c.blk(s);
  const int o = i * RS + x * NP;
  float cc[NP], r[NP], mt[NP];
  const float4* c4 = reinterpret_cast<const float4*>(blk + L.C + o);
  const float4* r4 = reinterpret_cast<const float4*>(blk + L.PG + o);
  const float4* mt4 = reinterpret_cast<const float4*>(blk + L.MR + x * NP);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float4 a = c4[q], b = r4[q], e = mt4[q];
    cc[4 * q] = a.x; cc[4 * q + 1] = a.y; cc[4 * q + 2] = a.z; cc[4 * q + 3] = a.w;
    r[4 * q] = b.x; r[4 * q + 1] = b.y; r[4 * q + 2] = b.z; r[4 * q + 3] = b.w;
    mt[4 * q] = e.x; mt[4 * q + 1] = e.y; mt[4 * q + 2] = e.z; mt[4 * q + 3] = e.w;
  }
  xi_step_core<DIM, NMAX, CAND, ATOMIC_DRIFT>(c, pc, s, i, x, keep_prev, fp, cc, r, mt, out, drift_bits);
}

// One-pass solve of the float32 form for samples of at most 16 robots: one
// lane per (sample, axis, robot), the robots of a (sample, axis) on NMAX
// consecutive lanes. Each lane sums its row's partials of F^T q, takes the
// lambda step (minus-sign reading of Eq. lambda_step) and r = rho g + lambda'
// + xi_bar, the robot sums of c and r by shuffles over its segment, one k of
// the mean term DW mean(c) + DS mean(r) (gathered by shuffles), and then the
// xi step (Eq. xi_step) from registers. The drift word must have been reset
// before (no pair test of this iteration reads it afterwards).
template <int DIM, int NMAX, bool CAND>
__device__ void solve_onepass(const Cta<DIM, NMAX>& c, const ProblemConsts& pc, int it, bool keep_prev,
                              float* hist, int total_samples, bool fp) {
  static_assert(32 % NMAX == 0 && NMAX <= 16, "one-pass solve: robots of a sample within one warp");
  constexpr int RS = DIM * NP;
  constexpr int SW = NMAX;
  const Lay& L = c.L;
  const int T = pc.T, N = c.N, G = c.G;
  const float rho = pc.rho;
  const float invN = 1.0f / (float)N;
  const bool want_res = hist != nullptr;
  const int nL = G * DIM * NMAX;
  const int j = c.lane & (SW - 1);
  const int segbase = c.lane & ~(SW - 1);
  for (int base = c.warp * 32; base < nL; base += c.nwarps * 32) {
    const int u = base + c.lane;
    const int sx = u / NMAX;                 // (sample, axis) of the segment
    const int s = sx / DIM, x = sx - s * DIM, i = j;
    const bool in_cta = u < nL;
    const bool valid = in_cta && i < N;
    float* blk = c.blk(in_cta ? s : 0);
    const int o = i * RS + x * NP;
    float cc[NP], r[NP], mt[NP];
    float dl2 = 0.0f;
    if (valid) {
      float lo[NP], xb[NP], g[NP];
      const float4* c4 = reinterpret_cast<const float4*>(blk + L.C + o);
      const float4* l4 = reinterpret_cast<const float4*>(blk + L.LAM + o);
      const float4* b4 = reinterpret_cast<const float4*>(blk + L.XIB + o);
      const float4* g4 = reinterpret_cast<const float4*>(blk + L.PG + o);
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        const float4 a = c4[w], l = l4[w], b = b4[w], e = g4[w];
        cc[4 * w] = a.x; cc[4 * w + 1] = a.y; cc[4 * w + 2] = a.z; cc[4 * w + 3] = a.w;
        lo[4 * w] = l.x; lo[4 * w + 1] = l.y; lo[4 * w + 2] = l.z; lo[4 * w + 3] = l.w;
        xb[4 * w] = b.x; xb[4 * w + 1] = b.y; xb[4 * w + 2] = b.z; xb[4 * w + 3] = b.w;
        g[4 * w] = e.x; g[4 * w + 1] = e.y; g[4 * w + 2] = e.z; g[4 * w + 3] = e.w;
      }
      for (int q = 1; q < L.NPG; ++q) {
        const float4* p4 = reinterpret_cast<const float4*>(blk + L.PQ1 + (q - 1) * NMAX * RS + o);
#pragma unroll
        for (int w = 0; w < 3; ++w) {
          const float4 e = p4[w];
          g[4 * w] += e.x; g[4 * w + 1] += e.y; g[4 * w + 2] += e.z; g[4 * w + 3] += e.w;
        }
      }
      float ln[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        if (k < NV) {
          const float lam = fmaf(rho, g[k], lo[k]);
          dl2 = fmaf(lam - lo[k], lam - lo[k], dl2);
          ln[k] = lam;
          r[k] = fmaf(rho, g[k], lam) + xb[k];
        } else {
          ln[k] = lo[k];
          r[k] = 0.0f;
        }
      }
      float4* lw = reinterpret_cast<float4*>(blk + L.LAM + o);
#pragma unroll
      for (int w = 0; w < 3; ++w) lw[w] = make_float4(ln[4 * w], ln[4 * w + 1], ln[4 * w + 2], ln[4 * w + 3]);
    } else {
#pragma unroll
      for (int k = 0; k < NP; ++k) cc[k] = r[k] = 0.0f;
    }
    float sc[NV], sr[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      sc[k] = cc[k];
      sr[k] = r[k];
    }
#pragma unroll
    for (int w = SW / 2; w >= 1; w >>= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        sc[k] += __shfl_xor_sync(FULL, sc[k], w);
        sr[k] += __shfl_xor_sync(FULL, sr[k], w);
      }
    float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = j + h * SW;
      if (h == 1 && SW >= NV) break;
      float dw[NV], ds[NV];
      row_from(c.OPS + OPS_DW + (k < NV ? k : 0) * NP, dw);
      row_from(c.OPS + OPS_DS + (k < NV ? k : 0) * NP, ds);
      float m0 = 0.0f, m1 = 0.0f;
#pragma unroll
      for (int m = 0; m < NV; ++m) {
        m0 = fmaf(dw[m], sc[m] * invN, m0);
        m1 = fmaf(ds[m], sr[m] * invN, m1);
      }
      if (h == 0) v0 = m0 + m1;
      else v1 = m0 + m1;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if (k < NV) {
        const float a0 = __shfl_sync(FULL, v0, segbase + (k % SW));
        const float a1 = (SW < NV) ? __shfl_sync(FULL, v1, segbase + (k % SW)) : 0.0f;
        mt[k] = k < SW ? a0 : a1;
      } else {
        mt[k] = 0.0f;
      }
    }
    if (fp) {   // ||lambda' - lambda||^2 of the segment's rows, in the FPP slots of its axis
#pragma unroll
      for (int w = SW / 2; w >= 1; w >>= 1) dl2 += __shfl_xor_sync(FULL, dl2, w);
      if (in_cta)
        for (int k = j; k < NV; k += SW) blk[L.FPP + x * NV + k] = k == 0 ? dl2 : 0.0f;
    }
    if (want_res && in_cta && x == 0 && j == 0) {   // history entry of the sample
      float r2 = 0.0f;
      for (int t = 0; t < T; ++t) r2 += blk[L.RS2 + t];
      for (int q = 0; q < L.NQ; ++q)
        for (int i2 = 0; i2 < N; ++i2) r2 += blk[L.RSB + q * NMAX + i2];
      hist[(size_t)it * total_samples + c.gsample0 + s] = sqrtf(r2);
    }
    float out[NP];
    int db = 0;
    if (valid) xi_step_core<DIM, NMAX, CAND, false>(c, pc, s, i, x, keep_prev, fp, cc, r, mt, out, &db);
    if (CAND) {
#pragma unroll
      for (int w = SW / 2; w >= 1; w >>= 1) db = max(db, __shfl_xor_sync(FULL, db, w));
      if (j == 0 && in_cta) atomicMax(reinterpret_cast<int*>(c.SAMP + L.RF), db);
    }
  }
}

// One iteration of f_FP on every sample of the CTA (time chunks, then the
// lambda step and the xi step). keep_prev stores xi^k in the EB region for
// the final residual. fp (when set) adds ||z^{k+1} - z^k||^2 per sample to FPR.
template <int DIM, int NMAX, bool MASKS = false, bool CAND = false>
__device__ void fwd_iteration(const Cta<DIM, NMAX>& c, const ProblemConsts& pc, const float* xi_bar, int it,
                              bool keep_prev, float* hist, int total_samples, bool fp, unsigned* mslot = nullptr,
                              bool prune = false) {
  constexpr int RS = DIM * NP;
  const Lay& L = c.L;
  const int T = pc.T, N = c.N, G = c.G, TC = L.TC;
  const bool want_res = hist != nullptr;
  const float rho = pc.rho;
  const float invN = 1.0f / (float)N;
  for (int t0 = 0; t0 < T; t0 += TC) {
    const int TCc = min(TC, T - t0);
    if (MASKS && mslot != nullptr) {
      unsigned* mk = mslot + c.mask0;
      pair_phase<DIM, NMAX, true, CAND>(c.SAMP, L, c.BASIS, G, N, t0, TCc, pc, want_res, c.warp, c.nwarps,
                                               c.lane, mk, prune);
      __syncthreads();
      contract_phase<DIM, NMAX, true>(c.SAMP, L, c.BASIS, G, N, t0, TCc, t0 == 0, pc, want_res, c.tid, c.nthr,
                                      mk);
    } else {
      pair_phase<DIM, NMAX, false, CAND>(c.SAMP, L, c.BASIS, G, N, t0, TCc, pc, want_res, c.warp,
                                                c.nwarps, c.lane, nullptr, prune);
      __syncthreads();
      canary_check(c.SAMP, L.SB, G);
      contract_phase<DIM>(c.SAMP, L, c.BASIS, G, N, t0, TCc, t0 == 0, pc, want_res, c.tid, c.nthr);
    }
    // one-pass solve: the drift word is reset once every pair test of the
    // iteration has read it (the barrier below orders it before the xi step)
    if (CAND && 32 % NMAX == 0 && NMAX <= 16 && t0 + TC >= T && c.tid == 0)
      *reinterpret_cast<int*>(c.SAMP + L.RF) = 0;
    __syncthreads();
    canary_check(c.SAMP, L.SB, G);
  }
  if constexpr (32 % NMAX == 0 && NMAX <= 16) {
    solve_onepass<DIM, NMAX, CAND>(c, pc, it, keep_prev, hist, total_samples, fp);
  } else {
    solve_lambda_means<DIM, NMAX, CAND>(c, pc, it, hist, total_samples, fp);
    __syncthreads();
    canary_check(c.SAMP, L.SB, G);
    // ---- solve phase 2: xi step, xi_i = W1 c_i + S1 r_i + (DW mean(c) +
    // DS mean(r)) + beta_i per (sample, robot, axis)
    for (int v = c.tid; v < G * N * DIM; v += c.nthr) {
      const int s = v / (N * DIM), i = (v / DIM) % N, x = v % DIM;
      float out[NP];
      xi_step_row<DIM, NMAX, CAND>(c, pc, s, i, x, keep_prev, fp, out);
    }
  }
  __syncthreads();
  canary_check(c.SAMP, L.SB, G);
  if (fp) {
    for (int s = c.tid; s < G; s += c.nthr) {
      float* blk = c.blk(s);
      float acc = 0.0f;
      for (int q = 0; q < DIM * NV; ++q) acc += blk[L.FPP + q];
      for (int q = 0; q < N * DIM; ++q) acc += blk[L.FPP + DIM * NV + q];
      blk[L.FPR] += acc;
    }
    // FPR is read only after the last iteration's barrier
  }
}

// Writes checkpoint `ck` = (xi, lambda) of every sample: layout
// [ck][2][total coefficients] (xi first, then lambda).
template <int DIM, int NMAX>
__device__ void write_checkpoint(const Cta<DIM, NMAX>& c, float* ckpt, int ck, long long total_coefs) {
  float* base = ckpt + (size_t)ck * 2 * total_coefs;
  store_state<DIM, NMAX>(c, base, base + total_coefs, 0);
}

// MASKS (with checkpoints): the iterations of the last checkpoint segment
// also write their activity masks for the adjoint.
template <int DIM, int NMAX, int MAXT, bool MASKS = false>
__global__ void __launch_bounds__(MAXT, 1) fused_fwd_kernel(const __grid_constant__ FusedArgs A) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const ProblemConsts& pc = A.pc;
  const int T = pc.T;
  constexpr bool CAND = true;   // pair pruning (the 16-bit forms too)
  const Cta<DIM, NMAX> c(A.sc, A.n_scenes, T, A.tc, A.nq, false, sm, CAND);
  if (c.G <= 0) return;
  const Lay& L = c.L;
  const int N = c.N, G = c.G;
  const bool fp = A.fp_res2 != nullptr;
  dbg_begin();

  prologue<DIM, NMAX>(c, T, A.basis, A.ops, A.start, A.goal, A.start_va, A.goal_va);
  load_state<DIM, NMAX>(c, A.xi0, A.lam0, A.xi_bar, A.xi_bar);
  canary_set(c.SAMP, L.SB, G, A.dbg_plant);
  for (int s = c.tid; s < G; s += c.nthr) {
    c.blk(s)[L.FPR] = 0.0f;
    if (CAND) *reinterpret_cast<int*>(c.blk(s) + L.RF) = __float_as_int(INFINITY);   // first test is full
  }
  __syncthreads();

  // checkpoints: (xi, lambda) at iterations 0, ck, 2 ck, ...; after them a
  // tail holding every iterate of the last segment (last_ck .. K), so that
  // the backward does not recompute that segment
  const int n_ck = (pc.K + A.ck_every - 1) / A.ck_every;
  const int last_ck = (n_ck - 1) * A.ck_every;
  float* tail = A.ckpt ? A.ckpt + (size_t)n_ck * 2 * A.total_coefs : nullptr;
  for (int it = 0; it < pc.K; ++it) {
    if (A.ckpt && it % A.ck_every == 0) write_checkpoint<DIM, NMAX>(c, A.ckpt, it / A.ck_every, A.total_coefs);
    if (tail && it >= last_ck) write_checkpoint<DIM, NMAX>(c, tail, it - last_ck, A.total_coefs);
    unsigned* ms = (MASKS && A.amask && it >= last_ck) ? A.amask + (size_t)(it - last_ck) * A.amask_slot : nullptr;
    fwd_iteration<DIM, NMAX, MASKS, CAND>(c, pc, A.xi_bar, it, it == pc.K - 1, A.hist, A.total_samples, fp,
                                                ms, A.prune != 0);
  }
  if (tail) write_checkpoint<DIM, NMAX>(c, tail, pc.K - last_ck, A.total_coefs);

  // ---- final residual, Eq. (primal_residual); robot rows beyond N of the
  // xi^{K-1} copy are zero-filled first
  constexpr int RS = DIM * NP;
  for (int v = c.tid; v < G * NMAX * RS; v += c.nthr) {
    const int s = v / (NMAX * RS), rem = v % (NMAX * RS);
    if (rem / RS >= N) c.blk(s)[L.EB + rem] = 0.0f;
  }
  __syncthreads();
  residual_phase<DIM, NMAX>(c.SAMP, L, c.BASIS, G, N, T, pc, c.warp, c.nwarps, c.lane);
  __syncthreads();
  for (int s = c.tid; s < G; s += c.nthr) {
    const float* blk = c.blk(s);
    float r2 = 0.0f;
    for (int t = 0; t < T; ++t) r2 += blk[L.RS2 + t];
    const float r = sqrtf(r2);
    A.resid_out[c.gsample0 + s] = r;
    if (fp) A.fp_res2[c.gsample0 + s] = blk[L.FPR];
    if (!isfinite(r)) atomicOr(A.status, ST_NONFINITE);
  }
  store_state<DIM, NMAX>(c, A.xi_out, A.lam_out, 0);
  canary_check(c.SAMP, L.SB, G);
  dbg_end(A.status);
}

template <int DIM, int NMAX, int MAXT, bool MASKS = false>
cudaError_t launch_t(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  auto k = fused_fwd_kernel<DIM, NMAX, MAXT, MASKS>;
  if (l.warps * 32 > MAXT) return cudaErrorInvalidConfiguration;
  k<<<l.n_ctas, l.warps * 32, l.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fused_impl
}  // namespace sf
