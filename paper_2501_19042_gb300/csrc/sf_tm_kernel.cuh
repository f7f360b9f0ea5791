// Tensor-memory form of the fused forward: the velocity and acceleration
// states of every iteration (v = Pd c, a = Pdd c for all samples, robots,
// axes and time steps; Eq. poly), which the ball rows need at every time
// step of every iteration, run on the 5th-generation tensor cores
// (tcgen05.mma, one issuing thread, accumulators in TMEM); everything else as
// in the float32 form, the positions of the pair rows included (so that pair
// pruning stays exact).
//
// Per CTA (G samples of one scene, G * NMAX <= 128) and time chunk of TC
// steps, one MMA group per (state, axis):
//   D[(s, i)][t] = sum_k A_x[(s, i)][k] B_m[t][k]
// with M = 128 rows (sample, robot) in TMEM lanes, N = TCW time steps in TMEM
// columns, K = 16 (the 11 coefficients, zero-padded). A holds the
// coefficient rows in TMEM, written by the xi step of the previous
// iteration; B holds the basis rows of the chunk in shared memory. Both
// operands are split into a rounded copy and its rounding remainder and the
// product is taken in three terms (hi hi + lo hi + hi lo), so that the states
// keep about 21 bits (tf32, fp16) or 16 bits (bf16) of the float32 inputs.
//
// A thread of warp w owns TMEM lane 32 (w % 4) + lane = (sample, robot) and
// the 8-step blocks of the chunk congruent to w / 4: it reads its robot's
// velocities and accelerations from TMEM, applies the ball projections
// (Appendix, d step with 0 <= d <= 1) and accumulates F^T of their residuals
// and of the pair residuals E (Eq. lambda_step) in registers.
//
// Order per chunk: pair phase (float32 lanes) -> barrier -> bounded wait for
// the chunk's MMAs -> TMEM pass (balls and F^T of the chunk) -> barrier ->
// the issuing thread starts the next chunk's MMAs, which run under the next
// pair phase. The MMAs of chunk 0 are issued after the xi step.
#pragma once
#include "sf_fused_kernel.cuh"
#include "sf_tmem.cuh"

namespace sf {
namespace fused_impl {

// Time after which a wait for an MMA group is abandoned, unless the launch
// sets its own (an MMA group of a chunk completes in a few microseconds).
constexpr uint64_t kTmWaitNs = 1000000000ull;

// Shared state of the tensor-memory form (static shared memory).
struct TmShared {
  uint64_t bar;       // MMA completion of the current chunk
  uint64_t limit_ns;  // bound of every wait on bar
  uint32_t tbase;     // TMEM base address
  uint32_t lost;      // parity of the phase a wait gave up on
  int abort;          // a wait ran out: no more MMAs, outputs flagged
};

template <int FMT>
__device__ __forceinline__ uint32_t pack16(float lo, float hi) {
  return tc::pack2<FMT>(lo, hi);
}

// B tables: Pd and Pdd rows (m = 1, 2) of the float32 basis [T][36]
// (global), rounded (table 2 (m - 1)) and the rounding remainder (table
// 2 (m - 1) + 1), time step t of sub-chunk j of chunk c at row
// (c nsub + j) TCW + (t - c TC - j TS); every other entry zero.
template <int FMT>
__device__ void tm_tables(unsigned char* tb, int T, int TC, const float* gb, int tid, int nthr) {
  const int TCW = tm_tcw(TC), TS = tm_ts(TC), NSUB = tm_nsub(TC);
  const int TAB = tm_tab_bytes(T, TC, FMT);
  // table row of time step t
  auto row_of = [&](int t) {
    const int ci = t / TC, tl = t - ci * TC, j = tl / TS;
    return (ci * NSUB + j) * TCW + (tl - j * TS);
  };
  uint32_t* w = reinterpret_cast<uint32_t*>(tb);
  for (int v = tid; v < TM_TABLES * TAB / 4; v += nthr) w[v] = 0u;
  __syncthreads();
  constexpr uint32_t SBO = tm_sbo(FMT);
  if constexpr (FMT == 0) {
    for (int v = tid; v < T * 2 * 12; v += nthr) {
      const int t = v / 24, m = (v / 12) % 2, k = v % 12;
      const float x = gb[(size_t)t * BASIS_ROW + (1 + m) * NP + k];
      const int row = row_of(t);
      const uint32_t off = (row >> 3) * SBO + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
      if (!dcheck(off + 4 <= (uint32_t)TAB, DS_TABLE)) continue;
      const uint32_t h = tcg::tf32_rna(x);
      const uint32_t l = tcg::tf32_rna(x - __uint_as_float(h));
      *reinterpret_cast<uint32_t*>(tb + (2 * m) * TAB + off) = h;
      *reinterpret_cast<uint32_t*>(tb + (2 * m + 1) * TAB + off) = l;
    }
  } else {
    for (int v = tid; v < T * 2 * 8; v += nthr) {
      const int t = v / 16, m = (v / 8) % 2, k0 = 2 * (v % 8);
      const float* row_ = gb + (size_t)t * BASIS_ROW + (1 + m) * NP;
      const float x0 = k0 < NV ? row_[k0] : 0.0f;
      const float x1 = k0 + 1 < NV ? row_[k0 + 1] : 0.0f;
      const int row = row_of(t);
      const uint32_t off = (row >> 3) * SBO + (k0 >> 3) * 128 + (row & 7) * 16 + (k0 & 7) * 2;
      if (!dcheck(off + 4 <= (uint32_t)TAB, DS_TABLE)) continue;
      *reinterpret_cast<uint32_t*>(tb + (2 * m) * TAB + off) = pack16<FMT>(x0, x1);
      *reinterpret_cast<uint32_t*>(tb + (2 * m + 1) * TAB + off) =
          pack16<FMT>(x0 - tc::round16<FMT>(x0), x1 - tc::round16<FMT>(x1));
    }
  }
}

// Writes the coefficient row c (entries >= NV ignored, k >= NV zero) of this
// lane to A_x in TMEM: rounded copy, then the rounding remainder. Warp-wide
// (every lane of the warp takes part).
template <int DIM, int FMT>
__device__ __forceinline__ void tm_write_a(uint32_t lanebase, int TCW, int x, const float (&c)[NP]) {
  constexpr int KA = tm_ka(FMT);
  const uint32_t col = (uint32_t)(2 * DIM * TCW + x * 2 * KA);
  if constexpr (FMT == 0) {
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float v = k < NV ? c[k] : 0.0f;
      hi[k] = tcg::tf32_rna(v);
      lo[k] = tcg::tf32_rna(v - __uint_as_float(hi[k]));
    }
    tcg::st16(lanebase + col, hi);
    tcg::st16(lanebase + col + 16, lo);
  } else {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float v0 = 2 * q < NV ? c[2 * q] : 0.0f;
      const float v1 = 2 * q + 1 < NV ? c[2 * q + 1] : 0.0f;
      hi[q] = pack16<FMT>(v0, v1);
      lo[q] = pack16<FMT>(v0 - tc::round16<FMT>(v0), v1 - tc::round16<FMT>(v1));
    }
    tcg::st8(lanebase + col, hi);
    tcg::st8(lanebase + col + 8, lo);
  }
}

// Issues the MMAs of global sub-chunk ci (velocities and accelerations of
// every row and axis) and commits them to the mbarrier. One thread.
template <int DIM, int FMT>
__device__ void tm_issue(uint32_t tbase, uint32_t tabs, int TAB, int ci, int TC, uint64_t* bar) {
  constexpr int KA = tm_ka(FMT);
  constexpr uint32_t SBO = tm_sbo(FMT), LBO = 128;
  const int TCW = tm_tcw(TC);
  const uint32_t id = tcg::idesc(FMT == 0 ? 2u : (FMT == 1 ? 1u : 0u), 128u, (uint32_t)TCW);
  const uint32_t acol = (uint32_t)(2 * DIM * TCW);
  const uint32_t choff = (uint32_t)(ci * TCW / 8) * SBO;
#pragma unroll
  for (int m = 0; m < 2; ++m) {
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      const uint32_t d = tbase + (uint32_t)((m * DIM + x) * TCW);
      const uint32_t ah = tbase + acol + (uint32_t)(x * 2 * KA), al = ah + KA;
      const uint32_t bh = tabs + (uint32_t)(2 * m * TAB) + choff, bl = bh + (uint32_t)TAB;
      if constexpr (FMT == 0) {
#pragma unroll
        for (int st = 0; st < 2; ++st) {
          const uint64_t dh = tcg::sdesc(bh + st * 2 * LBO, LBO, SBO);
          const uint64_t dl = tcg::sdesc(bl + st * 2 * LBO, LBO, SBO);
          tcg::mma_ts<0>(d, ah + 8 * st, dh, id, st > 0 ? 1u : 0u);
          tcg::mma_ts<0>(d, al + 8 * st, dh, id, 1u);
          tcg::mma_ts<0>(d, ah + 8 * st, dl, id, 1u);
        }
      } else {
        const uint64_t dh = tcg::sdesc(bh, LBO, SBO);
        const uint64_t dl = tcg::sdesc(bl, LBO, SBO);
        tcg::mma_ts<1>(d, ah, dh, id, 0u);
        tcg::mma_ts<1>(d, al, dh, id, 1u);
        tcg::mma_ts<1>(d, ah, dl, id, 1u);
      }
    }
  }
  tcg::commit(bar);
}

// Bounded wait for the MMAs of the current chunk; a wait that runs out latches
// the timeout status and stops further MMAs.
__device__ __forceinline__ void tm_wait(TmShared& ts, uint32_t& phase, int* status) {
  if (!ts.abort) {
    if (!tcg::mbar_wait(&ts.bar, phase, ts.limit_ns)) {
      ts.abort = 1;
      ts.lost = phase;
      atomicOr(status, ST_TIMEOUT);
    }
  }
  phase ^= 1u;
  tcg::fence_after();
}

// Lane mapping of the TMEM passes.
struct TmLane {
  int r, s, i, cg, ncg;
  bool valid;
  uint32_t lanebase;
};
template <int DIM, int NMAX>
__device__ __forceinline__ TmLane tm_lane(const Cta<DIM, NMAX>& c, uint32_t tbase) {
  TmLane q;
  const int q4 = c.warp & 3;
  q.cg = c.warp >> 2;
  q.ncg = c.nwarps >> 2;
  q.r = 32 * q4 + c.lane;
  q.s = q.r / NMAX;
  q.i = q.r - q.s * NMAX;
  q.valid = q.s < c.G && q.i < c.N;
  q.lanebase = tbase + ((uint32_t)(32 * q4) << 16);
  return q;
}

// Loads of one 8-step block of the TMEM pass: the lane's velocities and
// accelerations (tcgen05.ld, completed by the caller's wait) and the
// active-pair flags of the block's steps.
template <int DIM, int NMAX>
__device__ __forceinline__ void tm_block_load(const TmLane& q, const float* blk, const Lay& L, int TCW, int tb,
                                              int TCc, int eb0, uint32_t (&v)[DIM][8], uint32_t (&a)[DIM][8],
                                              float (&fl)[8]) {
  // (a block past its state's columns, which a debug build reports, is
  // redirected to the first block)
  if (!dcheck(tb + 8 <= TCW, DS_TMEM_COL)) tb = 0;
#pragma unroll
  for (int x = 0; x < DIM; ++x) {
    tcg::ld8(q.lanebase + (uint32_t)(x * TCW + tb), v[x]);
    tcg::ld8(q.lanebase + (uint32_t)((DIM + x) * TCW + tb), a[x]);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
    fl[j] = (tb + j < TCc && dcheck(L.EB + (eb0 + tb + j + 1) * L.EP <= L.RS2, DS_CHUNK_ROW))
                ? blk[L.EB + (eb0 + tb + j) * L.EP + NMAX * DIM]
                : 0.0f;
}

// One 8-step block of the TMEM pass on loaded values: every lane first
// evaluates its 24 conditions (velocity outside, acceleration outside, pair
// row active, per step) into one word; a single warp-wide OR then tells
// which of the (rare) projections and F^T updates the warp has to run. Those
// run in a loop over the set bits (one copy of the code, not one per step),
// re-reading the step's state from TMEM (the warp takes the same bits, so
// the warp-wide loads stay converged).
template <int DIM, int NMAX>
__device__ __forceinline__ void tm_block(const TmLane& q, const float* blk, const Lay& L, const ProblemConsts& pc,
                                         int t0, int tb, int TCc, int TCW, int eb0, const float* gbasis, float vm2,
                                         float am2, const uint32_t (&v)[DIM][8], const uint32_t (&a)[DIM][8],
                                         const float (&fl)[8], float (&g)[DIM][NV], float& rb, unsigned* mk) {
  uint32_t bj[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float nv = 0.0f, na = 0.0f;
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      const float vx = __uint_as_float(v[x][j]), ax = __uint_as_float(a[x][j]);
      nv = fmaf(vx, vx, nv);
      na = fmaf(ax, ax, na);
    }
    const bool live = q.valid && tb + j < TCc;
    bj[j] = ((live && nv > vm2) ? (1u << j) : 0u) | ((live && na > am2) ? (1u << (8 + j)) : 0u) |
            ((live && fl[j] != 0.0f) ? (1u << (16 + j)) : 0u);
  }
  // a tree of ORs (no serial chain through the steps)
  const uint32_t bits = ((bj[0] | bj[1]) | (bj[2] | bj[3])) | ((bj[4] | bj[5]) | (bj[6] | bj[7]));
  uint32_t any = __reduce_or_sync(FULL, bits);
#pragma unroll 1
  while (any) {
    const int bit = __ffs(any) - 1;
    any &= any - 1;
    const int kind = bit >> 3, j = bit & 7;   // 0 velocity, 1 acceleration, 2 pair rows
    const bool mine = (bits >> bit) & 1u;
    const float* brow = gbasis + (size_t)(t0 + tb + j) * BASIS_ROW;
    float w[DIM];
    if (kind < 2) {
      uint32_t r[DIM];
#pragma unroll
      for (int x = 0; x < DIM; ++x) tcg::ld1(q.lanebase + (uint32_t)((kind * DIM + x) * TCW + tb + j), r[x]);
      tcg::wait_ld();
      tcg::tie(r);
      // lanes whose row is inside the ball take q = 0 (w = 0)
      float qb[DIM], rl = 0.0f;
#pragma unroll
      for (int x = 0; x < DIM; ++x) w[x] = mine ? __uint_as_float(r[x]) : 0.0f;
      ball_residual<DIM>(w, kind == 0 ? pc.v_max : pc.a_max, qb, rl);
      rb += rl;
      if (mk && mine) {   // activity mask of the ball row (training forward)
        unsigned* mball = mk + ((size_t)q.s * L.T + t0 + tb + j) * mask_words(NMAX) + mask_pair_words(NMAX);
        const int mb = kind * NMAX + q.i;
        atomicOr(mball + (mb >> 5), 1u << (mb & 31));
      }
#pragma unroll
      for (int x = 0; x < DIM; ++x) w[x] = qb[x];
    } else {
      const float* eb = blk + L.EB + (eb0 + tb + j) * L.EP + q.i * DIM;
#pragma unroll
      for (int x = 0; x < DIM; ++x) w[x] = mine ? eb[x] : 0.0f;
    }
    float P[NV];
    row_from(brow + (kind == 2 ? 0 : (1 + kind) * NP), P);
#pragma unroll
    for (int x = 0; x < DIM; ++x)
#pragma unroll
      for (int k = 0; k < NV; ++k) g[x][k] = fmaf(P[k], w[x], g[x][k]);
  }
}

// TMEM pass of one sub-chunk [t0, t0 + TCc) (after the pair phase of its
// chunk, whose chunk-buffer rows start eb0 steps earlier): the velocity /
// acceleration ball rows of this lane's robot from TMEM, F^T of their
// residuals and of the pair residuals E (chunk-buffer rows whose
// active-pair flag is set) into g, the balls' squared residuals into rb.
// (Issuing a block's loads before evaluating the previous block needs a
// second register buffer, which made the kernel spill.)
template <int DIM, int NMAX>
__device__ void tm_chunk_pass(const Cta<DIM, NMAX>& c, const TmLane& q, const ProblemConsts& pc, int t0, int TCc,
                              int TCW, const float* gbasis, float (&g)[DIM][NV], float& rb, unsigned* mk,
                              int eb0) {
  const Lay& L = c.L;
  if (32 * (c.warp & 3) >= c.G * NMAX) return;   // a lane quarter with none of the CTA's rows
  const float* blk = c.blk(q.valid ? q.s : 0);
  const float vm2 = pc.use_v ? pc.v_max * pc.v_max : INFINITY;
  const float am2 = pc.use_a ? pc.a_max * pc.a_max : INFINITY;
  for (int bk = q.cg; bk * 8 < TCc; bk += q.ncg) {
    uint32_t v[DIM][8], a[DIM][8];
    float fl[8];
    tm_block_load<DIM, NMAX>(q, blk, L, TCW, bk * 8, TCc, eb0, v, a, fl);
    tcg::wait_ld();
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      tcg::tie(v[x]);
      tcg::tie(a[x]);
    }
    tm_block<DIM, NMAX>(q, blk, L, pc, t0, bk * 8, TCc, TCW, eb0, gbasis, vm2, am2, v, a, fl, g, rb, mk);
  }
}

// One iteration of f_FP in the tensor-memory form (the MMAs of chunk 0 are in
// flight on entry). Ends with the xi step, which rewrites A in TMEM.
template <int DIM, int NMAX, int FMT, bool CAND, bool TRAIN>
__device__ void tm_iteration(const Cta<DIM, NMAX>& c, const ProblemConsts& pc, int it, bool keep_prev, float* hist,
                             int total_samples, bool prune, const float* gbasis, TmShared& ts, uint32_t tabs,
                             uint32_t& phase, int* status, unsigned* mk, bool fp) {
  constexpr int RS = DIM * NP;
  const Lay& L = c.L;
  const int T = pc.T, TC = L.TC, TCW = tm_tcw(TC);
  const int nch = (T + TC - 1) / TC;
  const int TAB = tm_tab_bytes(T, TC, FMT);
  const bool want_res = hist != nullptr;
  const TmLane q = tm_lane(c, ts.tbase);
  float g[DIM][NV];
#pragma unroll
  for (int x = 0; x < DIM; ++x)
#pragma unroll
    for (int k = 0; k < NV; ++k) g[x][k] = 0.0f;
  float rb = 0.0f;
  const int NSUB = tm_nsub(TC), TS = tm_ts(TC);
  for (int ci = 0; ci < nch; ++ci) {
    const int t0 = ci * TC, TCc = min(TC, T - t0);
    if (TRAIN && mk)
      pair_phase<DIM, NMAX, true, CAND, true>(c.SAMP, L, gbasis, c.G, c.N, t0, TCc, pc, want_res, c.warp,
                                                     c.nwarps, c.lane, mk, prune);
    else
      pair_phase<DIM, NMAX, false, CAND, true>(c.SAMP, L, gbasis, c.G, c.N, t0, TCc, pc, want_res, c.warp,
                                                      c.nwarps, c.lane, nullptr, prune);
    __syncthreads();
    canary_check(c.SAMP, L.SB, c.G);
    // the chunk's TMEM sub-chunks; the MMAs of the next sub-chunk start as
    // soon as the pass of this one has read the states
    for (int j = 0; j < NSUB; ++j) {
      const int s0 = j * TS, SCc = min(TS, TCc - s0);
      tm_wait(ts, phase, status);
      if (SCc > 0) tm_chunk_pass<DIM, NMAX>(c, q, pc, t0 + s0, SCc, TCW, gbasis, g, rb, TRAIN ? mk : nullptr, s0);
      tcg::fence_before();
      __syncthreads();
      const int next = ci * NSUB + j + 1;
      if (c.tid == c.nthr - 32 && next < nch * NSUB && !ts.abort) {
        tcg::fence_after();
        tm_issue<DIM, FMT>(ts.tbase, tabs, TAB, next, TC, &ts.bar);
      }
    }
  }
  // the warp groups' partials of F^T q, summed through TMEM: every group
  // parks its partial ([axis][16] words) in the allocated columns (the states
  // and A are not needed again before the xi step rewrites A), then group c
  // adds axis c (c, c + ncg, ...) of all groups' partials in group order and
  // writes the sum to PG
  {
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      uint32_t part[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) part[k] = k < NV ? __float_as_uint(g[x][k]) : 0u;
      tcg::st16(q.lanebase + (uint32_t)((q.cg * DIM + x) * 16), part);
    }
    tcg::wait_st();
  }
  constexpr bool SEG = (NMAX % 32 == 0) || (32 % NMAX == 0);
  constexpr int SW = NMAX < 32 ? NMAX : 32;
  // one-pass solve for samples of at most 16 robots (the robot sums of a
  // 32-lane segment cost more shuffles than they save: 44.8 against 44.1 ms
  // on the 32-robot workload)
  constexpr bool ONEPASS = 32 % NMAX == 0 && NMAX <= 16;
  if (q.valid && want_res) c.blk(q.s)[L.RSB + q.cg * NMAX + q.i] = rb;
  // (one-pass solve: every pair test of this iteration has read the drift
  // word, the xi step below raises it again)
  if (CAND && ONEPASS && c.tid == 0) *reinterpret_cast<int*>(c.SAMP + L.RF) = 0;
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  if constexpr (ONEPASS) {
    // One pass per (row, axis) lane: the groups' partials summed from TMEM,
    // the lambda step (minus-sign reading of Eq. lambda_step), r = rho g +
    // lambda' + xi_bar, the sample's robot means by shuffles over its NMAX
    // consecutive lanes, the mean term DW mean(c) + DS mean(r) formed for
    // one k per lane and gathered by shuffles, then the xi step (Eq. xi_step)
    // from registers. No shared-memory round trip of g, r or the means.
    const int j = c.lane & (SW - 1);           // the lane's place in its sample's segment
    const int segbase = c.lane & ~(SW - 1);
    const float rho = pc.rho;
    const float invN = 1.0f / (float)c.N;
    float* blk = c.blk(q.s < c.G ? q.s : 0);   // (rows are read and written only by valid lanes)
    for (int x = q.cg; x < DIM; x += q.ncg) {
      float g[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) g[k] = 0.0f;
      for (int o = 0; o < q.ncg; ++o) {
        uint32_t pa[8], pb[8];
        tcg::ld8(q.lanebase + (uint32_t)((o * DIM + x) * 16), pa);
        tcg::ld8(q.lanebase + (uint32_t)((o * DIM + x) * 16 + 8), pb);
        tcg::wait_ld();
        tcg::tie(pa);
        tcg::tie(pb);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          g[k] += __uint_as_float(pa[k]);
          g[8 + k] += __uint_as_float(pb[k]);
        }
      }
      const int o = q.i * RS + x * NP;
      float cc[NP], r[NP], mt[NP];
      float dl2 = 0.0f;
      if (q.valid) {
        float lo[NP], xb[NP];
        const float4* c4 = reinterpret_cast<const float4*>(blk + L.C + o);
        const float4* l4 = reinterpret_cast<const float4*>(blk + L.LAM + o);
        const float4* b4 = reinterpret_cast<const float4*>(blk + L.XIB + o);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const float4 a = c4[u], l = l4[u], b = b4[u];
          cc[4 * u] = a.x; cc[4 * u + 1] = a.y; cc[4 * u + 2] = a.z; cc[4 * u + 3] = a.w;
          lo[4 * u] = l.x; lo[4 * u + 1] = l.y; lo[4 * u + 2] = l.z; lo[4 * u + 3] = l.w;
          xb[4 * u] = b.x; xb[4 * u + 1] = b.y; xb[4 * u + 2] = b.z; xb[4 * u + 3] = b.w;
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
        for (int u = 0; u < 3; ++u) lw[u] = make_float4(ln[4 * u], ln[4 * u + 1], ln[4 * u + 2], ln[4 * u + 3]);
      } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) cc[k] = r[k] = 0.0f;
      }
      // robot sums of c and r over the sample's segment (rows beyond N and
      // lanes beyond the CTA's samples add zero)
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
      // the mean term, one k (two when the segment has fewer than NV lanes)
      // per lane, then gathered
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
      if (TRAIN && fp) {   // ||lambda' - lambda||^2 of the sample's rows, in its FPP slots of this axis
#pragma unroll
        for (int w = SW / 2; w >= 1; w >>= 1) dl2 += __shfl_xor_sync(FULL, dl2, w);
        if (q.s < c.G)
          for (int k = j; k < NV; k += SW) blk[L.FPP + x * NV + k] = k == 0 ? dl2 : 0.0f;
      }
      if (want_res && x == 0 && j == 0 && q.s < c.G) {   // history entry of the sample
        float r2 = 0.0f;
        for (int t = 0; t < T; ++t) r2 += blk[L.RS2 + t];
        for (int gq = 0; gq < L.NQ; ++gq)
          for (int i = 0; i < c.N; ++i) r2 += blk[L.RSB + gq * NMAX + i];
        hist[(size_t)it * total_samples + c.gsample0 + q.s] = sqrtf(r2);
      }
      float out[NP];
      int db = 0;
      if (q.valid)
        xi_step_core<DIM, NMAX, CAND, false>(c, pc, q.s, q.i, x, keep_prev, TRAIN && fp, cc, r, mt, out, &db);
      if (CAND) {
#pragma unroll
        for (int w = SW / 2; w >= 1; w >>= 1) db = max(db, __shfl_xor_sync(FULL, db, w));
        if (j == 0 && q.s < c.G) atomicMax(reinterpret_cast<int*>(c.SAMP + L.RF), db);
      }
    }
    // the new rows to A in TMEM, once no warp reads its partials from columns
    // that A covers
    if (2 * TCW < 16 * q.ncg) {
      tcg::fence_before();
      __syncthreads();
      tcg::fence_after();
    }
    for (int x = q.cg; x < DIM; x += q.ncg) {
      float row[NP];
      const float* cr = blk + L.C + q.i * RS + x * NP;
#pragma unroll
      for (int k = 0; k < NP; ++k) row[k] = (q.valid && k < NV) ? cr[k] : 0.0f;
      tm_write_a<DIM, FMT>(q.lanebase, TCW, x, row);
    }
  } else {
  for (int x = q.cg; x < DIM; x += q.ncg) {
      float sum[16];
  #pragma unroll
      for (int k = 0; k < 16; ++k) sum[k] = 0.0f;
      for (int o = 0; o < q.ncg; ++o) {
        uint32_t pa[8], pb[8];
        tcg::ld8(q.lanebase + (uint32_t)((o * DIM + x) * 16), pa);
        tcg::ld8(q.lanebase + (uint32_t)((o * DIM + x) * 16 + 8), pb);
        tcg::wait_ld();
        tcg::tie(pa);
        tcg::tie(pb);
  #pragma unroll
        for (int k = 0; k < 8; ++k) {
          sum[k] += __uint_as_float(pa[k]);
          sum[8 + k] += __uint_as_float(pb[k]);
        }
      }
      if (q.valid) {
        float* pg = c.blk(q.s) + L.PG + q.i * RS + x * NP;
  #pragma unroll
        for (int k = 0; k < NV; ++k) pg[k] = sum[k];
      }
    }
    tcg::fence_before();
    __syncthreads();
    canary_check(c.SAMP, L.SB, c.G);
    solve_lambda_means<DIM, NMAX, CAND>(c, pc, it, hist, total_samples, TRAIN && fp);
    __syncthreads();
    canary_check(c.SAMP, L.SB, c.G);
    // xi step, one (sample, robot) row per lane and the axes over the warp
    // groups; the new rows also go to A in TMEM
    // the CTA's drift word: the lanes of one sample reduce their rows' drift
    // by shuffles first (a sample's rows are NMAX consecutive lanes), then one
    // atomic per sample and warp
    for (int x = q.cg; x < DIM; x += q.ncg) {
      float out[NP];
      int db = 0;
      if (q.valid) {
        if (SEG)
          xi_step_row<DIM, NMAX, CAND, false>(c, pc, q.s, q.i, x, keep_prev, TRAIN && fp, out, &db);
        else
          xi_step_row<DIM, NMAX, CAND, true>(c, pc, q.s, q.i, x, keep_prev, TRAIN && fp, out);
      } else {
  #pragma unroll
        for (int k = 0; k < NP; ++k) out[k] = 0.0f;
      }
      if (CAND && SEG) {
  #pragma unroll
        for (int o = SW / 2; o >= 1; o >>= 1) db = max(db, __shfl_xor_sync(FULL, db, o));
        if ((c.lane & (SW - 1)) == 0 && q.s < c.G) atomicMax(reinterpret_cast<int*>(c.SAMP + L.RF), db);
      }
    tm_write_a<DIM, FMT>(q.lanebase, TCW, x, out);
    }
  }
  tcg::wait_st();
  tcg::fence_before();
  __syncthreads();
  canary_check(c.SAMP, L.SB, c.G);
  if (TRAIN && fp) {
    // ||z^{k+1} - z^k||^2 of this iteration, added per sample
    for (int s = c.tid; s < c.G; s += c.nthr) {
      float* blk = c.blk(s);
      float acc = 0.0f;
      for (int w = 0; w < DIM * NV; ++w) acc += blk[L.FPP + w];
      for (int w = 0; w < c.N * DIM; ++w) acc += blk[L.FPP + DIM * NV + w];
      blk[L.FPR] += acc;
    }
    // FPR is read only after the last iteration's barrier
  }
}

// FMT: MMA operand format (0 tf32, 1 bf16, 2 fp16). TRAIN: the training
// forward (checkpoints, the last segment's iterates and activity masks, the
// fixed-point residual sum), as the float32 form's.
template <int DIM, int NMAX, int MAXT, int FMT, bool TRAIN = false>
__global__ void __launch_bounds__(MAXT, 1) tm_fwd_kernel(const __grid_constant__ FusedArgs A) {
  extern __shared__ float4 smem4[];
  __shared__ TmShared ts;
  float* sm = reinterpret_cast<float*>(smem4);
  const ProblemConsts& pc = A.pc;
  const int T = pc.T;
  constexpr bool CAND = true;
  const Cta<DIM, NMAX> c(A.sc, A.n_scenes, T, A.tc, A.nq, false, sm, CAND, FMT);
  if (c.G <= 0) return;
  dbg_begin();
  const Lay& L = c.L;
  const int TC = L.TC, TCW = tm_tcw(TC);
  const int TAB = tm_tab_bytes(T, TC, FMT);
  const int ncols = tm_alloc_cols(tm_cols(DIM, TC, FMT));
  unsigned char* tabs = reinterpret_cast<unsigned char*>(sm);
  const float* gbasis = c.BASIS;   // the float32 basis, copied to shared memory by the prologue

  tm_tables<FMT>(tabs, T, TC, reinterpret_cast<const float*>(A.basis), c.tid, c.nthr);   // from global memory
  prologue<DIM, NMAX>(c, T, A.basis, A.ops, A.start, A.goal, A.start_va, A.goal_va);
  load_state<DIM, NMAX>(c, A.xi0, A.lam0, A.xi_bar, A.xi_bar);
  canary_set(c.SAMP, L.SB, c.G, A.dbg_plant);
  for (int s = c.tid; s < c.G; s += c.nthr) {
    c.blk(s)[L.FPR] = 0.0f;
    *reinterpret_cast<int*>(c.blk(s) + L.RF) = __float_as_int(INFINITY);   // the first pair test is full
  }
  if (c.warp == 0) {
    tcg::alloc(&ts.tbase, (uint32_t)ncols);
    tcg::relinquish();
  }
  if (c.tid == 0) {
    tcg::mbar_init(&ts.bar, 1);
    ts.abort = 0;
    ts.lost = 0u;
    ts.limit_ns = A.wait_ns ? A.wait_ns : kTmWaitNs;
  }
  tcg::fence_smem_to_async();
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  {
    // A from the initial coefficients (rows beyond the CTA's samples / robots zero)
    constexpr int RS = DIM * NP;
    const TmLane q = tm_lane(c, ts.tbase);
    for (int x = q.cg; x < DIM; x += q.ncg) {
      float row[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) row[k] = q.valid ? c.blk(q.s)[L.C + q.i * RS + x * NP + k] : 0.0f;
      tm_write_a<DIM, FMT>(q.lanebase, TCW, x, row);
    }
    // lanes of warps beyond the axis groups: rows of axes never written by
    // them are written by the loop above (x runs over every axis)
    tcg::wait_st();
  }
  tcg::fence_before();
  __syncthreads();
  uint32_t phase = 0u;
  const uint32_t tabs_addr = tcg::smem_u32(tabs);
  // the MMAs are issued by lane 0 of the last warp, which the pair phase
  // leaves idle or least loaded (its (sample, step) lanes come last)
  const bool issuer = c.tid == c.nthr - 32;
  if (issuer && !A.skip_first_mma) {   // (skipped only by the timeout test)
    tcg::fence_after();
    tm_issue<DIM, FMT>(ts.tbase, tabs_addr, TAB, 0, TC, &ts.bar);
  }
  // checkpoints (training): (xi, lambda) at iterations 0, ck, 2 ck, ...,
  // then every iterate of the last segment
  const bool fp = TRAIN && A.fp_res2 != nullptr;
  const int n_ck = TRAIN ? (pc.K + A.ck_every - 1) / A.ck_every : 0;
  const int last_ck = TRAIN ? (n_ck - 1) * A.ck_every : 0;
  float* tail = (TRAIN && A.ckpt) ? A.ckpt + (size_t)n_ck * 2 * A.total_coefs : nullptr;
  for (int it = 0; it < pc.K; ++it) {
    unsigned* mk = nullptr;
    if constexpr (TRAIN) {
      if (A.ckpt && it % A.ck_every == 0) write_checkpoint<DIM, NMAX>(c, A.ckpt, it / A.ck_every, A.total_coefs);
      if (tail && it >= last_ck) write_checkpoint<DIM, NMAX>(c, tail, it - last_ck, A.total_coefs);
      if (A.amask && it >= last_ck) mk = A.amask + (size_t)(it - last_ck) * A.amask_slot + c.mask0;
    }
    tm_iteration<DIM, NMAX, FMT, CAND, TRAIN>(c, pc, it, it == pc.K - 1, A.hist, A.total_samples, A.prune != 0,
                                              gbasis, ts, tabs_addr, phase, A.status, mk, fp);
    if (it + 1 < pc.K && issuer && !ts.abort) {
      tcg::fence_after();
      tm_issue<DIM, FMT>(ts.tbase, tabs_addr, TAB, 0, TC, &ts.bar);
    }
  }
  if (tail) write_checkpoint<DIM, NMAX>(c, tail, pc.K - last_ck, A.total_coefs);
  // after an abandoned wait the MMA group it waited for may still be running:
  // wait for it once more (bounded) before the columns are freed
  if (ts.abort && c.tid == 0) tcg::mbar_wait(&ts.bar, ts.lost, ts.limit_ns);
  tcg::fence_after();
  __syncthreads();
  if (c.warp == 0) tcg::dealloc(ts.tbase, (uint32_t)ncols);

  // ---- final residual, Eq. (primal_residual); robot rows beyond N of the
  // xi^{K-1} copy are zero-filled first
  constexpr int RS = DIM * NP;
  const int N = c.N, G = c.G;
  for (int v = c.tid; v < G * NMAX * RS; v += c.nthr) {
    const int s = v / (NMAX * RS), rem = v % (NMAX * RS);
    if (rem / RS >= N) c.blk(s)[L.EB + rem] = 0.0f;
  }
  __syncthreads();
  residual_phase<DIM, NMAX>(c.SAMP, L, gbasis, G, N, T, pc, c.warp, c.nwarps, c.lane);
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

template <int DIM, int NMAX, int MAXT, int FMT, bool TRAIN = false>
cudaError_t launch_tm_t(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  auto k = tm_fwd_kernel<DIM, NMAX, MAXT, FMT, TRAIN>;
  if (l.warps * 32 > MAXT || (l.warps & 3) != 0 || l.gmax * NMAX > 128) return cudaErrorInvalidConfiguration;
  k<<<l.n_ctas, l.warps * 32, l.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fused_impl
}  // namespace sf
