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

// Polls of an mbarrier before a wait is abandoned (a completed MMA group
// takes a few microseconds; the limit is far above that).
constexpr uint32_t kTmWaitLimit = 1u << 22;

// Shared state of the tensor-memory form (static shared memory).
struct TmShared {
  uint64_t bar;       // MMA completion of the current chunk
  uint32_t tbase;     // TMEM base address
  int abort;          // a wait ran out: no more MMAs, outputs flagged
};

template <int FMT>
__device__ __forceinline__ uint32_t pack16(float lo, float hi) {
  return tc::pack2<FMT>(lo, hi);
}

// B tables: Pd and Pdd rows (m = 1, 2) of the float32 basis [T][36]
// (global), rounded (table 2 (m - 1)) and the rounding remainder (table
// 2 (m - 1) + 1), time step t of chunk c at row c * TCW + (t - c TC); every
// other entry zero.
template <int FMT>
__device__ void tm_tables(unsigned char* tb, int T, int TC, const float* gb, int tid, int nthr) {
  const int TCW = tm_tcw(TC);
  const int TAB = tm_tab_bytes(T, TC, FMT);
  uint32_t* w = reinterpret_cast<uint32_t*>(tb);
  for (int v = tid; v < TM_TABLES * TAB / 4; v += nthr) w[v] = 0u;
  __syncthreads();
  constexpr uint32_t SBO = tm_sbo(FMT);
  if constexpr (FMT == 0) {
    for (int v = tid; v < T * 2 * 12; v += nthr) {
      const int t = v / 24, m = (v / 12) % 2, k = v % 12;
      const float x = gb[(size_t)t * BASIS_ROW + (1 + m) * NP + k];
      const int ci = t / TC, row = ci * TCW + (t - ci * TC);
      const uint32_t off = (row >> 3) * SBO + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
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
      const int ci = t / TC, row = ci * TCW + (t - ci * TC);
      const uint32_t off = (row >> 3) * SBO + (k0 >> 3) * 128 + (row & 7) * 16 + (k0 & 7) * 2;
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

// Issues the MMAs of chunk ci (velocities and accelerations of every row and
// axis) and commits them to the mbarrier. One thread.
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
    if (!tcg::mbar_wait(&ts.bar, phase, kTmWaitLimit)) {
      ts.abort = 1;
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

// TMEM pass of one chunk (after its pair phase): the velocity / acceleration
// ball rows of this lane's robot from TMEM, F^T of their residuals and of the
// pair residuals E (chunk-buffer rows, skipped where the row's active-pair
// flag is clear on every lane of the warp) into g, the balls' squared
// residuals into rb.
template <int DIM, int NMAX>
__device__ void tm_chunk_pass(const Cta<DIM, NMAX>& c, const TmLane& q, const ProblemConsts& pc, int t0, int TCc,
                              int TCW, const float* gbasis, float (&g)[DIM][NV], float& rb) {
  const Lay& L = c.L;
  const float* blk = c.blk(q.valid ? q.s : 0);
  const float vm2 = pc.v_max * pc.v_max, am2 = pc.a_max * pc.a_max;
  for (int bk = q.cg; bk * 8 < TCc; bk += q.ncg) {
    const int tb = bk * 8;
    uint32_t v[DIM][8], a[DIM][8];
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      tcg::ld8(q.lanebase + (uint32_t)(x * TCW + tb), v[x]);
      tcg::ld8(q.lanebase + (uint32_t)((DIM + x) * TCW + tb), a[x]);
    }
    tcg::wait_ld();
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      tcg::tie(v[x]);
      tcg::tie(a[x]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int tl = tb + j;
      if (tl >= TCc) break;   // warp-uniform
      const bool live = q.valid;
      const float* brow = gbasis + (size_t)(t0 + tl) * BASIS_ROW;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        if (b == 0 ? !pc.use_v : !pc.use_a) continue;
        float w[DIM], n2 = 0.0f;
#pragma unroll
        for (int x = 0; x < DIM; ++x) {
          w[x] = live ? __uint_as_float(b == 0 ? v[x][j] : a[x][j]) : 0.0f;
          n2 = fmaf(w[x], w[x], n2);
        }
        const bool out = n2 > (b == 0 ? vm2 : am2);
        if (__any_sync(FULL, out)) {
          float qb[DIM], rl = 0.0f;
          ball_residual<DIM>(w, b == 0 ? pc.v_max : pc.a_max, qb, rl);
          rb += rl;
          float P[NV];
          row_from(brow + (1 + b) * NP, P);
#pragma unroll
          for (int x = 0; x < DIM; ++x)
#pragma unroll
            for (int k = 0; k < NV; ++k) g[x][k] = fmaf(P[k], qb[x], g[x][k]);
        }
      }
      const float* eb = blk + L.EB + tl * L.EP;
      const bool act = live && eb[NMAX * DIM] != 0.0f;
      if (__any_sync(FULL, act)) {
        float e[DIM];
#pragma unroll
        for (int x = 0; x < DIM; ++x) e[x] = act ? eb[q.i * DIM + x] : 0.0f;
        float P[NV];
        row_from(brow, P);
#pragma unroll
        for (int x = 0; x < DIM; ++x)
#pragma unroll
          for (int k = 0; k < NV; ++k) g[x][k] = fmaf(P[k], e[x], g[x][k]);
      }
    }
  }
}

// One iteration of f_FP in the tensor-memory form (the MMAs of chunk 0 are in
// flight on entry). Ends with the xi step, which rewrites A in TMEM.
template <int DIM, int NMAX, int FMT, bool CAND>
__device__ void tm_iteration(const Cta<DIM, NMAX>& c, const ProblemConsts& pc, int it, bool keep_prev, float* hist,
                             int total_samples, bool prune, const float* gbasis, TmShared& ts, uint32_t tabs,
                             uint32_t& phase, int* status) {
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
  for (int ci = 0; ci < nch; ++ci) {
    const int t0 = ci * TC, TCc = min(TC, T - t0);
    pair_phase<DIM, NMAX, false, false, CAND, true>(c.SAMP, L, gbasis, c.G, c.N, t0, TCc, pc, want_res, c.warp,
                                                    c.nwarps, c.lane, nullptr, prune);
    __syncthreads();
    tm_wait(ts, phase, status);
    tm_chunk_pass<DIM, NMAX>(c, q, pc, t0, TCc, TCW, gbasis, g, rb);
    tcg::fence_before();
    __syncthreads();
    if (c.tid == 0 && ci + 1 < nch && !ts.abort) {
      tcg::fence_after();
      tm_issue<DIM, FMT>(ts.tbase, tabs, TAB, ci + 1, TC, &ts.bar);
    }
  }
  if (q.valid) {
    float* blk = c.blk(q.s);
    float* pg = blk + L.PG + q.cg * NMAX * RS + q.i * RS;
#pragma unroll
    for (int x = 0; x < DIM; ++x)
#pragma unroll
      for (int k = 0; k < NV; ++k) pg[x * NP + k] = g[x][k];
    if (want_res) blk[L.RSB + q.cg * NMAX + q.i] = rb;
  }
  __syncthreads();
  solve_lambda_means<DIM, NMAX, CAND>(c, pc, it, hist, total_samples, false);
  __syncthreads();
  // xi step, one (sample, robot) row per lane and the axes over the warp
  // groups; the new rows also go to A in TMEM
  for (int x = q.cg; x < DIM; x += q.ncg) {
    float out[NP];
    if (q.valid) {
      xi_step_row<DIM, NMAX, CAND>(c, pc, q.s, q.i, x, keep_prev, false, out);
    } else {
#pragma unroll
      for (int k = 0; k < NP; ++k) out[k] = 0.0f;
    }
    tm_write_a<DIM, FMT>(q.lanebase, TCW, x, out);
  }
  tcg::wait_st();
  tcg::fence_before();
  __syncthreads();
}

// FMT: MMA operand format (0 tf32, 1 bf16, 2 fp16). Forward only (no
// checkpoints, no activity masks).
template <int DIM, int NMAX, int MAXT, int FMT>
__global__ void __launch_bounds__(MAXT, 1) tm_fwd_kernel(const __grid_constant__ FusedArgs A) {
  extern __shared__ float4 smem4[];
  __shared__ TmShared ts;
  float* sm = reinterpret_cast<float*>(smem4);
  const ProblemConsts& pc = A.pc;
  const int T = pc.T;
  constexpr bool CAND = true;
  const Cta<DIM, NMAX> c(A.sc, A.n_scenes, T, A.tc, A.nq, false, sm, false, CAND, FMT);
  if (c.G <= 0) return;
  const Lay& L = c.L;
  const int TC = L.TC, TCW = tm_tcw(TC);
  const int TAB = tm_tab_bytes(T, TC, FMT);
  const int ncols = tm_alloc_cols(tm_cols(DIM, TC, FMT));
  unsigned char* tabs = reinterpret_cast<unsigned char*>(sm);
  const float* gbasis = reinterpret_cast<const float*>(A.basis);

  tm_tables<FMT>(tabs, T, TC, gbasis, c.tid, c.nthr);
  prologue<DIM, NMAX, 3>(c, T, A.basis, A.ops, A.start, A.goal, A.start_va, A.goal_va);
  load_state<DIM, NMAX>(c, A.xi0, A.lam0, A.xi_bar, A.xi_bar);
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
  if (c.tid == 0) {
    tcg::fence_after();
    tm_issue<DIM, FMT>(ts.tbase, tabs_addr, TAB, 0, TC, &ts.bar);
  }
  for (int it = 0; it < pc.K; ++it) {
    tm_iteration<DIM, NMAX, FMT, CAND>(c, pc, it, it == pc.K - 1, A.hist, A.total_samples, A.prune != 0, gbasis, ts,
                                       tabs_addr, phase, A.status);
    if (it + 1 < pc.K && c.tid == 0 && !ts.abort) {
      tcg::fence_after();
      tm_issue<DIM, FMT>(ts.tbase, tabs_addr, TAB, 0, TC, &ts.bar);
    }
  }
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
    if (!isfinite(r)) atomicOr(A.status, ST_NONFINITE);
  }
  store_state<DIM, NMAX>(c, A.xi_out, A.lam_out, 0);
}

template <int DIM, int NMAX, int MAXT, int FMT>
cudaError_t launch_tm_t(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  auto k = tm_fwd_kernel<DIM, NMAX, MAXT, FMT>;
  if (l.warps * 32 > MAXT || (l.warps & 3) != 0 || l.gmax * NMAX > 128) return cudaErrorInvalidConfiguration;
  k<<<l.n_ctas, l.warps * 32, l.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fused_impl
}  // namespace sf
