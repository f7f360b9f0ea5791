// Adjoint (reverse mode) of the unrolled safety-filter iterations: the
// gradient of
//   L = <gx, xi^K> + <gl, lambda^K> + sum_s w_s sum_{k<K} ||z^{k+1} - z^k||^2
// (z = (xi, lambda); the sum is the first term of Eq. (NN_loss)) with respect
// to xi^0, lambda^0 and xi_bar. The paper notes that every step of f_FP has a
// closed form, so the unroll is differentiable (Sec. III-C); this kernel
// differentiates the steps by hand.
//
// Forward step written for the adjoint (per sample):
//   q = e(F xi) - F xi,  g = F^T q,  lambda' = lambda + rho g,
//   r = rho g + lambda' + xi_bar,  xi' = Wop xi + Sop r + beta,
// with Sop = Pi_dev (x) S1 + Pi_mean (x) S0 (symmetric) and Wop = Sop rho H.
// Given (xb, lb) = dL/d(xi', lambda'):
//   r_bar = Sop^T xb;  xi_bar_grad += r_bar;  lb_total = lb + r_bar;
//   g_bar = rho (r_bar + lb_total);  dL/dlambda = lb_total;
//   dL/dxi = Wop^T xb + F^T (J_e - I)^T F g_bar,
// where J_e is the Jacobian of the alpha / beta / d closed forms: for a pair
// row with scaled distance s2 < 1, e = delta / sqrt(s2); for a ball row
// outside the ball, e = r v / ||v||; inactive rows have J_e = I; at delta = 0
// J_e is taken as 0.
//
// The CTA recomputes each segment of checkpoint_every iterations forward from
// its checkpoint into a ring in global memory, then walks the segment back.
#pragma once
#include <cstring>
#include "sf_fused_kernel.cuh"

namespace sf {
namespace fused_impl {

struct BwdArgs {
  ProblemConsts pc;
  int n_scenes;
  const float4* basis;
  const float* ops;
  const float* start;
  const float* goal;
  const float* start_va;
  const float* goal_va;
  const float* xi_bar;
  const float* ckpt;       // [n_ck][2][total_coefs]
  int ck_every;
  long long total_coefs;
  float* ring;             // [ck_every + 1][2][total_coefs]
  const unsigned* tail_mask;   // activity masks of the last segment [ck_every][mask_slot]
  unsigned* ring_mask;         // activity masks of a recomputed segment [ck_every][mask_slot]
  long long mask_slot;
  const float* g_xi;       // dL/dxi^K or null
  const float* g_lam;      // dL/dlambda^K or null
  const float* g_fp;       // per-sample weight of sum ||z^{k+1} - z^k||^2, or null
  float* gx0;              // dL/dxi^0 (or null)
  float* gl0;              // dL/dlambda^0 (or null)
  float* gxb;              // dL/dxi_bar (or null); includes the xi^0 path when xi0_is_xi_bar
  int xi0_is_xi_bar;
  int tc, nq;
  int total_samples;
  int* status;
  SceneDesc sc[MAX_SCENES_PER_LAUNCH];
};

// Pair rows of the adjoint for one chunk: Delta_bar = (J_e - I)^T (u_i - u_j)
// with u = positions of g_bar, added to E_bar_i and subtracted from E_bar_j
// in the chunk buffer. Only the rows the forward iteration recorded as active
// (activity masks, slot mk) are visited: inactive rows have J_e = I.
template <int DIM, int NMAX>
__device__ void adj_pair_phase(const Cta<DIM, NMAX>& c, const ProblemConsts& pc, int t0, int TCc,
                               const unsigned* mk) {
  constexpr int RS = DIM * NP;
  constexpr int MW = mask_words(NMAX), PW = mask_pair_words(NMAX);
  const Lay& L = c.L;
  const int N = c.N;
  const int nA = c.G * TCc;
  for (int u = c.tid; u < nA; u += c.nthr) {
    const int s = u / TCc;
    const int tl = u - s * TCc;
    const int t = t0 + tl;
    float* blk = c.blk(s);
    float* eb = blk + L.EB + tl * L.EP;
    for (int q = 0; q < N * DIM; ++q) eb[q] = 0.0f;
    const uint4* m4 = reinterpret_cast<const uint4*>(mk + ((size_t)s * L.T + t) * MW);
    unsigned w[MW];
#pragma unroll
    for (int q = 0; q < MW / 4; ++q) {
      const uint4 v = m4[q];
      w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
    }
    // workspace rows: bits 2 NMAX .. 3 NMAX - 1 after the pair words
    constexpr int WB = 2 * NMAX, WW = PW + (WB >> 5);
    unsigned long long wsm = w[WW];
    if (WW + 1 < MW) wsm |= (unsigned long long)w[(WW + 1 < MW) ? WW + 1 : WW] << 32;
    wsm = (wsm >> (WB & 31)) & ((NMAX == 64 ? 0ull : (1ull << NMAX)) - 1ull);
    if (!pc.use_w) wsm = 0ull;
    unsigned any = 0u;
#pragma unroll
    for (int q = 0; q < PW; ++q) any |= w[q];
    if (!any && !wsm) continue;
    float Pr[NV];
    row_from(c.BASIS + (size_t)t * BASIS_ROW, Pr);
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      unsigned m = w[q];
      while (m) {
        int idx = q * 32 + __ffs(m) - 1;
        m &= m - 1;
        // row-major upper triangle: row i holds NMAX - 1 - i pairs
        int i = 0;
        while (idx >= NMAX - 1 - i) {
          idx -= NMAX - 1 - i;
          ++i;
        }
        const int j = i + 1 + idx;
        float pi[DIM], pj[DIM], ui[DIM], uj[DIM];
        state<DIM>(Pr, blk + L.C + i * RS, pi);
        state<DIM>(Pr, blk + L.C + j * RS, pj);
        state<DIM>(Pr, blk + L.U + i * RS, ui);
        state<DIM>(Pr, blk + L.U + j * RS, uj);
#pragma unroll
        for (int x = 0; x < DIM; ++x) {
          pi[x] *= (x == 2 ? pc.inv_b : pc.inv_a);
          pj[x] *= (x == 2 ? pc.inv_b : pc.inv_a);
        }
        float ds[DIM];
#pragma unroll
        for (int x = 0; x < DIM; ++x) ds[x] = pi[x] - pj[x];
        float s2 = 0.0f;
#pragma unroll
        for (int x = 0; x < DIM; ++x) s2 = fmaf(ds[x], ds[x], s2);
        // delta = M ds; M^-2 delta = ds / (a, a, b)
        float U[DIM], mm[DIM], d[DIM];
        float du = 0.0f;
#pragma unroll
        for (int x = 0; x < DIM; ++x) {
          const float ax = x == 2 ? pc.coll_b : pc.coll_a;
          d[x] = ds[x] * ax;
          mm[x] = ds[x] / ax;
          U[x] = ui[x] - uj[x];
          du = fmaf(d[x], U[x], du);
        }
        const bool zero = (s2 == 0.0f);
        const float inv = rsqrtf(zero ? 1.0f : s2);
        const float f = zero ? -1.0f : inv - 1.0f;
        const float wgt = zero ? 0.0f : inv * inv * inv * du;
#pragma unroll
        for (int x = 0; x < DIM; ++x) {
          const float db = fmaf(f, U[x], -wgt * mm[x]);
          eb[i * DIM + x] += db;
          eb[j * DIM + x] -= db;
        }
      }
    }
    // workspace rows outside the spheroid: e = p_w + D / sqrt(s2) with
    // D = p - p_w, s2 = ||M_w^-1 D||^2; (J_e - I)^T u = (s2^-1/2 - 1) u -
    // s2^-3/2 (D . u) M_w^-2 D, added to E_bar of the robot
    while (wsm) {
      const int i = __ffsll((long long)wsm) - 1;
      wsm &= wsm - 1ull;
      float pi[DIM], ui[DIM];
      state<DIM>(Pr, blk + L.C + i * RS, pi);
      state<DIM>(Pr, blk + L.U + i * RS, ui);
      float d[DIM], mm[DIM], s2 = 0.0f, du = 0.0f;
#pragma unroll
      for (int x = 0; x < DIM; ++x) {
        d[x] = pi[x] - pc.wc[x];
        mm[x] = d[x] * pc.winv[x] * pc.winv[x];
        s2 = fmaf(d[x], mm[x], s2);
        du = fmaf(d[x], ui[x], du);
      }
      const float inv = rsqrtf(s2);
      const float f = inv - 1.0f, wgt = inv * inv * inv * du;
#pragma unroll
      for (int x = 0; x < DIM; ++x) eb[i * DIM + x] += fmaf(f, ui[x], -wgt * mm[x]);
    }
  }
}

// Ball rows and the transposed contraction of the adjoint for one chunk:
// dL/dxi += F^T Delta_bar, per (sample, robot, range of t), into PG partials.
template <int DIM, int NMAX>
__device__ void adj_contract_phase(const Cta<DIM, NMAX>& c, const ProblemConsts& pc, int t0, int TCc,
                                   bool first_chunk, const unsigned* mk) {
  constexpr int MW = mask_words(NMAX), PW = mask_pair_words(NMAX);
  constexpr int RS = DIM * NP;
  const Lay& L = c.L;
  const int N = c.N, G = c.G, NQ = L.NQ;
  const int nB = NQ * G * N;
  const int TQ = (TCc + NQ - 1) / NQ;
  for (int base = c.warp * 32; base < nB; base += c.nwarps * 32) {
    const int u = base + c.lane;
    const bool uvalid = u < nB;
    const int uu = uvalid ? u : 0;
    const int i = uu % N;
    const int s = (uu / N) % G;
    const int tq = uu / (N * G);
    const int ta = tq * TQ;
    const int tb = uvalid ? min(ta + TQ, TCc) : ta;
    float* blk = c.blk(s);
    float cc[DIM][NV], gb[DIM][NV], g2[DIM][NV];
#pragma unroll
    for (int x = 0; x < DIM; ++x) {
      row_from(blk + L.C + i * RS + x * NP, cc[x]);
      row_from(blk + L.U + i * RS + x * NP, gb[x]);
#pragma unroll
      for (int k = 0; k < NV; ++k) g2[x][k] = 0.0f;
    }
    // uniform trip count over the warp so that the votes see every lane
    int trip = tb - ta;
    int wtrip = trip;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) wtrip = max(wtrip, __shfl_xor_sync(FULL, wtrip, o));
    for (int step = 0; step < wtrip; ++step) {
      const bool live = step < trip;
      const int tl = live ? ta + step : ta;
      const float* brow = c.BASIS + (size_t)(t0 + tl) * BASIS_ROW;
      float e[DIM], vb[DIM], ab[DIM];
      const float* ebp = blk + L.EB + tl * L.EP + i * DIM;
#pragma unroll
      for (int x = 0; x < DIM; ++x) { e[x] = live ? ebp[x] : 0.0f; vb[x] = 0.0f; ab[x] = 0.0f; }
      // ball rows outside their ball in the forward iteration (activity masks)
      bool vact = false, aact = false;
      if (live) {
        const unsigned* mb = mk + ((size_t)s * L.T + t0 + tl) * MW + PW;
        vact = (mb[i >> 5] >> (i & 31)) & 1u;
        aact = (mb[(NMAX + i) >> 5] >> ((NMAX + i) & 31)) & 1u;
      }
      if (pc.use_v && __any_sync(FULL, vact)) {
        float Pd[NV];
        row_from(brow + NP, Pd);
        float v[DIM], n2 = 0.0f;
#pragma unroll
        for (int x = 0; x < DIM; ++x) { v[x] = dot_reg(Pd, cc[x]); n2 = fmaf(v[x], v[x], n2); }
        const bool act = vact;
        {
          float U[DIM], du = 0.0f;
#pragma unroll
          for (int x = 0; x < DIM; ++x) { U[x] = dot_reg(Pd, gb[x]); du = fmaf(v[x], U[x], du); }
          const float inv = rsqrtf(act ? n2 : 1.0f);
          const float rr = pc.v_max * inv;
#pragma unroll
          for (int x = 0; x < DIM; ++x) vb[x] = act ? fmaf(rr - 1.0f, U[x], -rr * inv * inv * du * v[x]) : 0.0f;
        }
      }
      if (pc.use_a && __any_sync(FULL, aact)) {
        float Pdd[NV];
        row_from(brow + 2 * NP, Pdd);
        float a[DIM], n2 = 0.0f;
#pragma unroll
        for (int x = 0; x < DIM; ++x) { a[x] = dot_reg(Pdd, cc[x]); n2 = fmaf(a[x], a[x], n2); }
        const bool act = aact;
        {
          float U[DIM], du = 0.0f;
#pragma unroll
          for (int x = 0; x < DIM; ++x) { U[x] = dot_reg(Pdd, gb[x]); du = fmaf(a[x], U[x], du); }
          const float inv = rsqrtf(act ? n2 : 1.0f);
          const float rr = pc.a_max * inv;
#pragma unroll
          for (int x = 0; x < DIM; ++x) ab[x] = act ? fmaf(rr - 1.0f, U[x], -rr * inv * inv * du * a[x]) : 0.0f;
        }
      }
      bool ne = false, nb = false;
#pragma unroll
      for (int x = 0; x < DIM; ++x) {
        ne |= e[x] != 0.0f;
        nb |= (vb[x] != 0.0f) || (ab[x] != 0.0f);
      }
      if (__any_sync(FULL, ne)) {
        float P[NV];
        row_from(brow, P);
#pragma unroll
        for (int x = 0; x < DIM; ++x)
#pragma unroll
          for (int k = 0; k < NV; ++k) g2[x][k] = fmaf(P[k], e[x], g2[x][k]);
      }
      if (__any_sync(FULL, nb)) {
        float Pd[NV], Pdd[NV];
        row_from(brow + NP, Pd);
        row_from(brow + 2 * NP, Pdd);
#pragma unroll
        for (int x = 0; x < DIM; ++x)
#pragma unroll
          for (int k = 0; k < NV; ++k) g2[x][k] = fmaf(Pd[k], vb[x], fmaf(Pdd[k], ab[x], g2[x][k]));
      }
    }
    if (uvalid) {
      float* pg = blk + L.PG + tq * NMAX * RS + i * RS;
#pragma unroll
      for (int x = 0; x < DIM; ++x)
#pragma unroll
        for (int k = 0; k < NV; ++k) pg[x * NP + k] = first_chunk ? g2[x][k] : pg[x * NP + k] + g2[x][k];
    }
  }
}

// Ring slot j holds (xi^{kb+j}, lambda^{kb+j}) in the checkpoint layout.
__device__ __forceinline__ const float* ring_xi(const float* ring, int j, long long tot) {
  return ring + (size_t)j * 2 * tot;
}
__device__ __forceinline__ const float* ring_lam(const float* ring, int j, long long tot) {
  return ring + (size_t)j * 2 * tot + tot;
}

// Adjoint of iteration k (z^k -> z^{k+1}); XB, LB hold dL/dz^{k+1} on entry
// and dL/dz^k on exit.
template <int DIM, int NMAX>
__device__ void adjoint_step(const Cta<DIM, NMAX>& c, const BwdArgs& A, const float* ring, int j,
                             const unsigned* mslot) {
  constexpr int RS = DIM * NP;
  const Lay& L = c.L;
  const ProblemConsts& pc = A.pc;
  const int N = c.N, G = c.G, T = pc.T;
  const long long tot = A.total_coefs;
  const float rho = pc.rho;
  const float invN = 1.0f / (float)N;
  const float* xk = ring_xi(ring, j, tot);
  const float* xk1 = ring_xi(ring, j + 1, tot);
  const float* lk = ring_lam(ring, j, tot);
  const float* lk1 = ring_lam(ring, j + 1, tot);
  // (0) xi^k into C; fixed-point-residual term with respect to z^{k+1}
  for (int v = c.tid; v < G * NMAX * RS; v += c.nthr) {
    const int s = v / (NMAX * RS), rem = v % (NMAX * RS);
    const int i = rem / RS, x = (rem / NP) % DIM, k = rem % NP;
    float* blk = c.blk(s);
    float val = 0.0f;
    if (i < N && k < NV) {
      const long long g = c.gidx(s, x, i, k);
      val = xk[g];
      if (A.g_fp) {
        const float w2 = 2.0f * A.g_fp[c.gsample0 + s];
        blk[L.XB + rem] = fmaf(w2, xk1[g] - val, blk[L.XB + rem]);
        blk[L.LB + rem] = fmaf(w2, lk1[g] - lk[g], blk[L.LB + rem]);
      }
    }
    blk[L.C + rem] = val;
  }
  __syncthreads();
  // (1) robot mean of xb, and the mean terms of the transposed xi step:
  // MC = DS^T mean(xb), MR = DW^T mean(xb). Lanes (s, x, k) with k padded to
  // 16, so that the 11 k of one (s, x) share a half-warp and exchange their
  // means by shuffles.
  {
    const int nB1 = G * DIM * 16;
    const int lane = c.lane;
    for (int base = c.tid - lane; base < nB1; base += c.nthr) {
      const int v = base + lane;
      const int vq = v < nB1 ? v : 0;
      const int s = vq / (DIM * 16), x = (vq >> 4) % DIM, k = vq & 15;
      const bool act = v < nB1 && k < NV;
      float* blk = c.blk(s);
      float sm = 0.0f;
      if (act)
        for (int i = 0; i < N; ++i) sm += blk[L.XB + i * RS + x * NP + k];
      const float mx = sm * invN;
      const int kk = k < NV ? k : 0;
      float md = 0.0f, mw = 0.0f;
#pragma unroll
      for (int m = 0; m < NV; ++m) {
        const float xm = __shfl_sync(FULL, mx, (lane & 16) + m);
        md = fmaf(c.OPS[OPS_DS + m * NP + kk], xm, md);
        mw = fmaf(c.OPS[OPS_DW + m * NP + kk], xm, mw);
      }
      if (act) {
        blk[L.MC + x * NP + k] = md;
        blk[L.MR + x * NP + k] = mw;
      }
    }
  }
  __syncthreads();
  // (2) coefficient-space adjoint of the xi step and the lambda step
  for (int v = c.tid; v < G * N * DIM; v += c.nthr) {
    const int s = v / (N * DIM), i = (v / DIM) % N, x = v % DIM;
    float* blk = c.blk(s);
    const int o = i * RS + x * NP;
    float xb[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) xb[k] = blk[L.XB + o + k];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float u1 = blk[L.MC + x * NP + k], cw = blk[L.MR + x * NP + k];
#pragma unroll
      for (int m = 0; m < NV; ++m) {
        u1 = fmaf(c.OPS[OPS_S1 + m * NP + k], xb[m], u1);
        cw = fmaf(c.OPS[OPS_W1 + m * NP + k], xb[m], cw);
      }
      const float lt = blk[L.LB + o + k] + u1;
      blk[L.U + o + k] = rho * (u1 + lt);
      blk[L.GXB + o + k] += u1;
      blk[L.LB + o + k] = lt;
      blk[L.CW + o + k] = cw;
    }
  }
  __syncthreads();
  // (3) time-domain adjoint of the alpha / beta / d steps, in chunks
  for (int t0 = 0; t0 < T; t0 += L.TC) {
    const int TCc = min(L.TC, T - t0);
    adj_pair_phase<DIM, NMAX>(c, pc, t0, TCc, mslot + c.mask0);
    __syncthreads();
    adj_contract_phase<DIM, NMAX>(c, pc, t0, TCc, t0 == 0, mslot + c.mask0);
    __syncthreads();
  }
  // (4) dL/dxi^k = Wop^T xb + F^T Delta_bar; fixed-point term w.r.t. z^k
  for (int v = c.tid; v < G * NMAX * RS; v += c.nthr) {
    const int s = v / (NMAX * RS), rem = v % (NMAX * RS);
    const int i = rem / RS, x = (rem / NP) % DIM, k = rem % NP;
    if (i >= N || k >= NV) continue;
    float* blk = c.blk(s);
    float val = blk[L.CW + rem];
    for (int q = 0; q < L.NQ; ++q) val += blk[L.PG + q * NMAX * RS + rem];
    if (A.g_fp) {
      const long long g = c.gidx(s, x, i, k);
      const float w2 = 2.0f * A.g_fp[c.gsample0 + s];
      val = fmaf(-w2, xk1[g] - xk[g], val);
      blk[L.LB + rem] = fmaf(-w2, lk1[g] - lk[g], blk[L.LB + rem]);
    }
    blk[L.XB + rem] = val;
  }
  __syncthreads();
}

template <int DIM, int NMAX, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) fused_bwd_kernel(const __grid_constant__ BwdArgs A) {
  constexpr int RS = DIM * NP;
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const ProblemConsts& pc = A.pc;
  const int T = pc.T, K = pc.K;
  const Cta<DIM, NMAX> c(A.sc, A.n_scenes, T, A.tc, A.nq, true, sm);
  if (c.G <= 0) return;
  const Lay& L = c.L;
  const int N = c.N, G = c.G;
  const long long tot = A.total_coefs;
  dbg_begin();
  prologue<DIM, NMAX>(c, T, A.basis, A.ops, A.start, A.goal, A.start_va, A.goal_va);
  canary_set(c.SAMP, L.SB, G, 0);
  for (int v = c.tid; v < G * NMAX * RS; v += c.nthr) {
    const int s = v / (NMAX * RS), rem = v % (NMAX * RS);
    const int i = rem / RS, x = (rem / NP) % DIM, k = rem % NP;
    float* blk = c.blk(s);
    float xb = 0.0f, lb = 0.0f;
    if (i < N && k < NV) {
      const long long g = c.gidx(s, x, i, k);
      xb = A.g_xi ? A.g_xi[g] : 0.0f;
      lb = A.g_lam ? A.g_lam[g] : 0.0f;
    }
    blk[L.XB + rem] = xb;
    blk[L.LB + rem] = lb;
    blk[L.GXB + rem] = 0.0f;
    blk[L.U + rem] = 0.0f;
    blk[L.CW + rem] = 0.0f;
  }
  __syncthreads();
  const int ck = A.ck_every;
  const int nseg = (K + ck - 1) / ck;
  float* ring = A.ring;
  // the forward stored every iterate of the last segment after the
  // checkpoints; earlier segments are recomputed into the workspace ring
  const float* tail = A.ckpt + (size_t)nseg * 2 * tot;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int kb = seg * ck, ke = min(K, kb + ck);
    const float* rg = ring;
    const unsigned* mg = A.ring_mask;
    if (seg == nseg - 1) {
      rg = tail;
      mg = A.tail_mask;
    } else {
      const float* cx = A.ckpt + (size_t)seg * 2 * tot;
      load_state<DIM, NMAX>(c, cx, cx + tot, nullptr, A.xi_bar);
      __syncthreads();
      store_state<DIM, NMAX>(c, ring, ring + tot, 0);
      for (int k = kb; k < ke; ++k) {
        fwd_iteration<DIM, NMAX, true>(c, pc, A.xi_bar, k, false, nullptr, 0, false,
                                          A.ring_mask + (size_t)(k - kb) * A.mask_slot);
        float* slot = ring + (size_t)(k - kb + 1) * 2 * tot;
        store_state<DIM, NMAX>(c, slot, slot + tot, 0);
      }
    }
    __syncthreads();
    for (int k = ke - 1; k >= kb; --k)
      adjoint_step<DIM, NMAX>(c, A, rg, k - kb, mg + (size_t)(k - kb) * A.mask_slot);
  }
  for (int v = c.tid; v < G * DIM * N * NV; v += c.nthr) {
    const int s = v / (DIM * N * NV), rem = v % (DIM * N * NV);
    const int x = rem / (N * NV), i = (rem / NV) % N, k = rem % NV;
    const float* blk = c.blk(s);
    const int o = i * RS + x * NP + k;
    const long long g = c.coef0 + (long long)s * c.per_sample + rem;
    if (A.gx0) A.gx0[g] = blk[L.XB + o];
    if (A.gl0) A.gl0[g] = blk[L.LB + o];
    if (A.gxb) A.gxb[g] = blk[L.GXB + o] + (A.xi0_is_xi_bar ? blk[L.XB + o] : 0.0f);
  }
  canary_check(c.SAMP, L.SB, G);
  dbg_end(A.status);
}

template <int DIM, int NMAX, int MAXT>
cudaError_t launch_bwd_t(const BwdArgs& a, int n_ctas, int warps, size_t smem, cudaStream_t st) {
  auto k = fused_bwd_kernel<DIM, NMAX, MAXT>;
  if (warps * 32 > MAXT) return cudaErrorInvalidConfiguration;
  k<<<n_ctas, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

// Kernel parameters of the adjoint from the forward's scene table and
// problem constants plus the backward's own buffers and launch shape.
inline BwdArgs make_bwd_args(const FusedArgs& a, const BwdLaunchArgs& b, const FusedLaunch& l) {
  BwdArgs x;
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
  return x;
}

// Adjoint of one (dim, robot-count bucket): BwdArgs from the forward's
// arguments, then the launch.
template <int DIM, int NMAX, int MAXT>
cudaError_t launch_bwd_from(const FusedArgs& a, const BwdLaunchArgs& b, const FusedLaunch& l, cudaStream_t st) {
  return launch_bwd_t<DIM, NMAX, MAXT>(make_bwd_args(a, b, l), l.n_ctas, l.warps, l.smem, st);
}

}  // namespace fused_impl
}  // namespace sf
