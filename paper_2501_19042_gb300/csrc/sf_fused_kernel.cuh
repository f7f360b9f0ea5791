// Fused forward of the safety filter: one launch runs all K iterations of
// f_FP (Appendix, AM steps) for many samples, with every sample's
// coefficient-space state (xi, lambda, xi_bar) resident in shared memory.
//
// CTA = G samples of one scene. Per iteration:
//  * time phase, one warp per (sample, block of 32 time steps), lane = t:
//      positions p_i(t) = P[t] c_i for all robots (recomputed from the
//      resident coefficients, never stored), every pair (i < j) projected by
//      the alpha / beta / d closed forms, q = e - delta accumulated per robot
//      in registers (E_i += q, E_j -= q, blocks of 8 robots); then per robot
//      the velocity / acceleration ball projections and the transposed
//      contraction  g_i = sum_t P[t] E_i(t) + Pd[t] qv_i(t) + Pdd[t] qa_i(t)
//      (F^T of the residual, Eq. lambda_step), reduced over the 32 lanes by a
//      shuffle reduce-scatter and written per time block;
//  * solve phase: lambda' = lambda + rho g  (lambda step, minus-sign reading),
//      r = rho g + lambda' + xi_bar, robot means, and the xi step
//      c_i' = W1 c_i + S1 r_i + DW cbar + DS rbar + beta_i with the
//      pre-stored operators of the KKT system.
// After the last iteration one more time pass evaluates
//   ||r_p|| = ||F xi^K - e(xi^{K-1})||  (Eq. primal_residual)
// as  F(xi^K - xi^{K-1}) - q(xi^{K-1})  per row.
#pragma once
#include "sf_internal.cuh"

namespace sf {
namespace fused_impl {

constexpr unsigned FULL = 0xffffffffu;

template <int DIM, int NMAX>
struct Layout {
  static constexpr int RS = DIM * NP;  // floats per robot row [ax][12]
  int TB;                              // time blocks of 32
  int SB;                              // floats per sample block
  __host__ __device__ Layout(int T) {
    TB = (T + 31) / 32;
    SB = (4 + TB) * NMAX * RS + 2 * DIM * NP + ((TB + 3) / 4) * 4;
  }
  // offsets inside a sample block
  __host__ __device__ int C() const { return 0; }
  __host__ __device__ int LAM() const { return NMAX * RS; }
  __host__ __device__ int XIB() const { return 2 * NMAX * RS; }
  __host__ __device__ int CPREV() const { return 3 * NMAX * RS; }
  __host__ __device__ int GP(int tb) const { return (4 + tb) * NMAX * RS; }
  __host__ __device__ int MC() const { return (4 + TB) * NMAX * RS; }
  __host__ __device__ int MR() const { return (4 + TB) * NMAX * RS + DIM * NP; }
  __host__ __device__ int RESP() const { return (4 + TB) * NMAX * RS + 2 * DIM * NP; }
  static constexpr int head_floats() { return 4 * NV * NP + NMAX * RS; }  // OPS + BETA
};

__device__ __forceinline__ void load_row(const float4* __restrict__ basis, int t, int which, bool valid,
                                         float (&r)[NV]) {
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a;
  if (valid) {
    const float4* p = basis + (size_t)t * 9 + which * 3;
    a = __ldg(p);
    b = __ldg(p + 1);
    c = __ldg(p + 2);
  }
  r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
  r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
  r[8] = c.x; r[9] = c.y; r[10] = c.z;
}

// dot of a basis row with one 12-float coefficient row in shared memory
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

template <int DIM>
__device__ __forceinline__ void state(const float (&r)[NV], const float* Crow, float (&p)[DIM]) {
#pragma unroll
  for (int x = 0; x < DIM; ++x) p[x] = dot_row(r, Crow + x * NP);
}

template <int DIM>
__device__ __forceinline__ void state_diff(const float (&r)[NV], const float* Crow, const float* Prow,
                                           float (&p)[DIM]) {
#pragma unroll
  for (int x = 0; x < DIM; ++x) p[x] = dot_row(r, Crow + x * NP) - dot_row(r, Prow + x * NP);
}

// Reduce-scatter over the 32 lanes: afterwards v[0] on lane l holds the sum
// over all lanes of the input v[l].
__device__ __forceinline__ void reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int n = 16; n >= 1; n >>= 1) {
    const bool up = (lane & n) != 0;
#pragma unroll
    for (int j = 0; j < n; ++j) {
      const float send = up ? v[j] : v[j + n];
      const float keep = up ? v[j + n] : v[j];
      v[j] = keep + __shfl_xor_sync(FULL, send, n);
    }
  }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

// One (sample, time block) unit of an iteration. Writes this block's part of
// g = F^T (e - F xi) to GP ([NMAX][DIM][NP]) and its squared projection
// residual to *resp.
template <int DIM, int NMAX>
__device__ void time_unit(const float* __restrict__ C, const float4* __restrict__ basis, int T, int t,
                          int N, const ProblemConsts& pc, float* __restrict__ GP, float* resp, int lane) {
  constexpr int RS = DIM * NP;
  const bool valid = t < T;
  float Pr[NV];
  load_row(basis, t, 0, valid, Pr);
  float E[NMAX][DIM];
#pragma unroll
  for (int i = 0; i < NMAX; ++i)
#pragma unroll
    for (int x = 0; x < DIM; ++x) E[i][x] = 0.0f;
  float res2 = 0.0f;

  // all pairs (i < j), robots in blocks of 8: positions of the block in
  // registers, the later robots one at a time
#pragma unroll
  for (int I0 = 0; I0 < NMAX; I0 += 8) {
    if (I0 < N) {
      float pI[8][DIM];
#pragma unroll
      for (int a = 0; a < 8; ++a) state<DIM>(Pr, C + (I0 + a) * RS, pI[a]);
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = a + 1; b < 8; ++b) {
          if (I0 + b < N) {
            float q[DIM];
            pair_residual<DIM>(pI[a], pI[b], q, pc, res2);
#pragma unroll
            for (int x = 0; x < DIM; ++x) { E[I0 + a][x] += q[x]; E[I0 + b][x] -= q[x]; }
          }
        }
#pragma unroll
      for (int j = I0 + 8; j < NMAX; ++j) {
        if (j < N) {
          float pj[DIM];
          state<DIM>(Pr, C + j * RS, pj);
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            float q[DIM];
            pair_residual<DIM>(pI[a], pj, q, pc, res2);
#pragma unroll
            for (int x = 0; x < DIM; ++x) { E[I0 + a][x] += q[x]; E[j][x] -= q[x]; }
          }
        }
      }
    }
  }

  float Pd[NV], Pdd[NV];
  load_row(basis, t, 1, valid, Pd);
  load_row(basis, t, 2, valid, Pdd);
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
    if (i < N) {
      float qv[DIM], qa[DIM];
#pragma unroll
      for (int x = 0; x < DIM; ++x) { qv[x] = 0.0f; qa[x] = 0.0f; }
      if (pc.use_v) {
        float v[DIM];
        state<DIM>(Pd, C + i * RS, v);
        ball_residual<DIM>(v, pc.v_max, qv, res2);
      }
      if (pc.use_a) {
        float a[DIM];
        state<DIM>(Pdd, C + i * RS, a);
        ball_residual<DIM>(a, pc.a_max, qa, res2);
      }
      float h[32];
      float hlast = 0.0f;
#pragma unroll
      for (int x = 0; x < DIM; ++x)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const float val = fmaf(Pr[k], E[i][x], fmaf(Pd[k], qv[x], Pdd[k] * qa[x]));
          const int idx = x * NV + k;
          if (idx < 32) h[idx] = val; else hlast = val;
        }
#pragma unroll
      for (int idx = DIM * NV; idx < 32; ++idx) h[idx] = 0.0f;
      reduce_scatter32(h, lane);
      float* g = GP + i * RS;
      if (lane < DIM * NV && lane < 32) g[(lane / NV) * NP + lane % NV] = h[0];
      if (DIM * NV > 32) {
        hlast = warp_sum(hlast);
        if (lane == 0) g[(32 / NV) * NP + 32 % NV] = hlast;
      }
    }
  }
  res2 = valid ? res2 : 0.0f;
  res2 = warp_sum(res2);
  if (lane == 0) *resp = res2;
}

// Residual pass after the last iteration: ||F xi^K - e(xi^{K-1})||^2 of this
// unit, row by row as (F (xi^K - xi^{K-1}))_row - q_row(xi^{K-1}).
template <int DIM, int NMAX>
__device__ void residual_unit(const float* __restrict__ C, const float* __restrict__ Cp,
                              const float4* __restrict__ basis, int T, int t, int N,
                              const ProblemConsts& pc, float* resp) {
  constexpr int RS = DIM * NP;
  const bool valid = t < T;
  float Pr[NV];
  load_row(basis, t, 0, valid, Pr);
  float r2 = 0.0f, dummy = 0.0f;
#pragma unroll
  for (int I0 = 0; I0 < NMAX; I0 += 8) {
    if (I0 < N) {
      float pI[8][DIM], dI[8][DIM];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        state<DIM>(Pr, Cp + (I0 + a) * RS, pI[a]);
        state_diff<DIM>(Pr, C + (I0 + a) * RS, Cp + (I0 + a) * RS, dI[a]);
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
#pragma unroll
      for (int j = I0 + 8; j < NMAX; ++j) {
        if (j < N) {
          float pj[DIM], dj[DIM];
          state<DIM>(Pr, Cp + j * RS, pj);
          state_diff<DIM>(Pr, C + j * RS, Cp + j * RS, dj);
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
  }
  float Pd[NV], Pdd[NV];
  load_row(basis, t, 1, valid, Pd);
  load_row(basis, t, 2, valid, Pdd);
#pragma unroll
  for (int i = 0; i < NMAX; ++i) {
    if (i < N) {
      if (pc.use_v) {
        float v[DIM], dv[DIM], q[DIM];
        state<DIM>(Pd, Cp + i * RS, v);
        state_diff<DIM>(Pd, C + i * RS, Cp + i * RS, dv);
        ball_residual<DIM>(v, pc.v_max, q, dummy);
#pragma unroll
        for (int x = 0; x < DIM; ++x) { const float r = dv[x] - q[x]; r2 = fmaf(r, r, r2); }
      }
      if (pc.use_a) {
        float a[DIM], da[DIM], q[DIM];
        state<DIM>(Pdd, Cp + i * RS, a);
        state_diff<DIM>(Pdd, C + i * RS, Cp + i * RS, da);
        ball_residual<DIM>(a, pc.a_max, q, dummy);
#pragma unroll
        for (int x = 0; x < DIM; ++x) { const float r = da[x] - q[x]; r2 = fmaf(r, r, r2); }
      }
    }
  }
  r2 = valid ? r2 : 0.0f;
  r2 = warp_sum(r2);
  if ((threadIdx.x & 31) == 0) *resp = r2;
}

template <int DIM, int NMAX, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) fused_fwd_kernel(const __grid_constant__ FusedArgs A) {
  constexpr int RS = DIM * NP;
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const ProblemConsts& pc = A.pc;
  const int T = pc.T;
  const Layout<DIM, NMAX> L(T);
  const int TB = L.TB;

  // --- which scene / samples this CTA owns
  int sidx = 0;
  for (int q = 1; q < A.n_scenes; ++q) {
    if (A.sc[q].cta_begin <= (int)blockIdx.x) sidx = q;
    else break;
  }
  const int N = A.sc[sidx].N;
  const int Gs = A.sc[sidx].G;
  const int S = A.sc[sidx].S;
  const int s_first = ((int)blockIdx.x - A.sc[sidx].cta_begin) * Gs;
  const int G = min(Gs, S - s_first);
  const int robot_off = A.sc[sidx].robot_off;
  const int gsample0 = A.sc[sidx].sample_off + s_first;
  const long long per_sample = (long long)DIM * N * NV;
  const long long coef0 = A.sc[sidx].coef_off + (long long)s_first * per_sample;
  if (G <= 0) return;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  float* OPS = sm;
  float* BETA = sm + 4 * NV * NP;
  float* SAMP = sm + Layout<DIM, NMAX>::head_floats();

  // --- prologue: operators of this N, beta, per-sample state
  const float* gops = A.ops + (size_t)N * OPS_STRIDE;
  for (int v = tid; v < 4 * NV * NP; v += nthr) OPS[v] = gops[v];
  for (int v = tid; v < NMAX * RS; v += nthr) {
    const int i = v / RS, x = (v / NP) % DIM, k = v % NP;
    float beta = 0.0f;
    if (i < N && k < NV) {
      // b_i = (p, v, a at t = 0; p, v, a at t = H) of robot i along axis x
      float bi[6], bm[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) bm[q] = 0.0f;
      for (int j = 0; j < N; ++j) {
        const int rr = robot_off + j;
        float bj[6];
        bj[0] = A.start[rr * DIM + x];
        bj[1] = A.start_va ? A.start_va[(rr * 2 + 0) * DIM + x] : 0.0f;
        bj[2] = A.start_va ? A.start_va[(rr * 2 + 1) * DIM + x] : 0.0f;
        bj[3] = A.goal[rr * DIM + x];
        bj[4] = A.goal_va ? A.goal_va[(rr * 2 + 0) * DIM + x] : 0.0f;
        bj[5] = A.goal_va ? A.goal_va[(rr * 2 + 1) * DIM + x] : 0.0f;
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
    BETA[v] = beta;
  }
  for (int v = tid; v < G * NMAX * RS; v += nthr) {
    const int s = v / (NMAX * RS), rem = v % (NMAX * RS);
    const int i = rem / RS, x = (rem / NP) % DIM, k = rem % NP;
    float* blk = SAMP + (size_t)s * L.SB;
    float c = 0.0f, l = 0.0f, xb = 0.0f;
    if (i < N && k < NV) {
      const long long g = coef0 + s * per_sample + ((long long)x * N + i) * NV + k;
      xb = A.xi_bar[g];
      c = A.xi0 ? A.xi0[g] : xb;
      l = A.lam0 ? A.lam0[g] : 0.0f;
    }
    blk[L.C() + rem] = c;
    blk[L.LAM() + rem] = l;
    blk[L.XIB() + rem] = xb;
    blk[L.CPREV() + rem] = c;
    for (int tb = 0; tb < TB; ++tb) blk[L.GP(tb) + rem] = 0.0f;
  }
  __syncthreads();

  const int units = G * TB;
  const float rho = pc.rho;
  const float invN = 1.0f / (float)N;
  for (int it = 0; it < pc.K; ++it) {
    // ---- time phase
    for (int u = warp; u < units; u += nwarps) {
      const int s = u / TB, tb = u % TB;
      float* blk = SAMP + (size_t)s * L.SB;
      time_unit<DIM, NMAX>(blk + L.C(), A.basis, T, tb * 32 + lane, N, pc, blk + L.GP(tb),
                           blk + L.RESP() + tb, lane);
    }
    __syncthreads();
    // ---- solve phase 1: lambda step, r, robot means
    for (int v = tid; v < G * DIM * NV; v += nthr) {
      const int s = v / (DIM * NV), x = (v / NV) % DIM, k = v % NV;
      float* blk = SAMP + (size_t)s * L.SB;
      float sr = 0.0f, sc = 0.0f;
      for (int i = 0; i < N; ++i) {
        const int o = i * RS + x * NP + k;
        float g = 0.0f;
        for (int tb = 0; tb < TB; ++tb) g += blk[L.GP(tb) + o];
        const float lam = fmaf(rho, g, blk[L.LAM() + o]);
        blk[L.LAM() + o] = lam;
        const float r = fmaf(rho, g, lam) + blk[L.XIB() + o];
        blk[L.GP(0) + o] = r;
        sr += r;
        sc += blk[L.C() + o];
      }
      blk[L.MR() + x * NP + k] = sr * invN;
      blk[L.MC() + x * NP + k] = sc * invN;
      if (A.hist && x == 0 && k == 0) {
        float r2 = 0.0f;
        for (int tb = 0; tb < TB; ++tb) r2 += blk[L.RESP() + tb];
        A.hist[(size_t)it * A.total_samples + gsample0 + s] = sqrtf(r2);
      }
    }
    __syncthreads();
    // ---- solve phase 2: xi step
    const bool last = (it == pc.K - 1);
    for (int v = tid; v < G * N * DIM; v += nthr) {
      const int s = v / (N * DIM), i = (v / DIM) % N, x = v % DIM;
      float* blk = SAMP + (size_t)s * L.SB;
      const int o = i * RS + x * NP;
      float c[NP], r[NP], cm[NP], rm[NP];
      const float4* c4 = reinterpret_cast<const float4*>(blk + L.C() + o);
      const float4* r4 = reinterpret_cast<const float4*>(blk + L.GP(0) + o);
      const float4* cm4 = reinterpret_cast<const float4*>(blk + L.MC() + x * NP);
      const float4* rm4 = reinterpret_cast<const float4*>(blk + L.MR() + x * NP);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        float4 a = c4[q], b = r4[q], e = cm4[q], f = rm4[q];
        c[4 * q] = a.x; c[4 * q + 1] = a.y; c[4 * q + 2] = a.z; c[4 * q + 3] = a.w;
        r[4 * q] = b.x; r[4 * q + 1] = b.y; r[4 * q + 2] = b.z; r[4 * q + 3] = b.w;
        cm[4 * q] = e.x; cm[4 * q + 1] = e.y; cm[4 * q + 2] = e.z; cm[4 * q + 3] = e.w;
        rm[4 * q] = f.x; rm[4 * q + 1] = f.y; rm[4 * q + 2] = f.z; rm[4 * q + 3] = f.w;
      }
      float out[NP];
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        float acc = BETA[o + k];
#pragma unroll
        for (int m = 0; m < NV; ++m) {
          acc = fmaf(OPS[OPS_W1 + k * NP + m], c[m], acc);
          acc = fmaf(OPS[OPS_S1 + k * NP + m], r[m], acc);
          acc = fmaf(OPS[OPS_DW + k * NP + m], cm[m], acc);
          acc = fmaf(OPS[OPS_DS + k * NP + m], rm[m], acc);
        }
        out[k] = acc;
      }
      out[NV] = 0.0f;
      float4* o4 = reinterpret_cast<float4*>(blk + L.C() + o);
      float4* p4 = reinterpret_cast<float4*>(blk + L.CPREV() + o);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (last) p4[q] = make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
        o4[q] = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
      }
    }
    __syncthreads();
  }

  // ---- final residual, Eq. (primal_residual)
  for (int u = warp; u < units; u += nwarps) {
    const int s = u / TB, tb = u % TB;
    float* blk = SAMP + (size_t)s * L.SB;
    residual_unit<DIM, NMAX>(blk + L.C(), blk + L.CPREV(), A.basis, T, tb * 32 + lane, N, pc,
                             blk + L.RESP() + tb);
  }
  __syncthreads();
  for (int s = tid; s < G; s += nthr) {
    const float* blk = SAMP + (size_t)s * L.SB;
    float r2 = 0.0f;
    for (int tb = 0; tb < TB; ++tb) r2 += blk[L.RESP() + tb];
    const float r = sqrtf(r2);
    A.resid_out[gsample0 + s] = r;
    if (!isfinite(r)) atomicOr(A.status, ST_NONFINITE);
  }
  for (int v = tid; v < G * DIM * N * NV; v += nthr) {
    const int s = v / (DIM * N * NV), rem = v % (DIM * N * NV);
    const int x = rem / (N * NV), i = (rem / NV) % N, k = rem % NV;
    const float* blk = SAMP + (size_t)s * L.SB;
    const int o = i * RS + x * NP + k;
    const long long g = coef0 + (long long)s * per_sample + rem;
    A.xi_out[g] = blk[L.C() + o];
    A.lam_out[g] = blk[L.LAM() + o];
  }
}

template <int DIM, int NMAX, int MAXT>
cudaError_t launch_t(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st) {
  auto k = fused_fwd_kernel<DIM, NMAX, MAXT>;
  if (l.warps * 32 > MAXT) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem);
  if (e != cudaSuccess) return e;
  k<<<l.n_ctas, l.warps * 32, l.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fused_impl
}  // namespace sf
