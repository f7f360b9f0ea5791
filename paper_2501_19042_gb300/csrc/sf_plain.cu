// Plain form of the safety filter: one scene at a time, one launch per step
// of f_FP (Appendix, AM steps), states and residuals kept in HBM workspace
// between the steps. This is the straightforward float32 GPU mapping that the
// fused form is measured against.
//
// Per iteration:
//   states    p, v, a of every (sample, robot, axis, t)                 Eq. (poly)
//   project   alpha / beta / d steps for every pair row and the
//             velocity / acceleration rows: q = e - F xi              Eqs. (alpha_step)-(d_step)
//   transpose g = F^T q                                                 Eq. (lambda_step)
//   solve     lambda' = lambda + rho g; xi step with the pre-stored
//             KKT operators                                             Eq. (xi_step)
#include "sf_internal.cuh"

namespace sf {
namespace {

// X, Q layout: [S][3][dim][N][T]
__device__ __forceinline__ size_t xoff(int s, int blk, int x, int i, int t, int dim, int N, int T) {
  return ((((size_t)s * 3 + blk) * dim + x) * N + i) * (size_t)T + t;
}

__global__ void beta_kernel(PlainArgs a) {
  const int dim = a.pc.dim, N = a.N;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= dim * N * NP) return;
  const int x = v / (N * NP), i = (v / NP) % N, k = v % NP;
  float beta = 0.0f;
  if (k < NV) {
    float bi[6], bm[6];
    for (int q = 0; q < 6; ++q) bm[q] = bi[q] = 0.0f;
    for (int j = 0; j < N; ++j) {
      float bj[6];
      bj[0] = a.start[j * dim + x];
      bj[1] = a.start_va ? a.start_va[(j * 2 + 0) * dim + x] : 0.0f;
      bj[2] = a.start_va ? a.start_va[(j * 2 + 1) * dim + x] : 0.0f;
      bj[3] = a.goal[j * dim + x];
      bj[4] = a.goal_va ? a.goal_va[(j * 2 + 0) * dim + x] : 0.0f;
      bj[5] = a.goal_va ? a.goal_va[(j * 2 + 1) * dim + x] : 0.0f;
      for (int q = 0; q < 6; ++q) {
        bm[q] += bj[q];
        if (j == i) bi[q] = bj[q];
      }
    }
    const float* o = a.ops + (size_t)N * OPS_STRIDE;
    for (int q = 0; q < 6; ++q) {
      const float r0 = o[OPS_R0 + k * 8 + q], r1 = o[OPS_R1 + k * 8 + q];
      beta += r1 * bi[q] + (r0 - r1) * (bm[q] / (float)N);
    }
  }
  a.beta[v] = beta;
}

__global__ void init_kernel(PlainArgs a, const float* xi0, const float* lam0, long long n) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  a.xi[v] = xi0 ? xi0[v] : a.xi_bar[v];
  a.lam[v] = lam0 ? lam0[v] : 0.0f;
}

__global__ void states_kernel(PlainArgs a, const float* __restrict__ coef, float* __restrict__ X) {
  const int dim = a.pc.dim, N = a.N, T = a.pc.T;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (long long)a.S * N * T) return;
  const int t = v % T;
  const int i = (v / T) % N;
  const int s = v / ((long long)T * N);
  const float* brow = reinterpret_cast<const float*>(a.basis) + (size_t)t * BASIS_ROW;
  for (int x = 0; x < dim; ++x) {
    const float* c = coef + (((size_t)s * dim + x) * N + i) * NV;
    float p = 0.f, vv = 0.f, aa = 0.f;
    for (int k = 0; k < NV; ++k) {
      const float ck = c[k];
      p = fmaf(brow[k], ck, p);
      vv = fmaf(brow[NP + k], ck, vv);
      aa = fmaf(brow[2 * NP + k], ck, aa);
    }
    X[xoff(s, 0, x, i, t, dim, N, T)] = p;
    X[xoff(s, 1, x, i, t, dim, N, T)] = vv;
    X[xoff(s, 2, x, i, t, dim, N, T)] = aa;
  }
}

template <int DIM>
__global__ void project_kernel(PlainArgs a, int it) {
  const int N = a.N, T = a.pc.T;
  const int s = blockIdx.x;
  const float* X = a.X;
  float r2 = 0.0f;
  for (int u = threadIdx.x; u < N * T; u += blockDim.x) {
    const int i = u / T, t = u % T;
    float pi[DIM], E[DIM];
    for (int x = 0; x < DIM; ++x) { pi[x] = X[xoff(s, 0, x, i, t, DIM, N, T)]; E[x] = 0.f; }
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      float pj[DIM], q[DIM], dummy = 0.f;
      for (int x = 0; x < DIM; ++x) pj[x] = X[xoff(s, 0, x, j, t, DIM, N, T)];
      // row (min, max) of F: delta = p_min - p_max
      if (i < j) {
        pair_residual<DIM>(pi, pj, q, a.pc, r2);
        for (int x = 0; x < DIM; ++x) E[x] += q[x];
      } else {
        pair_residual<DIM>(pj, pi, q, a.pc, dummy);
        for (int x = 0; x < DIM; ++x) E[x] -= q[x];
      }
    }
    if (a.pc.use_w) {   // workspace row of robot i (its F row is P, like the pair rows)
      float q[DIM];
      ws_residual<DIM>(pi, a.pc, q, r2);
      for (int x = 0; x < DIM; ++x) E[x] += q[x];
    }
    float v[DIM], acc[DIM], qv[DIM], qa[DIM];
    for (int x = 0; x < DIM; ++x) {
      v[x] = X[xoff(s, 1, x, i, t, DIM, N, T)];
      acc[x] = X[xoff(s, 2, x, i, t, DIM, N, T)];
      qv[x] = qa[x] = 0.f;
    }
    if (a.pc.use_v) ball_residual<DIM>(v, a.pc.v_max, qv, r2);
    if (a.pc.use_a) ball_residual<DIM>(acc, a.pc.a_max, qa, r2);
    for (int x = 0; x < DIM; ++x) {
      a.Q[xoff(s, 0, x, i, t, DIM, N, T)] = E[x];
      a.Q[xoff(s, 1, x, i, t, DIM, N, T)] = qv[x];
      a.Q[xoff(s, 2, x, i, t, DIM, N, T)] = qa[x];
    }
  }
  __shared__ float red[32];
  for (int o = 16; o >= 1; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    if (a.hist) a.hist[(size_t)it * a.hist_stride + s] = sqrtf(tot);
  }
}

__global__ void transpose_kernel(PlainArgs a) {
  const int dim = a.pc.dim, N = a.N, T = a.pc.T;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= (long long)a.S * dim * N * NV) return;
  const int k = v % NV;
  const int i = (v / NV) % N;
  const int x = (v / ((long long)NV * N)) % dim;
  const int s = v / ((long long)NV * N * dim);
  const float* B = reinterpret_cast<const float*>(a.basis);
  const float* qe = a.Q + xoff(s, 0, x, i, 0, dim, N, T);
  const float* qv = a.Q + xoff(s, 1, x, i, 0, dim, N, T);
  const float* qa = a.Q + xoff(s, 2, x, i, 0, dim, N, T);
  float g = 0.f;
  for (int t = 0; t < T; ++t) {
    const float* row = B + (size_t)t * BASIS_ROW;
    g = fmaf(row[k], qe[t], g);
    g = fmaf(row[NP + k], qv[t], g);
    g = fmaf(row[2 * NP + k], qa[t], g);
  }
  a.g[v] = g;
}

// block per sample; xi step of the Appendix with the mean / deviation split
__global__ void solve_kernel(PlainArgs a, int last) {
  extern __shared__ float sh[];
  const int dim = a.pc.dim, N = a.N;
  const int s = blockIdx.x;
  const int n = dim * N * NV;
  float* c = sh;                // [dim][N][NV]
  float* r = sh + n;            // [dim][N][NV]
  float* cm = sh + 2 * n;       // [dim][NV]
  float* rm = cm + dim * NV;    // [dim][NV]
  const size_t base = (size_t)s * n;
  const float rho = a.pc.rho;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    const float g = a.g[base + v];
    const float lam = fmaf(rho, g, a.lam[base + v]);
    a.lam[base + v] = lam;
    r[v] = fmaf(rho, g, lam) + a.xi_bar[base + v];
    c[v] = a.xi[base + v];
    if (last) a.xprev[base + v] = c[v];
  }
  __syncthreads();
  for (int v = threadIdx.x; v < dim * NV; v += blockDim.x) {
    const int x = v / NV, k = v % NV;
    float sc = 0.f, sr = 0.f;
    for (int i = 0; i < N; ++i) {
      sc += c[(x * N + i) * NV + k];
      sr += r[(x * N + i) * NV + k];
    }
    cm[v] = sc / (float)N;
    rm[v] = sr / (float)N;
  }
  __syncthreads();
  const float* o = a.ops + (size_t)N * OPS_STRIDE;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    const int x = v / (N * NV), i = (v / NV) % N, k = v % NV;
    float acc = a.beta[(x * N + i) * NP + k];
    const float* ci = c + (x * N + i) * NV;
    const float* ri = r + (x * N + i) * NV;
    for (int m = 0; m < NV; ++m) {
      acc = fmaf(o[OPS_W1 + k * NP + m], ci[m], acc);
      acc = fmaf(o[OPS_S1 + k * NP + m], ri[m], acc);
      acc = fmaf(o[OPS_DW + k * NP + m], cm[x * NV + m], acc);
      acc = fmaf(o[OPS_DS + k * NP + m], rm[x * NV + m], acc);
    }
    a.xi[base + v] = acc;
  }
}

// ||F xi^K - e(xi^{K-1})||: X holds the states of xi^{K-1}, Q those of xi^K.
template <int DIM>
__global__ void residual_kernel(PlainArgs a) {
  const int N = a.N, T = a.pc.T;
  const int s = blockIdx.x;
  float r2 = 0.0f;
  for (int u = threadIdx.x; u < N * T; u += blockDim.x) {
    const int i = u / T, t = u % T;
    float po[DIM], pn[DIM];
    for (int x = 0; x < DIM; ++x) {
      po[x] = a.X[xoff(s, 0, x, i, t, DIM, N, T)];
      pn[x] = a.Q[xoff(s, 0, x, i, t, DIM, N, T)];
    }
    for (int j = i + 1; j < N; ++j) {
      float qo[DIM], pjo[DIM], dummy = 0.f;
      for (int x = 0; x < DIM; ++x) pjo[x] = a.X[xoff(s, 0, x, j, t, DIM, N, T)];
      pair_residual<DIM>(po, pjo, qo, a.pc, dummy);
      for (int x = 0; x < DIM; ++x) {
        const float dnew = pn[x] - a.Q[xoff(s, 0, x, j, t, DIM, N, T)];
        const float e = (po[x] - pjo[x]) + qo[x];
        const float rr = dnew - e;
        r2 = fmaf(rr, rr, r2);
      }
    }
    if (a.pc.use_w) {
      float q[DIM], dummy = 0.f;
      ws_residual<DIM>(po, a.pc, q, dummy);
      for (int x = 0; x < DIM; ++x) {
        const float rr = pn[x] - (po[x] + q[x]);
        r2 = fmaf(rr, rr, r2);
      }
    }
    for (int blk = 1; blk <= 2; ++blk) {
      if ((blk == 1 && !a.pc.use_v) || (blk == 2 && !a.pc.use_a)) continue;
      float vo[DIM], q[DIM], dummy = 0.f;
      for (int x = 0; x < DIM; ++x) vo[x] = a.X[xoff(s, blk, x, i, t, DIM, N, T)];
      ball_residual<DIM>(vo, blk == 1 ? a.pc.v_max : a.pc.a_max, q, dummy);
      for (int x = 0; x < DIM; ++x) {
        const float rr = a.Q[xoff(s, blk, x, i, t, DIM, N, T)] - (vo[x] + q[x]);
        r2 = fmaf(rr, rr, r2);
      }
    }
  }
  __shared__ float red[32];
  for (int o = 16; o >= 1; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    const float res = sqrtf(tot);
    a.resid_out[s] = res;
    if (!isfinite(res)) atomicOr(a.status, ST_NONFINITE);
  }
}

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

size_t plain_workspace_floats(int dim, int N, int S, int T) {
  const size_t n = (size_t)S * dim * N * NV;
  const size_t xs = (size_t)S * 3 * dim * N * (size_t)T;
  return (size_t)dim * N * NP + 2 * xs + 2 * n + (size_t)S + 64;
}

cudaError_t launch_plain(const PlainArgs& a, const float* xi0, const float* lam0, cudaStream_t st) {
  const int dim = a.pc.dim, N = a.N, S = a.S, T = a.pc.T, K = a.pc.K;
  if (S == 0) return cudaSuccess;
  const long long n = (long long)S * dim * N * NV;
  beta_kernel<<<nblk((long long)dim * N * NP, 128), 128, 0, st>>>(a);
  init_kernel<<<nblk(n, 256), 256, 0, st>>>(a, xi0, lam0, n);
  const size_t solve_smem = sizeof(float) * (2 * (size_t)dim * N * NV + 2 * (size_t)dim * NV);
  for (int it = 0; it < K; ++it) {
    states_kernel<<<nblk((long long)S * N * T, 256), 256, 0, st>>>(a, a.xi, a.X);
    if (dim == 3) project_kernel<3><<<S, 256, 0, st>>>(a, it);
    else project_kernel<2><<<S, 256, 0, st>>>(a, it);
    transpose_kernel<<<nblk(n, 256), 256, 0, st>>>(a);
    solve_kernel<<<S, 256, solve_smem, st>>>(a, it == K - 1);
  }
  states_kernel<<<nblk((long long)S * N * T, 256), 256, 0, st>>>(a, a.xprev, a.X);
  states_kernel<<<nblk((long long)S * N * T, 256), 256, 0, st>>>(a, a.xi, a.Q);
  if (dim == 3) residual_kernel<3><<<S, 256, 0, st>>>(a);
  else residual_kernel<2><<<S, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sf
