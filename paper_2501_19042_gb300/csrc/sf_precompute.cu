// One-time float64 precompute of a handle (Appendix, xi step: "M is
// independent of the input ... its factorizations can be pre-stored").
//
//  1. Bernstein matrices P, Pd, Pdd of Eq. (poly) on tau_j = j/(T-1),
//     Pd = (1/t_f) dB/dtau, Pdd = (1/t_f^2) d2B/dtau2.
//  2. Gram matrices Q = P^T P and G = Pd^T Pd + Pdd^T Pdd (blocks switched
//     off by the problem are left out).
//  3. For every N: the KKT matrix of the xi step,
//       [[I + rho F^T F, A^T], [A, 0]],
//     F^T F = (N I - 1 1^T) (x) Q + I (x) G. The complete-graph Laplacian
//     N I - 1 1^T has eigenvalue 0 on the robot mean and N on every deviation
//     from it, and A = I (x) A1 acts per robot, so the system splits into one
//     17 x 17 "mean" KKT with I + rho G and identical 17 x 17 "deviation" KKTs
//     with I + rho G + rho N Q. Each is inverted by Gauss-Jordan with partial
//     pivoting; from the inverse [[S, R], [R^T, *]] the xi step needs S, R
//     and W = S rho H_k = S (M_k - I).
//  4. The same inverse with M = I (the decoders' equality-only QP layer)
//     into the operator slot of N = 0.
#include "sf_internal.cuh"

namespace sf {
namespace {

constexpr int KD = NV + 6;  // 17

__device__ double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

__device__ double binom_d(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

__device__ double bern_d(int n, int k, double tau) {
  if (n < 0 || k < 0 || k > n) return 0.0;
  return binom_d(n, k) * ipow(tau, k) * ipow(1.0 - tau, n - k);
}

// scratch64 layout: P64 [T][NV], Pd64, Pdd64, Q [NV][NV], G [NV][NV]
__global__ void basis_kernel(int T, int order, double t_final, float* basis32, double* s64) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int n = order;
  const double tau = (double)t / (double)(T - 1);
  double* P = s64;
  double* Pd = s64 + (size_t)T * NV;
  double* Pdd = s64 + 2 * (size_t)T * NV;
  float* row = basis32 + (size_t)t * BASIS_ROW;
  for (int k = 0; k < NP; ++k) {
    double p = 0.0, d1 = 0.0, d2 = 0.0;
    if (k <= n) {
      p = bern_d(n, k, tau);
      d1 = (double)n * (bern_d(n - 1, k - 1, tau) - bern_d(n - 1, k, tau)) / t_final;
      d2 = (double)n * (double)(n - 1) *
           (bern_d(n - 2, k - 2, tau) - 2.0 * bern_d(n - 2, k - 1, tau) + bern_d(n - 2, k, tau)) /
           (t_final * t_final);
    }
    if (k < NV) {
      P[t * NV + k] = p;
      Pd[t * NV + k] = d1;
      Pdd[t * NV + k] = d2;
    }
    row[k] = (float)p;
    row[NP + k] = (float)d1;
    row[2 * NP + k] = (float)d2;
  }
}

__global__ void gram_kernel(int T, int use_v, int use_a, int use_w, double* s64) {
  const int k = threadIdx.x / NV, m = threadIdx.x % NV;
  if (threadIdx.x >= NV * NV) return;
  const double* P = s64;
  const double* Pd = s64 + (size_t)T * NV;
  const double* Pdd = s64 + 2 * (size_t)T * NV;
  double* Q = s64 + 3 * (size_t)T * NV;
  double* G = Q + NV * NV;
  double q = 0.0, g = 0.0;
  for (int t = 0; t < T; ++t) {
    q += P[t * NV + k] * P[t * NV + m];
    if (use_v) g += Pd[t * NV + k] * Pd[t * NV + m];
    if (use_a) g += Pdd[t * NV + k] * Pdd[t * NV + m];
    if (use_w) g += P[t * NV + k] * P[t * NV + m];   // workspace rows F_w = I (x) P
  }
  Q[k * NV + m] = q;
  G[k * NV + m] = g;
}

// Inverts the KKT matrix [[M, A1^T], [A1, 0]] (KD x KD) by Gauss-Jordan with
// partial pivoting; returns S (NV x NV), R (NV x 6) and W = S (M - I).
__device__ bool kkt_operators(const double* M, const double* A1, double* S, double* R, double* W) {
  double aug[KD][2 * KD];
  for (int r = 0; r < KD; ++r)
    for (int c = 0; c < 2 * KD; ++c) aug[r][c] = 0.0;
  for (int r = 0; r < NV; ++r)
    for (int c = 0; c < NV; ++c) aug[r][c] = M[r * NV + c];
  for (int q = 0; q < 6; ++q)
    for (int c = 0; c < NV; ++c) {
      aug[NV + q][c] = A1[q * NV + c];
      aug[c][NV + q] = A1[q * NV + c];
    }
  for (int r = 0; r < KD; ++r) aug[r][KD + r] = 1.0;
  for (int col = 0; col < KD; ++col) {
    int p = col;
    double best = fabs(aug[col][col]);
    for (int r = col + 1; r < KD; ++r)
      if (fabs(aug[r][col]) > best) { best = fabs(aug[r][col]); p = r; }
    if (best == 0.0) return false;
    if (p != col)
      for (int c = 0; c < 2 * KD; ++c) { double t = aug[col][c]; aug[col][c] = aug[p][c]; aug[p][c] = t; }
    const double inv = 1.0 / aug[col][col];
    for (int c = 0; c < 2 * KD; ++c) aug[col][c] *= inv;
    for (int r = 0; r < KD; ++r) {
      if (r == col) continue;
      const double f = aug[r][col];
      if (f != 0.0)
        for (int c = 0; c < 2 * KD; ++c) aug[r][c] -= f * aug[col][c];
    }
  }
  for (int r = 0; r < NV; ++r) {
    for (int c = 0; c < NV; ++c) S[r * NV + c] = aug[r][KD + c];
    for (int q = 0; q < 6; ++q) R[r * 6 + q] = aug[r][KD + NV + q];
  }
  for (int r = 0; r < NV; ++r)
    for (int c = 0; c < NV; ++c) {
      double w = 0.0;
      for (int m = 0; m < NV; ++m) w += S[r * NV + m] * (M[m * NV + c] - (m == c ? 1.0 : 0.0));
      W[r * NV + c] = w;
    }
  return true;
}

__global__ void kkt_kernel(int T, double rho, int max_robots, double* s64, float* ops32, int* fail) {
  const int N = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (N > max_robots) return;
  const double* P = s64;
  const double* Pd = s64 + (size_t)T * NV;
  const double* Pdd = s64 + 2 * (size_t)T * NV;
  const double* Q = s64 + 3 * (size_t)T * NV;
  const double* G = Q + NV * NV;
  // Eq. (boundary_con): rows (p, pdot, pddot) at t = 0 and at t = H.
  double A1[6 * NV];
  for (int k = 0; k < NV; ++k) {
    A1[0 * NV + k] = P[k];
    A1[1 * NV + k] = Pd[k];
    A1[2 * NV + k] = Pdd[k];
    A1[3 * NV + k] = P[(T - 1) * NV + k];
    A1[4 * NV + k] = Pd[(T - 1) * NV + k];
    A1[5 * NV + k] = Pdd[(T - 1) * NV + k];
  }
  double M[NV * NV], S0[NV * NV], R0[NV * 6], W0[NV * NV], S1[NV * NV], R1[NV * 6], W1[NV * NV];
  if (N == 1) {
    // slot 0: the decoders' QP layer, [[I, A1^T], [A1, 0]]^-1 -> Pi (S1 field), R (R1 field)
    for (int r = 0; r < NV; ++r)
      for (int c = 0; c < NV; ++c) M[r * NV + c] = (r == c ? 1.0 : 0.0);
    if (!kkt_operators(M, A1, S0, R0, W0)) { atomicOr(fail, 1); return; }
    float* o0 = ops32;
    for (int r = 0; r < NV; ++r) {
      for (int c = 0; c < NP; ++c) o0[OPS_S1 + r * NP + c] = c < NV ? (float)S0[r * NV + c] : 0.0f;
      for (int q = 0; q < 8; ++q) o0[OPS_R1 + r * 8 + q] = q < 6 ? (float)R0[r * 6 + q] : 0.0f;
    }
  }
  for (int r = 0; r < NV; ++r)
    for (int c = 0; c < NV; ++c) M[r * NV + c] = (r == c ? 1.0 : 0.0) + rho * G[r * NV + c];
  bool ok = kkt_operators(M, A1, S0, R0, W0);
  for (int r = 0; r < NV; ++r)
    for (int c = 0; c < NV; ++c) M[r * NV + c] += rho * (double)N * Q[r * NV + c];
  ok = ok && kkt_operators(M, A1, S1, R1, W1);
  if (!ok) { atomicOr(fail, 1); return; }
  float* o = ops32 + (size_t)N * OPS_STRIDE;
  for (int r = 0; r < NV; ++r) {
    for (int c = 0; c < NP; ++c) {
      const bool in = c < NV;
      o[OPS_W1 + r * NP + c] = in ? (float)W1[r * NV + c] : 0.0f;
      o[OPS_S1 + r * NP + c] = in ? (float)S1[r * NV + c] : 0.0f;
      o[OPS_DW + r * NP + c] = in ? (float)(W0[r * NV + c] - W1[r * NV + c]) : 0.0f;
      o[OPS_DS + r * NP + c] = in ? (float)(S0[r * NV + c] - S1[r * NV + c]) : 0.0f;
    }
    for (int q = 0; q < 8; ++q) {
      o[OPS_R0 + r * 8 + q] = q < 6 ? (float)R0[r * 6 + q] : 0.0f;
      o[OPS_R1 + r * 8 + q] = q < 6 ? (float)R1[r * 6 + q] : 0.0f;
    }
  }
}

}  // namespace

size_t precompute_scratch_doubles(int T, int order, int max_robots) {
  (void)order;
  (void)max_robots;
  return 3 * (size_t)T * NV + 2 * NV * NV + 8;
}

cudaError_t launch_precompute(int T, int order, double t_final, double rho, int use_v, int use_a, int use_w,
                              int max_robots, float* basis32, float* ops32, double* scratch64,
                              cudaStream_t st) {
  int* fail = reinterpret_cast<int*>(scratch64 + 3 * (size_t)T * NV + 2 * NV * NV);
  cudaError_t e = cudaMemsetAsync(fail, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ops32, 0, sizeof(float) * (size_t)(max_robots + 1) * OPS_STRIDE, st);
  if (e != cudaSuccess) return e;
  basis_kernel<<<(T + 127) / 128, 128, 0, st>>>(T, order, t_final, basis32, scratch64);
  gram_kernel<<<1, NV * NV, 0, st>>>(T, use_v, use_a, use_w, scratch64);
  kkt_kernel<<<(max_robots + 31) / 32, 32, 0, st>>>(T, rho, max_robots, scratch64, ops32, fail);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int hfail = 0;
  e = cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  return hfail ? cudaErrorInvalidValue : cudaSuccess;
}

}  // namespace sf
