// Internal declarations of the GB300 safety-filter library: data layouts on
// the device, launch descriptors and the per-element closed forms shared by
// the fused, plain and adjoint kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sf.h"

namespace sf {

// Coefficients per robot-axis in the kernels: Bernstein order 10 (nvar = 11),
// stored padded to 12 floats so that a row is three float4.
constexpr int NV = 11;
constexpr int NP = 12;

// Basis table: per time step t, 36 floats = P[t][0..11], Pd[t][0..11],
// Pdd[t][0..11] (entry 11 of each row is 0).
constexpr int BASIS_ROW = 3 * NP;

// xi-step operators for one value of N (all float32, [k][m], m padded to 12):
//   W1 = S_dev rho H_dev, S1 = S_dev, DW = W_mean - W_dev, DS = S_mean - S_dev,
//   R0 = R_mean, R1 = R_dev ([k][q], q < 6, padded to 8).
// The xi step then is, per robot i and axis (Appendix, xi step, with the
// mean / deviation split of I + rho F^T F):
//   c_i' = W1 c_i + S1 r_i + DW cbar + DS rbar + beta_i,
//   beta_i = R1 b_i + (R0 - R1) bbar,   r = rho g + lambda' + xi_bar.
constexpr int OPS_W1 = 0;
constexpr int OPS_S1 = 1 * NV * NP;
constexpr int OPS_DW = 2 * NV * NP;
constexpr int OPS_DS = 3 * NV * NP;
constexpr int OPS_R0 = 4 * NV * NP;
constexpr int OPS_R1 = 4 * NV * NP + NV * 8;
constexpr int OPS_STRIDE = 4 * NV * NP + 2 * NV * 8;  // floats per N

// Scenes per launch descriptor (kernel parameter space).
constexpr int MAX_SCENES_PER_LAUNCH = 192;

struct SceneDesc {
  int N;           // robots
  int S;           // samples
  int G;           // samples per CTA (fused) / unused (plain)
  int cta_begin;   // first CTA of this scene in the launch
  int robot_off;   // row offset into start / goal
  int sample_off;  // global index of the scene's first sample
  long long coef_off;  // float offset of the scene's first sample in coefficient arrays
  long long mask_off;  // word offset of the scene's first sample in an activity-mask slot
};

// Activity masks (written by forward iterations that feed the adjoint): per
// (sample, t) a row of mask_words(NMAX) words, first the pair rows (bit
// pair_bit(i, j) for i < j, row-major over the upper triangle of NMAX x NMAX),
// then the rows of robot i (bit i: velocity outside its ball, bit NMAX + i:
// acceleration outside its ball, bit 2 NMAX + i: position outside the
// workspace), zero-padded to a multiple of 4 words.
__host__ __device__ constexpr int mask_pair_words(int nmax) { return (nmax * (nmax - 1) / 2 + 31) / 32; }
__host__ __device__ constexpr int mask_words(int nmax) {
  return ((mask_pair_words(nmax) + (3 * nmax + 31) / 32) + 3) / 4 * 4;
}
__host__ __device__ constexpr int pair_bit(int nmax, int i, int j) { return i * nmax - i * (i + 1) / 2 + (j - i - 1); }

// Bounded-wait / status words latched on the device.
enum : int { ST_NONFINITE = 1, ST_TIMEOUT = 2, ST_DEBUG = 4 };   // ST_DEBUG: site in bits 8..15

struct ProblemConsts {
  int dim, T, K;
  float rho;
  float inv_a2, inv_b2;  // 1/a^2, 1/b^2 of the collision spheroid
  float inv_a, inv_b;    // 1/a, 1/b
  float coll_a, coll_b;  // a, b
  float tie;             // e of a pair at delta = 0: (0,0,b) in 3D, (a,0) in 2D
  float v_max, a_max;
  int use_v, use_a;
  // workspace spheroid, Eq. (workspace_con): centre, semi-axes, their inverses, and the
  // map of collision-scaled positions ps = p M_a^-1 to workspace-scaled
  // offsets (p - p_w) M_w^-1 = ps * wk - wo
  int use_w;
  float wc[3], wa[3], winv[3], wk[3], wo[3];
};

struct FusedArgs {
  ProblemConsts pc;
  int n_scenes;
  const float4* basis;     // [T][9] float4
  const float* ops;        // [max_robots + 1][OPS_STRIDE]
  const float* start;      // [sum N][dim]
  const float* goal;
  const float* start_va;   // [sum N][2][dim] or null
  const float* goal_va;
  const float* xi_bar;
  const float* xi0;        // or null (sample init)
  const float* lam0;       // or null (zero)
  float* xi_out;
  float* lam_out;
  float* resid_out;        // [total samples]
  float* hist;             // [K][total samples] or null
  int total_samples;
  int* status;
  int tc;                  // time steps per chunk
  int nq;                  // time ranges per chunk in the contraction phase
  float* ckpt;             // [n_ck][2][total_coefs] or null
  int ck_every;            // checkpoint period
  long long total_coefs;
  float* fp_res2;          // [total samples] sum_k ||z^{k+1} - z^k||^2, or null
  unsigned* amask;         // activity masks of the last checkpoint segment [ck_every][slot], or null
  long long amask_slot;    // words per mask slot (one iteration, all samples)
  int prune;               // float32 form: exact pair pruning on (1) or every pair tested (0)
  unsigned long long wait_ns;   // tensor-memory form: bound of each MMA wait (0: the default)
  int skip_first_mma;      // tensor-memory form: the first MMA group is not issued (timeout test)
  int dbg_plant;           // debug builds: a wrong canary word is planted (test of the checks)
  SceneDesc sc[MAX_SCENES_PER_LAUNCH];
};

// ---- per-element closed forms (Appendix, alpha / beta / d steps) ----------
//
// Pair block: with scaled distance s2 = (dx^2 + dy^2)/a^2 + dz^2/b^2, the
// alpha / beta / d closed forms give e = delta when s2 >= 1 and
// e = delta / sqrt(s2) otherwise (d clipped to 1); at delta = 0 the tie-break
// alpha = beta = 0 gives e = (0, 0, b) (3D) or (a, 0) (2D). Returned is
// q = e - delta and its squared norm is added to res2.
template <int DIM>
__device__ __forceinline__ void pair_residual(const float* pi, const float* pj, float* q,
                                              const ProblemConsts& pc, float& res2) {
  float d[DIM];
#pragma unroll
  for (int x = 0; x < DIM; ++x) d[x] = pi[x] - pj[x];
  float s2;
  if (DIM == 3)
    s2 = fmaf(d[2] * d[2], pc.inv_b2, (d[0] * d[0] + d[1] * d[1]) * pc.inv_a2);
  else
    s2 = (d[0] * d[0] + d[1] * d[1]) * pc.inv_a2;
  const bool zero = (s2 == 0.0f);
  float s = fmaxf(rsqrtf(s2) - 1.0f, 0.0f);
  s = zero ? 0.0f : s;
#pragma unroll
  for (int x = 0; x < DIM; ++x) q[x] = s * d[x];
  if (zero) q[DIM == 3 ? 2 : 0] = pc.tie;
#pragma unroll
  for (int x = 0; x < DIM; ++x) res2 = fmaf(q[x], q[x], res2);
}

// Velocity / acceleration block (polar form with centre 0, d in [0, 1]): the
// Euclidean ball projection. q = e - v = -max(0, 1 - r/||v||) v; at v = 0, q = 0.
template <int DIM>
__device__ __forceinline__ void ball_residual(const float* v, float r, float* q, float& res2) {
  float n2 = 0.0f;
#pragma unroll
  for (int x = 0; x < DIM; ++x) n2 = fmaf(v[x], v[x], n2);
  const float s = fmaxf(fmaf(-r, rsqrtf(n2), 1.0f), 0.0f);
#pragma unroll
  for (int x = 0; x < DIM; ++x) {
    q[x] = -s * v[x];
    res2 = fmaf(q[x], q[x], res2);
  }
}

// Workspace block (polar form of Eq. workspace_polar, centre p_w, semi-axes
// (a_w, a_w, b_w), d in [0, 1]): with the scaled offset s2 = ||M_w^-1 (p - p_w)||^2
// the closed forms give e = p when s2 <= 1 and e = p_w + (p - p_w) / sqrt(s2)
// otherwise. q = e - p (position p unscaled); |q|^2 is added to res2.
template <int DIM>
__device__ __forceinline__ void ws_residual(const float* p, const ProblemConsts& pc, float* q, float& res2) {
  float d[DIM], s2 = 0.0f;
#pragma unroll
  for (int x = 0; x < DIM; ++x) {
    d[x] = p[x] - pc.wc[x];
    const float w = d[x] * pc.winv[x];
    s2 = fmaf(w, w, s2);
  }
  const float f = s2 > 1.0f ? rsqrtf(s2) - 1.0f : 0.0f;
#pragma unroll
  for (int x = 0; x < DIM; ++x) {
    q[x] = f * d[x];
    res2 = fmaf(q[x], q[x], res2);
  }
}

// ---- host-side launchers (defined in the .cu files) ------------------------
cudaError_t launch_precompute(int T, int order, double t_final, double rho, int use_v, int use_a, int use_w,
                              int max_robots, float* basis32, float* ops32, double* scratch64,
                              cudaStream_t st);
size_t precompute_scratch_doubles(int T, int order, int max_robots);

struct FusedLaunch {
  int nmax;     // 8, 16 or 32
  int warps;    // warps per CTA
  int gmax;     // largest samples-per-CTA of the scenes in this launch
  int n_ctas;
  int tc, nq;   // time chunk, contraction ranges
  size_t smem;  // dynamic shared memory bytes
  int prec;     // 0 float32 form, 3 / 4 / 5 tensor-memory form with tf32 / bf16 /
                // fp16 operands (PREC_TM_*)
};
// Internal form codes (FusedLaunch::prec) of the tensor-memory form.
constexpr int PREC_TM_TF32 = 3, PREC_TM_BF16 = 4, PREC_TM_FP16 = 5;
// Dynamic shared memory the tensor-memory form leaves to its static part.
constexpr size_t TM_STATIC_SMEM_RESERVE = 256;
size_t fused_smem_bytes(int dim, int nmax, int T, int gmax, int tc, int nq, bool bwd = false, int prec = 0);
cudaError_t launch_fused(const FusedArgs& a, const FusedLaunch& l, cudaStream_t st);
int fused_max_warps(int nmax, bool bwd);
cudaError_t prepare_kernels(int dim, int smem, int prec);

// Launch shape of the fused kernel for one group of scenes: samples per CTA,
// warps, time chunk, contraction ranges (cost model over the candidates,
// shared-memory bound checked).
struct FusedPlan {
  int G, warps, tc, nq;
  size_t smem;
  double cost;
};
FusedPlan plan_fused(int dim, int nmax, int T, const int* n_robots, const int* n_samples, int n_scenes,
                     int num_sms, size_t smem_cap, int force_G, int force_warps, int force_tc,
                     bool bwd = false, FusedPlan* top = nullptr, int n_top = 0, int prec = 0);

// Backward launch: everything the adjoint kernel needs besides the scene
// table (which it shares with FusedArgs).
struct BwdLaunchArgs {
  const float* ckpt;
  int ck_every;
  long long total_coefs;
  float* ring;
  const unsigned* tail_mask;   // masks of the last segment, written by the training forward
  unsigned* ring_mask;         // masks of a recomputed segment [ck_every][slot]
  long long mask_slot;
  const float* g_xi;
  const float* g_lam;
  const float* g_fp;
  float* gx0;
  float* gl0;
  float* gxb;
  int xi0_is_xi_bar;
};
cudaError_t launch_backward(const FusedArgs& a, const BwdLaunchArgs& b, const FusedLaunch& l, cudaStream_t st);

struct PlainArgs {
  ProblemConsts pc;
  const float4* basis;
  const float* ops;
  int N, S;
  const float* start;     // [N][dim] of this scene
  const float* goal;
  const float* start_va;
  const float* goal_va;
  const float* xi_bar;    // [S][dim][N][NV] for this scene
  float* xi;              // iterate (xi_out), [S][dim][N][NV]
  float* lam;             // multiplier (lambda_out)
  float* resid_out;       // [S]
  float* hist;            // [K][total] pointer already offset to this scene, or null
  int hist_stride;        // total samples
  // workspace (all float)
  float* beta;            // [dim][N][NP]
  float* X;               // states p, v, a: [S][3][dim][N][T]
  float* Q;               // residuals E, qv, qa: [S][3][dim][N][T]
  float* g;               // F^T q: [S][dim][N][NV]
  float* xprev;           // [S][dim][N][NV]
  float* r2;              // [S]
  int* status;
};
size_t plain_workspace_floats(int dim, int N, int S, int T);

// The decoders' QP layer (sf_eqqp.cu): per coefficient row, xi = Pi xi' + R b
// (forward) or Pi g and R^T g (backward).
struct EqScene {
  long long row_begin;  // first coefficient row (sample, axis, robot) of the scene
  int N;
  int robot_off;
};
struct EqArgs {
  const float* in;      // xi' (forward) or dL/dxi (backward), rows of 11
  float* out;           // xi (forward) or dL/dxi' (backward)
  float* grad_b;        // backward: dL/db [rows][6] or null
  const float* start;
  const float* goal;
  const float* start_va;
  const float* goal_va;
  long long rows;
  int dim, n_scenes, backward;
  float Pi[NV * NV];    // Pi and R in the parameter space: the FMAs read them as
  float R[NV * 6];      // constant operands (no load instruction per entry)
  EqScene sc[MAX_SCENES_PER_LAUNCH];
};
cudaError_t launch_eq(const EqArgs& a, cudaStream_t st);
cudaError_t launch_plain(const PlainArgs& a, const float* xi0, const float* lam0, cudaStream_t st);

}  // namespace sf
