// The generative decoders' differentiable QP layer (Sec. III-A / B: Eq.
// (sf_form) with only the equality constraints of Eq. (boundary_con)): the
// Euclidean projection of xi' onto {xi : A xi = b}. A is block diagonal with
// one 6 x 11 block A1 per (axis, robot), so per coefficient row (sample,
// axis, robot)
//   xi = Pi xi' + R b,   Pi = I - A1^T (A1 A1^T)^-1 A1,   R = A1^T (A1 A1^T)^-1,
// with Pi and R the xi-rows of the inverse of [[I, A1^T], [A1, 0]] (computed
// once per handle in float64). The adjoint is dL/dxi' = Pi g (Pi is
// symmetric) and dL/db = R^T g.
//
// HBM-bound: 44 bytes read and 44 written per row. A block stages 256
// contiguous rows through shared memory so that global loads and stores are
// fully coalesced (rows are 11 floats, not 16-byte multiples); Pi and R sit
// in the kernel parameters, so the 187 multiply-adds of a row need no loads
// of matrix entries.
#include "sf_internal.cuh"

namespace sf {
namespace {

constexpr int EQ_ROWS = 256;   // rows per block (one thread per row)
static_assert(EQ_ROWS * NV / 4 <= 3 * EQ_ROWS, "16-byte staging takes at most 3 loads per thread");

__device__ __forceinline__ int find_scene(const EqArgs& a, long long row) {
  int lo = 0, hi = a.n_scenes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.sc[mid].row_begin <= row) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(EQ_ROWS) eq_kernel(const __grid_constant__ EqArgs a) {
  __shared__ __align__(16) float buf[EQ_ROWS * NV];
  const int tid = threadIdx.x;
  const float* Pi = a.Pi;
  const float* Rm = a.R;
  const long long r0 = (long long)blockIdx.x * EQ_ROWS;
  const int nrows = (int)min((long long)EQ_ROWS, a.rows - r0);
  const float* src = a.in + r0 * NV;
  const int nf = nrows * NV;
  // 16-byte loads when the block's rows start on a 16-byte boundary (r0 is a
  // multiple of 256 rows, so this holds whenever the array base does)
  if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
    // all of a thread's 16-byte loads are issued before any is stored, so
    // that they are in flight together (EQ_ROWS * 11 / 4 / EQ_ROWS <= 3)
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4 r[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int v = tid + j * EQ_ROWS;
      if (v < nf / 4) r[j] = s4[v];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int v = tid + j * EQ_ROWS;
      if (v < nf / 4) reinterpret_cast<float4*>(buf)[v] = r[j];
    }
    for (int v = (nf / 4) * 4 + tid; v < nf; v += EQ_ROWS) buf[v] = src[v];
  } else {
    for (int v = tid; v < nf; v += EQ_ROWS) buf[v] = src[v];
  }
  __syncthreads();
  if (tid < nrows) {
    const long long row = r0 + tid;
    float v[NV], o[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = buf[tid * NV + k];   // stride 11: no bank conflicts
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < NV; ++m) acc = fmaf(Pi[k * NV + m], v[m], acc);
      o[k] = acc;
    }
    const EqScene& sc = a.sc[find_scene(a, row)];
    const unsigned rel = (unsigned)(row - sc.row_begin);   // < 2^31 rows per scene (checked on the host)
    const unsigned qd = rel / (unsigned)sc.N;
    const int i = (int)(rel - qd * (unsigned)sc.N), x = (int)(qd % (unsigned)a.dim);
    const int rr = sc.robot_off + i;
    if (a.backward) {
      if (a.grad_b) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          float acc = 0.0f;
#pragma unroll
          for (int k = 0; k < NV; ++k) acc = fmaf(Rm[k * 6 + q], v[k], acc);
          a.grad_b[row * 6 + q] = acc;
        }
      }
    } else {
      float b[6];
      b[0] = a.start[rr * a.dim + x];
      b[1] = a.start_va ? a.start_va[(rr * 2 + 0) * a.dim + x] : 0.0f;
      b[2] = a.start_va ? a.start_va[(rr * 2 + 1) * a.dim + x] : 0.0f;
      b[3] = a.goal[rr * a.dim + x];
      b[4] = a.goal_va ? a.goal_va[(rr * 2 + 0) * a.dim + x] : 0.0f;
      b[5] = a.goal_va ? a.goal_va[(rr * 2 + 1) * a.dim + x] : 0.0f;
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int q = 0; q < 6; ++q) o[k] = fmaf(Rm[k * 6 + q], b[q], o[k]);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) buf[tid * NV + k] = o[k];
  }
  __syncthreads();
  float* dst = a.out + r0 * NV;
  if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int v = tid; v < nf / 4; v += EQ_ROWS) d4[v] = reinterpret_cast<const float4*>(buf)[v];
    for (int v = (nf / 4) * 4 + tid; v < nf; v += EQ_ROWS) dst[v] = buf[v];
  } else {
    for (int v = tid; v < nf; v += EQ_ROWS) dst[v] = buf[v];
  }
}

}  // namespace

cudaError_t launch_eq(const EqArgs& a, cudaStream_t st) {
  if (a.rows <= 0) return cudaSuccess;
  const long long blocks = (a.rows + EQ_ROWS - 1) / EQ_ROWS;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  eq_kernel<<<(unsigned)blocks, EQ_ROWS, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sf
