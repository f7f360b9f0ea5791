/*
 * sf.h — C ABI of the GB300-native batched safety filter (SF) of Swarm-Gen,
 * arXiv 2501.19042 (Sec. III-C and Appendix, "Custom SF optimizer").
 *
 * The library projects many sampled joint swarm trajectories onto the
 * feasible set of Eq. (sf_form): boundary conditions A xi = b
 * (Eq. boundary_con), velocity / acceleration bounds, and collision avoidance
 * between every pair of robots at every time step (Eq. inter_robot_con). It
 * runs the paper's fixed-point iteration f_FP (Eq. fixed_point), whose steps
 * are the alpha / beta / d closed forms, the multiplier update and the
 * equality-constrained xi step of the Appendix.
 *
 * Conventions
 *  - Every call returns an sf_status; no C++ exception crosses the ABI.
 *    sf_last_error() gives a human-readable message for the last failure on a
 *    handle.
 *  - Sizes and shapes are validated on the host before any launch.
 *  - Device pointers are CUDA device memory owned by the caller; the library
 *    never frees them. The handle owns only its precomputed basis matrices and
 *    solve operators.
 *  - Compute calls are asynchronous on the caller's stream (passed as a
 *    cudaStream_t cast to void*; NULL is the legacy default stream). No
 *    implicit host synchronisation, except where a function says so.
 *  - Device-side errors (non-finite values) are latched in a device word;
 *    sf_sync_status() synchronises the stream and returns them. The only
 *    device-side wait is the tensor-memory form's wait for its own MMAs
 *    (tcgen05.commit to an mbarrier); it gives up after one second of the
 *    GPU's global timer, stops issuing MMAs, drains (bounded) and frees its
 *    tensor memory, and latches SF_ERR_TIMEOUT (outputs of that call are
 *    then undefined; the context stays usable).
 *  - Layouts (row-major, float32 unless stated):
 *      coefficients (xi_bar, xi0, lambda0, xi_out, lambda_out, gradients):
 *        per sample [dim][N][nvar], nvar = order + 1 (the paper's xi vector,
 *        Sec. II-B: all robots' x coefficients, then y, then z); samples of a
 *        scene are contiguous and scenes follow each other.
 *      start, goal: [sum_s N_s][dim];  start_va, goal_va: [sum_s N_s][2][dim]
 *        holding (velocity, acceleration).
 *      per-sample scalars (residual_out): [sum_s S_s];
 *      residual_hist: [K][sum_s S_s].
 */
#ifndef GB300_SWARM_SF_H
#define GB300_SWARM_SF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SF_ABI_VERSION 1
#define SF_MAX_SCENES 4096   /* scenes in one sf_batch */
#define SF_MAX_ROBOTS 32     /* N per scene */
#define SF_MAX_T 1024        /* time steps */

typedef enum {
  SF_OK = 0,
  SF_ERR_INVALID_ARG = 1,   /* bad size, shape, pointer or value */
  SF_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  SF_ERR_OOM = 3,           /* handle-owned allocation failed */
  SF_ERR_TIMEOUT = 4,       /* a bounded device wait ran out */
  SF_ERR_NONFINITE = 5,     /* a non-finite value reached the output */
  SF_ERR_UNSUPPORTED = 6,   /* valid request this build does not implement */
  SF_ERR_WORKSPACE = 7,     /* workspace missing or too small */
  SF_ERR_DEBUG_CHECK = 8    /* a library built with SF_DEBUG_CHECKS found a shared-memory canary
                               overwritten or an index out of range (the access was skipped) */
} sf_status;

/* Arithmetic of the coefficient-to-state products (velocities and
 * accelerations of Eq. (poly), which the ball rows need at every time step
 * of every iteration). The positions of the pair rows, F^T of the residual
 * in the lambda step of the Appendix, the projections, residuals,
 * multiplier updates and the xi step are float32 in every mode; the
 * one-time factorisation of the KKT matrix is float64.
 * In the 16-bit modes (and in float32 with SF_OPT_TENSOR_MEMORY) the fused
 * forward takes those products on the 5th-generation tensor cores through
 * tensor memory (tcgen05 MMAs, float32 accumulation): both operands are
 * split into a rounded part and its rounding remainder, and the product is
 * taken in three terms (the remainder x remainder term dropped), which keeps
 * about 16 bits (bf16) or 21 bits (tf32, fp16) of the operands. The plain
 * form is float32 only (SF_ERR_UNSUPPORTED on a 16-bit handle); the adjoint
 * runs in float32 in every mode. */
typedef enum {
  SF_PREC_FP32 = 0,  /* float32 everywhere */
  SF_PREC_BF16 = 1,  /* tensor-memory MMAs with bf16 operands, float32 accumulation */
  SF_PREC_FP16 = 2   /* tensor-memory MMAs with fp16 operands, float32 accumulation */
} sf_precision;

/* How the iteration is laid out on the GPU. */
typedef enum {
  SF_FORM_FUSED = 0, /* one persistent launch: state resident on chip for all K iterations */
  SF_FORM_PLAIN = 1  /* one launch per step per iteration, time-domain arrays in HBM (workspace) */
} sf_form;

/* Problem constants shared by every scene of a handle (paper Sec. II and the
 * Appendix). */
typedef struct {
  int dim;             /* 2 or 3 */
  int order;           /* Bernstein order of Eq. (poly); nvar = order + 1; this build: 10 */
  int T;               /* time steps on tau_j = j/(T-1); 2..SF_MAX_T */
  double t_final;      /* horizon H in seconds, > 0 */
  double rho;          /* weight of Eq. (aug_lag), > 0 */
  double coll_a;       /* collision semi-axes (a, a, b) of M_a, Eq. (inter_robot_con); > 0 */
  double coll_b;
  double v_max;        /* velocity bound (norm); <= 0 disables the block */
  double a_max;        /* acceleration bound (norm); <= 0 disables the block */
  int use_workspace;   /* 1: every position stays in the workspace spheroid of Eq. (workspace_con) */
  double ws_center[3]; /* its centre p_w (first dim entries used) */
  double ws_a, ws_b;   /* its semi-axes (a_w, a_w, b_w), > 0 when use_workspace (ws_b unused in 2D) */
  int max_robots;      /* largest N of any scene used with the handle, 1..SF_MAX_ROBOTS */
  int precision;       /* sf_precision */
  int checkpoint_every;/* k of the checkpointed backward; 0 = no gradient support */
} sf_problem;

/* A batch of scenes. Scene s has N_s robots and S_s samples. */
typedef struct {
  int n_scenes;              /* 1..SF_MAX_SCENES */
  const int *n_robots;       /* HOST [n_scenes], each 1..max_robots */
  const int *n_samples;      /* HOST [n_scenes], each >= 0 */
  const float *start;        /* device [sum N_s][dim] start positions (b_0, Eq. boundary_con) */
  const float *goal;         /* device [sum N_s][dim] goal positions (b_H) */
  const float *start_va;     /* device [sum N_s][2][dim] start velocity, acceleration; NULL = 0 */
  const float *goal_va;      /* device [sum N_s][2][dim] goal velocity, acceleration; NULL = 0 */
  const float *xi_bar;       /* device coefficients of the sampled trajectories (Eq. sf_form) */
} sf_batch;

typedef struct sf_handle sf_handle;

/* Creates a handle on CUDA device `device`: computes on the GPU, in float64,
 * the Bernstein matrices of Eq. (poly) and, for every N in 1..max_robots, the
 * solution operators of the xi step (the KKT matrix of the Appendix is
 * input-independent, so its factorisation is pre-stored). Synchronises the
 * device once. *out is NULL on failure. */
sf_status sf_create(const sf_problem *problem, int device, sf_handle **out);

/* Frees the handle and its device memory. NULL is a no-op. */
void sf_destroy(sf_handle *h);

/* Last error message of the handle (static storage until the next call on it). */
const char *sf_last_error(const sf_handle *h);

/* Device workspace, in bytes, that sf_project needs for `batch` in `form`
 * with `K` iterations. The fused form needs 0 unless residual_hist or
 * checkpoints are requested; the plain form holds its time-domain arrays
 * here. Returns 0 and sets the error on invalid input. */
size_t sf_workspace_bytes(const sf_handle *h, const sf_batch *batch, int form, int K);

/* Bytes of the checkpoint buffer sf_project / sf_project_train write for
 * sf_project_backward: (xi, lambda) of every sample every checkpoint_every
 * iterations, followed by every iterate of the last segment (so that the
 * backward recomputes all segments but the last). */
size_t sf_checkpoint_bytes(const sf_handle *h, const sf_batch *batch, int K);

/* Runs K >= 1 iterations of f_FP on every sample of the batch.
 *   xi0, lambda0   device initial iterate, same layout as xi_bar; NULL gives
 *                  the sample init xi0 = xi_bar, lambda0 = 0.
 *   xi_out, lambda_out   device, the K-th iterate (required).
 *   residual_out   device [sum S_s]: ||r_p||_2 of Eq. (primal_residual) after
 *                  iteration K, i.e. ||F xi^K - e(xi^{K-1})||_2 (required).
 *   residual_hist  device [K][sum S_s] or NULL: ||F xi^k - e(xi^k)||_2 at the
 *                  start of iteration k (the projection residual).
 *   workspace      device, sf_workspace_bytes() bytes (may be NULL when 0).
 *   checkpoints    device, sf_checkpoint_bytes() bytes, or NULL for no gradient.
 * The output buffers must not overlap the inputs. */
sf_status sf_project(sf_handle *h, void *stream, const sf_batch *batch, int K, int form,
                     const float *xi0, const float *lambda0, float *xi_out, float *lambda_out,
                     float *residual_out, float *residual_hist, void *workspace,
                     size_t workspace_bytes, void *checkpoints);

/* Device staging bytes sf_project_host needs for `batch` (whose pointers are
 * host pointers in that call): the inputs, the outputs and, for the plain
 * form, its workspace. */
size_t sf_host_staging_bytes(const sf_handle *h, const sf_batch *batch, int form, int K);

/* sf_project on HOST buffers: copies the batch (and xi0 / lambda0 when not
 * NULL) into `staging` (device, sf_host_staging_bytes() bytes), runs the
 * same launches as sf_project, copies xi, lambda and the residuals back into
 * the host arrays, and synchronises `stream` before returning. Pinned host
 * memory gives asynchronous copies; pageable memory works but copies
 * synchronously. */
sf_status sf_project_host(sf_handle *h, void *stream, const sf_batch *batch, int K, int form,
                          const float *xi0, const float *lambda0, float *xi_out,
                          float *lambda_out, float *residual_out, void *staging,
                          size_t staging_bytes);

/* Number of kernels the handle has launched so far (all calls, all streams).
 * Lets a caller count the library's launches inside a timed region. */
unsigned long long sf_launch_count(const sf_handle *h);

/* Launch shape of the fused form: samples per CTA (G), warps per CTA, time
 * steps per chunk (tc; even in the 16-bit modes). Values <= 0 leave that
 * choice to the library's cost model. Applies to later sf_project calls on
 * the handle; a shape that does not fit in shared memory (or an odd tc in a
 * 16-bit mode) makes them fail with SF_ERR_UNSUPPORTED. With the shape
 * forced, the order of every reduction follows from the shape and the
 * robot-count bucket alone, so a sample's results do not depend on which
 * other scenes and samples share the call (a batch split over ranks gives
 * the same bits as the whole batch). */
sf_status sf_set_launch_shape(sf_handle *h, int samples_per_cta, int warps, int time_chunk);

/* Options of a handle (sf_set_option). */
typedef enum {
  /* 1 (default): between full pair tests, the float32 fused forward tests
   * only the pair rows that were within scaled distance 1.5 at the last full
   * test of the sample; a full test is rerun as soon as the sample's
   * coefficients may have moved its positions by 0.25 (scaled) or more, in a
   * bound that holds for every t (Bernstein weights are non-negative and sum
   * to 1); with the workspace block, the workspace rows of robots that were
   * within 0.1 (workspace-scaled) of its boundary are retested likewise. The
   * result is the same as testing every row. 0: every row every iteration.
   * The decision is taken per sample. No effect in the plain form and the
   * backward's recompute. */
  SF_OPT_PAIR_PRUNING = 1,
  /* Form of the fused forward of a float32 handle (sf_project and
   * sf_project_train). 1: the velocity / acceleration products on the tensor
   * cores through tensor memory (tcgen05 MMAs, the coefficient rows of a
   * CTA's samples as the A operand in TMEM, the basis rows of a time chunk as
   * the B operand in shared memory, three-term split of tf32 operands); the
   * rest stays on the float32 lanes. 0: the float32 form, products on the
   * lanes too. 2 (the default): per launch group, the form measured faster
   * on a GB300: the tensor-memory form for 3D scenes of 9..24 robots when its
   * launch shape fills at least 96 of a CTA's 128 TMEM lanes (6 samples per
   * CTA at 9..16 robots, 4 at 17..24; about 600 or more samples of such
   * scenes), the float32 form otherwise. Both forms give outputs within
   * rounding of each other. 16-bit handles always use the tensor-memory
   * form. */
  SF_OPT_TENSOR_MEMORY = 2,
  /* Test of the timeout path, value in microseconds (0 = off, the default):
   * the tensor-memory form does not issue the first MMA group of each CTA
   * and bounds every MMA wait by `value` microseconds, so the first wait runs
   * out with nothing in flight and sf_sync_status reports SF_ERR_TIMEOUT.
   * Outputs of such calls are undefined. No effect on the float32 form. */
  SF_OPT_TEST_WAIT_TIMEOUT = 3,
  /* Test of the debug-build checks (libraries built with SF_DEBUG_CHECKS
   * only; SF_ERR_UNSUPPORTED otherwise). 1: the fused kernels write a wrong
   * value into the canary word at the end of each CTA's last sample block,
   * so sf_sync_status reports SF_ERR_DEBUG_CHECK. Outputs are unaffected. */
  SF_OPT_TEST_CANARY = 4
} sf_option;

/* Sets option `option` of the handle to `value` (for later calls).
 * SF_ERR_INVALID_ARG for an unknown option or value. */
sf_status sf_set_option(sf_handle *h, int option, int value);

/* Shape of the last fused launch of the handle: out[0..3] = G, warps, tc and
 * the number of time ranges of the contraction phase. */
sf_status sf_get_launch_shape(const sf_handle *h, int *out4);

/* Form of the last fused launch of the handle (the last launch group of a
 * batch with several robot-count buckets): 1 the tensor-memory form, 0 the
 * float32 form. */
sf_status sf_get_launch_form(const sf_handle *h, int *tensor_memory);

/* The launch shape the library's cost model picks for one fused forward
 * launch group, without a device and without a handle: n_scenes scenes of
 * n_robots[q] robots and n_samples[q] samples (host arrays; every n_robots[q]
 * in the same robot-count bucket 1-8, 9-16, 17-24 or 25-32), dim axes, T
 * time steps, precision an sf_precision, on a GPU with num_sms SMs and
 * smem_per_block_optin bytes of opt-in shared memory per block. Writes out4
 * = G, warps, tc, nq (as sf_get_launch_shape) and, when out_smem is not NULL,
 * the dynamic shared memory per CTA. SF_ERR_INVALID_ARG for bad arguments,
 * SF_ERR_UNSUPPORTED when no shape fits in shared memory. */
sf_status sf_plan_launch(int dim, int T, int n_scenes, const int *n_robots, const int *n_samples, int precision,
                         int num_sms, size_t smem_per_block_optin, int *out4, size_t *out_smem);

/* Measurement-based choice of the fused launch shape for this batch's scene
 * mix: for every launch group (scenes sharing a robot-count bucket) the
 * n_candidates cheapest shapes of the cost model are each run with K_probe
 * iterations on `stream` and timed with CUDA events; the fastest is stored
 * in the handle and used by later sf_project / sf_graph_capture calls for
 * the same scene mix. Writes scratch results into xi_out, lambda_out,
 * residual_out (device, sized as for sf_project). Synchronises `stream`. */
sf_status sf_autotune(sf_handle *h, void *stream, const sf_batch *batch, int K_probe,
                      int n_candidates, float *xi_out, float *lambda_out, float *residual_out);

/* A CUDA graph of one sf_project call with fixed pointers: the launches of
 * every robot-count group (concurrent branches when there are several) in
 * one graph. The buffers passed at capture must stay allocated while the
 * graph is used; their contents may change between launches. */
typedef struct sf_graph sf_graph;
sf_status sf_graph_capture(sf_handle *h, const sf_batch *batch, int K, int form, const float *xi0,
                           const float *lambda0, float *xi_out, float *lambda_out,
                           float *residual_out, float *residual_hist, void *workspace,
                           size_t workspace_bytes, sf_graph **out);
/* Launches the graph on `stream` (asynchronous). */
sf_status sf_graph_launch(sf_graph *g, void *stream);
/* Frees the graph. NULL is a no-op. */
void sf_graph_destroy(sf_graph *g);

/* Plain form without any device allocation. The paper has no counterpart to
 * this entry point; it exists for callers that cannot allocate device
 * memory at call time, for example a host framework that owns every device
 * allocation and forbids its plug-ins to call cudaMalloc, or a control loop
 * that may not make calls whose latency is unbounded or that can
 * synchronise the device.
 *
 * It runs the same kernels as sf_project(..., SF_FORM_PLAIN, ...), but their
 * scratch (the time-domain arrays) lives in one buffer built into the
 * library: a static device array of SF_NOALLOC_SCRATCH_BYTES (32 MiB) that
 * every GPU which loads the library holds until the process exits. The
 * caller still passes all inputs and outputs (device memory, as in
 * sf_project). A batch whose largest scene needs more scratch than the
 * buffer holds is rejected with SF_ERR_INVALID_ARG before any launch (need:
 * about 4 * S * N * dim * (6 T + 2 * nvar) bytes for a scene of S samples).
 * The call itself allocates nothing: no cudaMalloc, no cudaFree.
 *
 * The first call on a device looks up the device address of the buffer
 * (cudaGetSymbolAddress with that device current); make that first call
 * before capturing the stream into a graph. The address is looked up again
 * when the device's context has changed since (after cudaDeviceReset); a
 * handle itself does not survive cudaDeviceReset (its device memory is
 * gone), so destroy handles before a reset and create new ones after it. All calls share the one buffer
 * and it keeps the last call's contents; every kernel writes each scratch
 * element before reading it, so nothing has to be cleared between calls.
 * Two calls whose work overlaps on the GPU (different streams, or different
 * handles on the same device) race on the buffer and give wrong results:
 * serialise them. residual_hist may be NULL. */
#define SF_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
sf_status sf_project_plain_noalloc(sf_handle *h, void *stream, const sf_batch *batch, int K,
                                   const float *xi0, const float *lambda0, float *xi_out,
                                   float *lambda_out, float *residual_out, float *residual_hist);

/* Forward for training (fused form, SF_PREC_FP32): as sf_project, and in
 * addition
 *   fp_res2_out  device [sum S_s] or NULL: sum over k < K of
 *                ||z^{k+1} - z^k||^2 with z = (xi, lambda), the first term of
 *                Eq. (NN_loss) (the fixed-point residual of the unroll);
 *   checkpoints  device, sf_checkpoint_bytes() bytes (required): (xi, lambda)
 *                of every sample at iterations 0, k, 2k, ... (k =
 *                checkpoint_every of the problem), layout
 *                [n_checkpoints][2][total coefficients], then the iterates
 *                last_checkpoint .. K in the same [slot][2][total] layout.
 * Needs a handle created with checkpoint_every > 0. */
sf_status sf_project_train(sf_handle *h, void *stream, const sf_batch *batch, int K,
                           const float *xi0, const float *lambda0, float *xi_out, float *lambda_out,
                           float *residual_out, float *fp_res2_out, void *checkpoints);

/* Device workspace of sf_project_backward: the iterates of one checkpoint
 * segment ((checkpoint_every + 1) x 2 x total coefficients floats), then the
 * activity masks of that segment's iterations. */
size_t sf_backward_workspace_bytes(const sf_handle *h, const sf_batch *batch, int K);

/* Reverse mode through the K unrolled iterations of a previous
 * sf_project_train call with the same batch, K and initial iterate (the
 * paper trains its initialisation network through the unrolled solver,
 * Sec. III-C, Eq. NN_loss). With
 *   L = <grad_xi_out, xi^K> + <grad_lambda_out, lambda^K>
 *       + sum_s grad_fp_res2[s] * fp_res2[s],
 * it writes dL/dxi^0 (grad_xi0), dL/dlambda^0 (grad_lambda0) and dL/dxi_bar
 * (grad_xi_bar); any of the three may be NULL, and so may each of the three
 * incoming gradients (= 0). init_from_xi_bar != 0 states that the forward
 * ran with xi0 == NULL (xi^0 = xi_bar); grad_xi_bar then includes that path.
 * Each segment of checkpoint_every iterations is recomputed from its
 * checkpoint into `workspace` (sf_backward_workspace_bytes() bytes) and
 * walked back. At non-differentiable points the Jacobian of the closed-form
 * steps is taken as the one-sided value of the active or inactive branch;
 * at delta = 0 the Jacobian of e is 0. */
sf_status sf_project_backward(sf_handle *h, void *stream, const sf_batch *batch, int K,
                              int init_from_xi_bar, const void *checkpoints,
                              const float *grad_xi_out, const float *grad_lambda_out,
                              const float *grad_fp_res2, float *grad_xi0, float *grad_lambda0,
                              float *grad_xi_bar, void *workspace, size_t workspace_bytes);

/* The generative decoders' differentiable QP layer (Sec. III-A / B: Eq.
 * (sf_form) without the inequality constraints; the paper has no separate
 * equation number). For every (sample, axis, robot) coefficient row of
 * batch->xi_bar (here the decoder output xi'),
 *   xi_out = argmin ||xi - xi'||^2  subject to  A1 xi = b,
 * with A1 the boundary rows of Eq. (boundary_con) and b = (start position,
 * start velocity, start acceleration, goal position, goal velocity, goal
 * acceleration) of that robot and axis (velocities / accelerations 0 when
 * start_va / goal_va are NULL). Closed form: xi_out = Pi xi' + R b with the
 * float64-precomputed Pi = I - A1^T (A1 A1^T)^-1 A1 and R = A1^T (A1 A1^T)^-1.
 * xi_out: device, same layout and size as xi_bar; must not alias it.
 * Asynchronous on `stream`. Errors: SF_ERR_INVALID_ARG for a malformed batch
 * or NULL output. */
sf_status sf_eq_project(sf_handle *h, void *stream, const sf_batch *batch, float *xi_out);

/* Adjoint of sf_eq_project: for dL/dxi_out = grad_out (device, xi_bar's
 * layout), grad_in = dL/dxi' = Pi grad_out (Pi is symmetric) and, when
 * grad_b is not NULL, grad_b[row][6] = dL/db = R^T grad_out per coefficient
 * row (sample, axis, robot), in the order of b above. The batch's xi_bar is
 * not read (it must still be a valid pointer). */
sf_status sf_eq_project_backward(sf_handle *h, void *stream, const sf_batch *batch, const float *grad_out,
                                 float *grad_in, float *grad_b);

/* Synchronises `stream` and returns any device-side error latched by earlier
 * calls on the handle (SF_ERR_TIMEOUT, SF_ERR_DEBUG_CHECK, SF_ERR_NONFINITE,
 * in this order of precedence), clearing it. */
sf_status sf_sync_status(sf_handle *h, void *stream);

/* Measurement, not part of the solver: throughput of the float32-lane pipes
 * that bound the fused forward, on device `device` (made current for the
 * call, restored after). Writes fused multiply-adds per second (an FMA
 * counts once; whole-GPU launch of 8 independent chains per thread, 2048
 * threads per SM, best of 5 CUDA-event-timed launches), reciprocal square
 * roots per second (the same on rsqrt), and the clock in MHz at which 128
 * lanes per SM, one FMA each per cycle, give the measured FMA rate.
 * Allocates and frees a few kB of device memory; synchronises the device.
 * SF_ERR_INVALID_ARG for a NULL output, SF_ERR_CUDA on a CUDA error. */
sf_status sf_lane_peaks(int device, double *fma_per_s, double *mufu_per_s, double *lane_mhz);

#ifdef __cplusplus
}
#endif
#endif
