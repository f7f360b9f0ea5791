/*
 * FP64 CPU oracle of the Swarm-Gen safety filter (SF), arXiv 2501.19042.
 *
 * TEST INFRASTRUCTURE ONLY. This library is the plain, slow, obviously
 * correct restatement of the paper's fixed-point solver that the CUDA path is
 * checked against. Only the test suite, the smoke check and the CPU baseline
 * leg of the benchmark may load it. It shares no code, header, table or
 * constant with the CUDA library, and it never calls it.
 *
 * What it follows (paper sections / equations):
 *   - Sec. II-B, Eq. (poly): p = W c per robot and axis; W is taken as the
 *     Bernstein basis of the given order on the grid tau_j = j/(T-1).
 *   - Sec. II-A, Eq. (boundary_con): position, velocity and acceleration of
 *     every robot fixed at t=0 and t=H (the rows of A, b).
 *   - Appendix, Eqs. (inter_agent_polar), (workspace_polar), (reform_*),
 *     (f_e): the constraints rewritten as F xi = e(alpha, beta, d) with
 *     d in [d_min, d_max]; velocity and acceleration bounds use the same
 *     polar form with centre 0 and 0 <= d <= 1.
 *   - Appendix, Eq. (aug_lag) and the AM steps (alpha_step), (beta_step),
 *     (d_step), (lambda_step), (xi_step): one fixed-point iteration f_FP.
 *   - Appendix, Eq. (primal_residual): r_p = F xi^{k+1} - e^{k+1}.
 *
 * Readings taken where the paper is garbled or silent are listed in the
 * repository design notes; the ones that change arithmetic are repeated next
 * to the code that implements them in sf_oracle.c.
 *
 * Layouts (row-major, double):
 *   xi, lambda, xi_bar : [dim][N][nvar]     (paper Sec. II-B, the xi vector)
 *   start, goal        : [N][dim]           positions
 *   start_va, goal_va  : [N][2][dim]        (velocity, acceleration); NULL = 0
 *   P, Pd, Pdd         : [T][nvar]
 */
#ifndef SF_ORACLE_H
#define SF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim;            /* 2 or 3 */
  int n_robots;       /* N >= 1 */
  int order;          /* Bernstein order; nvar = order + 1 */
  int T;              /* time steps, tau_j = j / (T - 1), T >= 2 */
  double t_final;     /* horizon H in seconds */
  double rho;         /* augmented-Lagrangian weight, Eq. (aug_lag) */
  double coll_a;      /* collision semi-axes (a, a, b), Eq. (inter_robot_con) */
  double coll_b;
  double v_max;       /* <= 0 disables the velocity block */
  double a_max;       /* <= 0 disables the acceleration block */
  int use_workspace;  /* Eq. (workspace_con); 0 = off */
  double ws_center[3];
  double ws_a, ws_b;
} oracle_problem;

/* Generic operator set for one AM / fixed-point iteration on a flat problem:
 * xi has n entries, F has m rows. Used by the SF and by small hand-made
 * instances in the tests. */
typedef struct {
  int n, m;
  void *ctx;
  void (*apply_F)(void *ctx, const double *xi, double *Fxi);        /* m <- n */
  void (*apply_Ft)(void *ctx, const double *y, double *out);        /* n <- m */
  void (*project)(void *ctx, const double *Fxi, double *e);         /* alpha, beta, d steps */
  void (*solve_xi)(void *ctx, const double *rhs, double *xi);       /* xi-step: KKT solve */
} oracle_am_ops;

/* One iteration of f_FP (Appendix, AM steps):
 *   e    <- project(F xi)                     alpha, beta, d steps
 *   lam  <- lam - rho F^T (F xi - e)          lambda step (sign reading)
 *   xi   <- solve(rho F^T e + lam + xi_bar)   xi step with eta of the paper
 * e_out (m entries, may be NULL) receives e; work needs 2*m + n doubles.
 * proj_res2 (may be NULL) receives ||F xi_old - e||^2. */
void oracle_am_step(const oracle_am_ops *ops, double rho, const double *xi_bar,
                    double *xi, double *lam, double *e_out, double *work,
                    double *proj_res2);

/* Bernstein basis and its time derivatives, [T][order+1] each. */
int oracle_basis(int order, int T, double t_final, double *P, double *Pd, double *Pdd);

/* Closed-form alpha/beta/d step for one pair block (Eq. inter_agent_polar):
 * delta, e have dim entries; d is clipped to [1, inf). */
void oracle_pair_project(double a, double b, int dim, const double *delta, double *e);
/* Same polar form with centre 0, semi-axes (r, r, r) and d in [0, 1]. */
void oracle_ball_project(double r, int dim, const double *v, double *e);
/* Workspace spheroid (Eq. workspace_polar): centre c, semi-axes (a, a, b), d in [0, 1]. */
void oracle_spheroid_in_project(double a, double b, int dim, const double *c,
                                const double *p, double *e);

/* Rows of F for one axis block (pairs, then velocity, then acceleration, then
 * workspace rows), given the problem. */
int oracle_rows_per_axis(const oracle_problem *pb);

/* Opaque SF context: basis, A, b, dense KKT factor, scratch. */
typedef struct oracle_sf oracle_sf;
oracle_sf *oracle_sf_create(const oracle_problem *pb, const double *start, const double *goal,
                            const double *start_va, const double *goal_va);
void oracle_sf_destroy(oracle_sf *s);
/* The operator set of this SF instance (n = dim*N*nvar, m = dim*rows_per_axis). */
void oracle_sf_ops(oracle_sf *s, oracle_am_ops *ops);
/* Dense explicit F (m x n, row-major) built row by row from its definition;
 * only for small problems (returns -1 if m*n > 2^26). */
int oracle_sf_dense_F(oracle_sf *s, double *F);
/* Dense A (dim*N*6 x n) and b (dim*N*6). Row order [axis][robot][6]. */
void oracle_sf_dense_A(oracle_sf *s, double *A, double *b);
/* The KKT matrix of one axis, [[I + rho F_ax^T F_ax, A_ax^T], [A_ax, 0]], size
 * (N*nvar + 6N)^2, as factored by the oracle. */
/* QP layer of the decoders (Sec. III-A / B): xi_out = argmin ||xi - xi_in||^2
 * subject to A xi = b (boundary conditions of every robot); layout
 * [dim][N][nvar]. The adjoint maps dL/dxi_out = g to dL/dxi_in (g_in) and
 * dL/db (g_b, [dim][N][6], may be NULL). Return 0, or -1 on a singular block. */
int oracle_eq_project(oracle_sf *s, const double *xi_in, double *xi_out);
int oracle_eq_project_adjoint(oracle_sf *s, const double *g, double *g_in, double *g_b);
int oracle_sf_kkt_size(oracle_sf *s);
void oracle_sf_kkt_matrix(oracle_sf *s, double *K);

/* Run K iterations from (xi0, lam0) for one sample.
 *   xi0 == NULL  -> xi0 = xi_bar (sample init); lam0 == NULL -> 0.
 *   rp_hist[k]   = ||F xi^{k+1} - e^{k+1}||_2         (Eq. primal_residual)
 *   proj_hist[k] = ||F xi^{k}   - e^{k+1}||_2         (projection residual)
 *   viol         = max over rows of the constraint violation of xi^K
 *                  (a - ||delta|| for pairs with a == b, ||v|| - v_max, ...)
 * Any output pointer may be NULL. Returns 0 on success. */
int oracle_sf_run(oracle_sf *s, const double *xi_bar, const double *xi0, const double *lam0,
                  int K, double *xi_out, double *lam_out, double *rp_hist,
                  double *proj_hist, double *viol);

/* Batch entry point over S independent samples of one scene, on n_threads POSIX
 * threads (each sample gets its own context; arithmetic is unchanged).
 * Arrays are per-sample concatenations of the single-sample layouts. xi0 and
 * lam0 may be NULL. rp_final[s] = rp_hist[K-1] of sample s. */
int oracle_sf_run_batch(const oracle_problem *pb, const double *start, const double *goal,
                        const double *start_va, const double *goal_va, int S,
                        const double *xi_bar, const double *xi0, const double *lam0, int K,
                        double *xi_out, double *lam_out, double *rp_final,
                        double *rp_hist /* [S][K] or NULL */,
                        double *proj_hist /* [S][K] or NULL */, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
