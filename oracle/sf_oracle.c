/*
 * FP64 CPU oracle of the Swarm-Gen safety filter (arXiv 2501.19042).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark; never by the product path. Independent of
 * the CUDA library (no shared code, header or table).
 *
 * Every function restates one passage of the paper; the passage is named in
 * the comment above it. Compiled with -O2 -fno-fast-math -ffp-contract=off so
 * that each operation rounds once, in the order written.
 */
#include "sf_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Sec. II-B, Eq. (poly): the basis matrix W and its time derivatives.        */
/* The paper does not name the basis family; it is taken as Bernstein of the   */
/* given order on tau_j = j/(T-1), so row 0 is t = 0 and row T-1 is t = H.     */
/* d/dt = (1/H) d/dtau.                                                        */
/* ------------------------------------------------------------------------- */

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}

/* B_{k,n}(tau) = C(n,k) tau^k (1 - tau)^(n-k); zero outside 0 <= k <= n. */
static double bern(int n, int k, double tau) {
  if (n < 0 || k < 0 || k > n) return 0.0;
  return binom(n, k) * pow(tau, (double)k) * pow(1.0 - tau, (double)(n - k));
}

int oracle_basis(int order, int T, double t_final, double *P, double *Pd, double *Pdd) {
  if (order < 2 || T < 2 || !(t_final > 0.0)) return -1;
  const int n = order, nvar = order + 1;
  for (int j = 0; j < T; ++j) {
    const double tau = (double)j / (double)(T - 1);
    for (int k = 0; k < nvar; ++k) {
      P[j * nvar + k] = bern(n, k, tau);
      /* dB_{k,n}/dtau = n (B_{k-1,n-1} - B_{k,n-1}) */
      const double d1 = (double)n * (bern(n - 1, k - 1, tau) - bern(n - 1, k, tau));
      /* d2B_{k,n}/dtau2 = n (n-1) (B_{k-2,n-2} - 2 B_{k-1,n-2} + B_{k,n-2}) */
      const double d2 = (double)n * (double)(n - 1) *
                        (bern(n - 2, k - 2, tau) - 2.0 * bern(n - 2, k - 1, tau) +
                         bern(n - 2, k, tau));
      Pd[j * nvar + k] = d1 / t_final;
      Pdd[j * nvar + k] = d2 / (t_final * t_final);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Appendix, Eqs. (alpha_step), (beta_step), (d_step) on one block of the      */
/* polar form of Eq. (inter_agent_polar) / (workspace_polar):                  */
/*   delta = d (a cos(alpha) sin(beta), a sin(alpha) sin(beta), b cos(beta)).  */
/* For fixed d and beta, the AL term is smallest at alpha = atan2(dy, dx).     */
/* Given alpha, beta is taken in the scaled coordinates (delta_xy/a, dz/b),    */
/* which is the exact minimiser when a == b. Given alpha and beta the term is  */
/* a 1-D least squares in d, solved and clipped to [dmin, dmax].               */
/* Tie-break: a zero component enters atan2 as +0, so delta = 0 gives          */
/* alpha = beta = 0.                                                           */
/* ------------------------------------------------------------------------- */

static void polar_project(double a, double b, int dim, const double *delta, double dmin,
                          double dmax, double *e) {
  if (dim == 2) {
    const double dx = delta[0] + 0.0, dy = delta[1] + 0.0;
    const double alpha = atan2(dy, dx);
    const double ca = cos(alpha), sa = sin(alpha);
    double d = (a * ca * dx + a * sa * dy) / (a * a);
    if (d < dmin) d = dmin;
    if (d > dmax) d = dmax;
    e[0] = d * a * ca;
    e[1] = d * a * sa;
    return;
  }
  const double dx = delta[0] + 0.0, dy = delta[1] + 0.0, dz = delta[2] + 0.0;
  const double alpha = atan2(dy, dx);
  const double ca = cos(alpha), sa = sin(alpha);
  const double u = dx * ca + dy * sa;
  const double beta = atan2(u / a + 0.0, dz / b + 0.0);
  const double cb = cos(beta), sb = sin(beta);
  const double num = a * ca * sb * dx + a * sa * sb * dy + b * cb * dz;
  const double den = a * a * sb * sb + b * b * cb * cb;
  double d = num / den;
  if (d < dmin) d = dmin;
  if (d > dmax) d = dmax;
  e[0] = d * a * ca * sb;
  e[1] = d * a * sa * sb;
  e[2] = d * b * cb;
}

void oracle_pair_project(double a, double b, int dim, const double *delta, double *e) {
  polar_project(a, b, dim, delta, 1.0, INFINITY, e);
}

void oracle_ball_project(double r, int dim, const double *v, double *e) {
  polar_project(r, r, dim, v, 0.0, 1.0, e);
}

void oracle_spheroid_in_project(double a, double b, int dim, const double *c, const double *p,
                                double *e) {
  double rel[3], er[3];
  for (int x = 0; x < dim; ++x) rel[x] = p[x] - c[x];
  polar_project(a, b, dim, rel, 0.0, 1.0, er);
  for (int x = 0; x < dim; ++x) e[x] = c[x] + er[x];
}

/* ------------------------------------------------------------------------- */
/* Appendix, Eq. (oracle_am_step): one fixed-point iteration f_FP.             */
/* Readings: the lambda step is taken with the minus sign, which is the dual   */
/* ascent step for the -<lambda, xi> term of Eq. (aug_lag) and the eta of the  */
/* xi step; the printed plus sign diverges. The lambda step uses the old xi    */
/* and the new e, as printed. The xi step solves the KKT system                */
/* [[I + rho F^T F, A^T], [A, 0]] [xi; nu] = [rho F^T e + lambda + xi_bar; b]. */
/* ------------------------------------------------------------------------- */

void oracle_am_step(const oracle_am_ops *ops, double rho, const double *xi_bar, double *xi,
                    double *lam, double *e_out, double *work, double *proj_res2) {
  const int n = ops->n, m = ops->m;
  double *Fx = work;          /* m */
  double *e = work + m;       /* m */
  double *t = work + 2 * m;   /* n */
  ops->apply_F(ops->ctx, xi, Fx);
  ops->project(ops->ctx, Fx, e);                    /* alpha, beta, d steps */
  double r2 = 0.0;
  for (int r = 0; r < m; ++r) {
    const double q = Fx[r] - e[r];
    r2 += q * q;
    Fx[r] = q;                                      /* F xi^k - e^{k+1} */
  }
  if (proj_res2) *proj_res2 = r2;
  ops->apply_Ft(ops->ctx, Fx, t);
  for (int i = 0; i < n; ++i) lam[i] = lam[i] - rho * t[i];   /* lambda step */
  ops->apply_Ft(ops->ctx, e, t);
  for (int i = 0; i < n; ++i) t[i] = rho * t[i] + lam[i] + xi_bar[i];  /* eta */
  ops->solve_xi(ops->ctx, t, xi);                   /* xi step */
  if (e_out) memcpy(e_out, e, sizeof(double) * (size_t)m);
}

/* ------------------------------------------------------------------------- */
/* The SF instance: F of the Appendix (Eqs. reform_*, f_e), A and b of        */
/* Eq. (boundary_con), and the dense KKT of the xi step, factored once.        */
/* ------------------------------------------------------------------------- */

struct oracle_sf {
  oracle_problem pb;
  int nvar, npair, rows_ax, n, m;
  int off_v, off_a, off_w;          /* row offsets of the blocks in one axis */
  int *pi, *pj;                     /* pair list, (0,1), (0,2), ..., (N-2,N-1) */
  double *P, *Pd, *Pdd;             /* [T][nvar] */
  double *A1;                       /* [6][nvar]: rows P_0, Pd_0, Pdd_0, P_H, Pd_H, Pdd_H */
  double *b;                        /* [dim][N][6] */
  int kdim;                         /* N*nvar + 6N */
  double *LU;                       /* kdim x kdim, row-major, with piv */
  int *piv;
};

int oracle_rows_per_axis(const oracle_problem *pb) {
  const int N = pb->n_robots, T = pb->T;
  int rows = N * (N - 1) / 2 * T;
  if (pb->v_max > 0.0) rows += N * T;
  if (pb->a_max > 0.0) rows += N * T;
  if (pb->use_workspace) rows += N * T;
  return rows;
}

/* F of one axis applied to that axis' coefficients c [N][nvar] -> y [rows_ax].
 * Pair row (p, t) is e_i - e_j of robot pair p = (i, j), times P row t
 * (F_o of the Appendix); the velocity, acceleration and workspace rows are
 * I (x) Pd, I (x) Pdd and I (x) P (F_w of the Appendix). */
static void F_axis(const oracle_sf *s, const double *c, double *y) {
  const int T = s->pb.T, nv = s->nvar, N = s->pb.n_robots;
  for (int p = 0; p < s->npair; ++p) {
    const double *ci = c + s->pi[p] * nv, *cj = c + s->pj[p] * nv;
    for (int t = 0; t < T; ++t) {
      double acc = 0.0;
      for (int k = 0; k < nv; ++k) acc += s->P[t * nv + k] * (ci[k] - cj[k]);
      y[p * T + t] = acc;
    }
  }
  for (int i = 0; i < N; ++i) {
    const double *ci = c + i * nv;
    for (int t = 0; t < T; ++t) {
      double pv = 0.0, pa = 0.0, pp = 0.0;
      for (int k = 0; k < nv; ++k) {
        pv += s->Pd[t * nv + k] * ci[k];
        pa += s->Pdd[t * nv + k] * ci[k];
        pp += s->P[t * nv + k] * ci[k];
      }
      if (s->off_v >= 0) y[s->off_v + i * T + t] = pv;
      if (s->off_a >= 0) y[s->off_a + i * T + t] = pa;
      if (s->off_w >= 0) y[s->off_w + i * T + t] = pp;
    }
  }
}

/* F^T of one axis: y [rows_ax] -> c [N][nvar]. */
static void Ft_axis(const oracle_sf *s, const double *y, double *c) {
  const int T = s->pb.T, nv = s->nvar, N = s->pb.n_robots;
  for (int i = 0; i < N * nv; ++i) c[i] = 0.0;
  for (int p = 0; p < s->npair; ++p) {
    double *ci = c + s->pi[p] * nv, *cj = c + s->pj[p] * nv;
    for (int t = 0; t < T; ++t) {
      const double v = y[p * T + t];
      for (int k = 0; k < nv; ++k) {
        ci[k] += s->P[t * nv + k] * v;
        cj[k] -= s->P[t * nv + k] * v;
      }
    }
  }
  for (int i = 0; i < N; ++i) {
    double *ci = c + i * nv;
    for (int t = 0; t < T; ++t) {
      for (int k = 0; k < nv; ++k) {
        if (s->off_v >= 0) ci[k] += s->Pd[t * nv + k] * y[s->off_v + i * T + t];
        if (s->off_a >= 0) ci[k] += s->Pdd[t * nv + k] * y[s->off_a + i * T + t];
        if (s->off_w >= 0) ci[k] += s->P[t * nv + k] * y[s->off_w + i * T + t];
      }
    }
  }
}

static void sf_apply_F(void *ctx, const double *xi, double *Fx) {
  const oracle_sf *s = (const oracle_sf *)ctx;
  const int per_ax = s->pb.n_robots * s->nvar;
  for (int ax = 0; ax < s->pb.dim; ++ax) F_axis(s, xi + ax * per_ax, Fx + ax * s->rows_ax);
}

static void sf_apply_Ft(void *ctx, const double *y, double *xi) {
  const oracle_sf *s = (const oracle_sf *)ctx;
  const int per_ax = s->pb.n_robots * s->nvar;
  for (int ax = 0; ax < s->pb.dim; ++ax) Ft_axis(s, y + ax * s->rows_ax, xi + ax * per_ax);
}

/* alpha, beta, d steps over all blocks: every row group gathers its dim
 * components (one per axis block of F) and is projected as one vector. */
static void sf_project(void *ctx, const double *Fx, double *e) {
  const oracle_sf *s = (const oracle_sf *)ctx;
  const int dim = s->pb.dim, T = s->pb.T, N = s->pb.n_robots, R = s->rows_ax;
  double v[3], ev[3];
  for (int r = 0; r < s->npair * T; ++r) {
    for (int x = 0; x < dim; ++x) v[x] = Fx[x * R + r];
    oracle_pair_project(s->pb.coll_a, s->pb.coll_b, dim, v, ev);
    for (int x = 0; x < dim; ++x) e[x * R + r] = ev[x];
  }
  for (int r = 0; r < N * T; ++r) {
    if (s->off_v >= 0) {
      for (int x = 0; x < dim; ++x) v[x] = Fx[x * R + s->off_v + r];
      oracle_ball_project(s->pb.v_max, dim, v, ev);
      for (int x = 0; x < dim; ++x) e[x * R + s->off_v + r] = ev[x];
    }
    if (s->off_a >= 0) {
      for (int x = 0; x < dim; ++x) v[x] = Fx[x * R + s->off_a + r];
      oracle_ball_project(s->pb.a_max, dim, v, ev);
      for (int x = 0; x < dim; ++x) e[x * R + s->off_a + r] = ev[x];
    }
    if (s->off_w >= 0) {
      for (int x = 0; x < dim; ++x) v[x] = Fx[x * R + s->off_w + r];
      oracle_spheroid_in_project(s->pb.ws_a, s->pb.ws_b, dim, s->pb.ws_center, v, ev);
      for (int x = 0; x < dim; ++x) e[x * R + s->off_w + r] = ev[x];
    }
  }
}

/* LU with partial pivoting (Doolittle), in place. Returns -1 if singular. */
static int lu_factor(double *M, int n, int *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(M[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(M[i * n + k]) > best) { best = fabs(M[i * n + k]); p = i; }
    if (best == 0.0) return -1;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) { double tmp = M[k * n + j]; M[k * n + j] = M[p * n + j]; M[p * n + j] = tmp; }
    for (int i = k + 1; i < n; ++i) {
      const double l = M[i * n + k] / M[k * n + k];
      M[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) M[i * n + j] -= l * M[k * n + j];
    }
  }
  return 0;
}

static void lu_solve(const double *LU, int n, const int *piv, double *x) {
  for (int k = 0; k < n; ++k) {
    const int p = piv[k];
    if (p != k) { double tmp = x[k]; x[k] = x[p]; x[p] = tmp; }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) x[i] -= LU[i * n + j] * x[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) x[i] -= LU[i * n + j] * x[j];
    x[i] /= LU[i * n + i];
  }
}

/* Builds [[I + rho F_ax^T F_ax, A_ax^T], [A_ax, 0]] for one axis (the same for
 * every axis). F_ax^T F_ax is assembled column by column from F_ax and F_ax^T
 * applied to unit vectors, i.e. from the definition of F. */
static void build_kkt(const oracle_sf *s, double *K) {
  const int N = s->pb.n_robots, nv = s->nvar, nc = N * nv, kd = s->kdim;
  memset(K, 0, sizeof(double) * (size_t)kd * (size_t)kd);
  double *unit = (double *)calloc((size_t)nc, sizeof(double));
  double *y = (double *)malloc(sizeof(double) * (size_t)s->rows_ax);
  double *col = (double *)malloc(sizeof(double) * (size_t)nc);
  for (int c = 0; c < nc; ++c) {
    unit[c] = 1.0;
    F_axis(s, unit, y);
    Ft_axis(s, y, col);
    unit[c] = 0.0;
    for (int r = 0; r < nc; ++r) K[r * kd + c] = s->pb.rho * col[r] + (r == c ? 1.0 : 0.0);
  }
  for (int i = 0; i < N; ++i)
    for (int q = 0; q < 6; ++q)
      for (int k = 0; k < nv; ++k) {
        const int row = nc + i * 6 + q, cc = i * nv + k;
        K[row * kd + cc] = s->A1[q * nv + k];
        K[cc * kd + row] = s->A1[q * nv + k];
      }
  free(unit); free(y); free(col);
}

/* xi step: per axis, solve the KKT system with right-hand side [rhs_ax; b_ax]
 * and keep the xi part. */
static void sf_solve_xi(void *ctx, const double *rhs, double *xi) {
  const oracle_sf *s = (const oracle_sf *)ctx;
  const int N = s->pb.n_robots, nv = s->nvar, nc = N * nv, kd = s->kdim;
  double *x = (double *)malloc(sizeof(double) * (size_t)kd);
  for (int ax = 0; ax < s->pb.dim; ++ax) {
    memcpy(x, rhs + ax * nc, sizeof(double) * (size_t)nc);
    for (int i = 0; i < N; ++i)
      for (int q = 0; q < 6; ++q) x[nc + i * 6 + q] = s->b[(ax * N + i) * 6 + q];
    lu_solve(s->LU, kd, s->piv, x);
    memcpy(xi + ax * nc, x, sizeof(double) * (size_t)nc);
  }
  free(x);
}

oracle_sf *oracle_sf_create(const oracle_problem *pb, const double *start, const double *goal,
                            const double *start_va, const double *goal_va) {
  if (!pb || (pb->dim != 2 && pb->dim != 3) || pb->n_robots < 1 || pb->order < 2 || pb->T < 2 ||
      !(pb->t_final > 0) || !(pb->rho > 0) || !(pb->coll_a > 0) || !(pb->coll_b > 0))
    return NULL;
  oracle_sf *s = (oracle_sf *)calloc(1, sizeof(oracle_sf));
  s->pb = *pb;
  const int N = pb->n_robots, T = pb->T, dim = pb->dim;
  s->nvar = pb->order + 1;
  s->npair = N * (N - 1) / 2;
  int off = s->npair * T;
  s->off_v = s->off_a = s->off_w = -1;
  if (pb->v_max > 0.0) { s->off_v = off; off += N * T; }
  if (pb->a_max > 0.0) { s->off_a = off; off += N * T; }
  if (pb->use_workspace) { s->off_w = off; off += N * T; }
  s->rows_ax = off;
  s->n = dim * N * s->nvar;
  s->m = dim * s->rows_ax;
  s->pi = (int *)malloc(sizeof(int) * (size_t)(s->npair > 0 ? s->npair : 1));
  s->pj = (int *)malloc(sizeof(int) * (size_t)(s->npair > 0 ? s->npair : 1));
  int p = 0;
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) { s->pi[p] = i; s->pj[p] = j; ++p; }
  const int nv = s->nvar;
  s->P = (double *)malloc(sizeof(double) * (size_t)(T * nv));
  s->Pd = (double *)malloc(sizeof(double) * (size_t)(T * nv));
  s->Pdd = (double *)malloc(sizeof(double) * (size_t)(T * nv));
  oracle_basis(pb->order, T, pb->t_final, s->P, s->Pd, s->Pdd);
  /* Eq. (boundary_con): (p, pdot, pddot) at t = 0 and t = H. The paper prints
   * (p, pddot, pddot) at H; read as (p, pdot, pddot). */
  s->A1 = (double *)malloc(sizeof(double) * (size_t)(6 * nv));
  for (int k = 0; k < nv; ++k) {
    s->A1[0 * nv + k] = s->P[k];
    s->A1[1 * nv + k] = s->Pd[k];
    s->A1[2 * nv + k] = s->Pdd[k];
    s->A1[3 * nv + k] = s->P[(T - 1) * nv + k];
    s->A1[4 * nv + k] = s->Pd[(T - 1) * nv + k];
    s->A1[5 * nv + k] = s->Pdd[(T - 1) * nv + k];
  }
  s->b = (double *)malloc(sizeof(double) * (size_t)(dim * N * 6));
  for (int ax = 0; ax < dim; ++ax)
    for (int i = 0; i < N; ++i) {
      double *bb = s->b + (ax * N + i) * 6;
      bb[0] = start[i * dim + ax];
      bb[1] = start_va ? start_va[(i * 2 + 0) * dim + ax] : 0.0;
      bb[2] = start_va ? start_va[(i * 2 + 1) * dim + ax] : 0.0;
      bb[3] = goal[i * dim + ax];
      bb[4] = goal_va ? goal_va[(i * 2 + 0) * dim + ax] : 0.0;
      bb[5] = goal_va ? goal_va[(i * 2 + 1) * dim + ax] : 0.0;
    }
  s->kdim = N * nv + 6 * N;
  s->LU = (double *)malloc(sizeof(double) * (size_t)s->kdim * (size_t)s->kdim);
  s->piv = (int *)malloc(sizeof(int) * (size_t)s->kdim);
  build_kkt(s, s->LU);
  if (lu_factor(s->LU, s->kdim, s->piv) != 0) { oracle_sf_destroy(s); return NULL; }
  return s;
}

void oracle_sf_destroy(oracle_sf *s) {
  if (!s) return;
  free(s->pi); free(s->pj); free(s->P); free(s->Pd); free(s->Pdd);
  free(s->A1); free(s->b); free(s->LU); free(s->piv);
  free(s);
}

void oracle_sf_ops(oracle_sf *s, oracle_am_ops *ops) {
  ops->n = s->n;
  ops->m = s->m;
  ops->ctx = s;
  ops->apply_F = sf_apply_F;
  ops->apply_Ft = sf_apply_Ft;
  ops->project = sf_project;
  ops->solve_xi = sf_solve_xi;
}

int oracle_sf_dense_F(oracle_sf *s, double *F) {
  if ((double)s->m * (double)s->n > 67108864.0) return -1;
  double *unit = (double *)calloc((size_t)s->n, sizeof(double));
  double *col = (double *)malloc(sizeof(double) * (size_t)s->m);
  for (int c = 0; c < s->n; ++c) {
    unit[c] = 1.0;
    sf_apply_F(s, unit, col);
    unit[c] = 0.0;
    for (int r = 0; r < s->m; ++r) F[(size_t)r * (size_t)s->n + (size_t)c] = col[r];
  }
  free(unit); free(col);
  return 0;
}

void oracle_sf_dense_A(oracle_sf *s, double *A, double *b) {
  const int N = s->pb.n_robots, nv = s->nvar, dim = s->pb.dim, n = s->n;
  memset(A, 0, sizeof(double) * (size_t)(dim * N * 6) * (size_t)n);
  for (int ax = 0; ax < dim; ++ax)
    for (int i = 0; i < N; ++i)
      for (int q = 0; q < 6; ++q) {
        const int row = (ax * N + i) * 6 + q;
        for (int k = 0; k < nv; ++k) A[(size_t)row * n + (ax * N + i) * nv + k] = s->A1[q * nv + k];
        b[row] = s->b[row];
      }
}

/* ------------------------------------------------------------------------- */
/* The differentiable QP layer of the generative decoders (Sec. III-A / B:     */
/* Eq. (sf_form) without the inequality constraints): the Euclidean           */
/* projection of xi' onto {xi : A xi = b}, i.e. the solution of               */
/*   [[I, A^T], [A, 0]] [xi; nu] = [xi'; b].                                   */
/* A is block diagonal with the 6 x nvar block A1 per (axis, robot), so the    */
/* system is solved per block with the oracle's own LU (not the closed form).  */
/* The adjoint of xi' -> xi is the same solve with right-hand side [g; 0]:     */
/* the KKT matrix is symmetric, so its inverse maps [g; 0] to                 */
/* [dL/dxi'; dL/db].                                                           */
/* ------------------------------------------------------------------------- */

static int eq_block_solve(const oracle_sf *s, const double *top, const double *bot, double *x_out,
                          double *nu_out) {
  const int nv = s->nvar, kd = nv + 6;
  double *K = (double *)calloc((size_t)kd * kd, sizeof(double));
  double *r = (double *)malloc(sizeof(double) * (size_t)kd);
  int *piv = (int *)malloc(sizeof(int) * (size_t)kd);
  for (int k = 0; k < nv; ++k) K[k * kd + k] = 1.0;
  for (int q = 0; q < 6; ++q)
    for (int k = 0; k < nv; ++k) {
      K[(nv + q) * kd + k] = s->A1[q * nv + k];
      K[k * kd + nv + q] = s->A1[q * nv + k];
    }
  for (int k = 0; k < nv; ++k) r[k] = top[k];
  for (int q = 0; q < 6; ++q) r[nv + q] = bot ? bot[q] : 0.0;
  const int rc = lu_factor(K, kd, piv);
  if (rc == 0) {
    lu_solve(K, kd, piv, r);
    for (int k = 0; k < nv; ++k) x_out[k] = r[k];
    if (nu_out)
      for (int q = 0; q < 6; ++q) nu_out[q] = r[nv + q];
  }
  free(K); free(r); free(piv);
  return rc;
}

int oracle_eq_project(oracle_sf *s, const double *xi_in, double *xi_out) {
  const int N = s->pb.n_robots, nv = s->nvar, dim = s->pb.dim;
  for (int ax = 0; ax < dim; ++ax)
    for (int i = 0; i < N; ++i) {
      const int o = (ax * N + i) * nv;
      if (eq_block_solve(s, xi_in + o, s->b + (ax * N + i) * 6, xi_out + o, NULL) != 0) return -1;
    }
  return 0;
}

int oracle_eq_project_adjoint(oracle_sf *s, const double *g, double *g_in, double *g_b) {
  const int N = s->pb.n_robots, nv = s->nvar, dim = s->pb.dim;
  for (int ax = 0; ax < dim; ++ax)
    for (int i = 0; i < N; ++i) {
      const int o = (ax * N + i) * nv;
      if (eq_block_solve(s, g + o, NULL, g_in + o, g_b ? g_b + (ax * N + i) * 6 : NULL) != 0) return -1;
    }
  return 0;
}

int oracle_sf_kkt_size(oracle_sf *s) { return s->kdim; }

void oracle_sf_kkt_matrix(oracle_sf *s, double *K) { build_kkt(s, K); }

/* Largest constraint violation of the trajectories of xi: pairs by the
 * ellipsoidal form of Eq. (inter_robot_con) written as a distance
 * (1 - ||M_a^-1 delta||) * min(a, b), velocity / acceleration by how far the
 * norm exceeds the bound, workspace by Eq. (workspace_con) likewise. */
static double violation(const oracle_sf *s, const double *Fx) {
  const int dim = s->pb.dim, T = s->pb.T, N = s->pb.n_robots, R = s->rows_ax;
  const double a = s->pb.coll_a, b = s->pb.coll_b;
  const double scale = a < b ? a : b;
  double worst = 0.0;
  for (int r = 0; r < s->npair * T; ++r) {
    double q = 0.0;
    for (int x = 0; x < dim; ++x) {
      const double v = Fx[x * R + r] / (x == 2 ? b : a);
      q += v * v;
    }
    const double g = (1.0 - sqrt(q)) * scale;
    if (g > worst) worst = g;
  }
  for (int r = 0; r < N * T; ++r) {
    if (s->off_v >= 0) {
      double q = 0.0;
      for (int x = 0; x < dim; ++x) q += Fx[x * R + s->off_v + r] * Fx[x * R + s->off_v + r];
      if (sqrt(q) - s->pb.v_max > worst) worst = sqrt(q) - s->pb.v_max;
    }
    if (s->off_a >= 0) {
      double q = 0.0;
      for (int x = 0; x < dim; ++x) q += Fx[x * R + s->off_a + r] * Fx[x * R + s->off_a + r];
      if (sqrt(q) - s->pb.a_max > worst) worst = sqrt(q) - s->pb.a_max;
    }
    if (s->off_w >= 0) {
      double q = 0.0;
      for (int x = 0; x < dim; ++x) {
        const double v = (Fx[x * R + s->off_w + r] - s->pb.ws_center[x]) /
                         (x == 2 ? s->pb.ws_b : s->pb.ws_a);
        q += v * v;
      }
      const double g = (sqrt(q) - 1.0) * (s->pb.ws_a < s->pb.ws_b ? s->pb.ws_a : s->pb.ws_b);
      if (g > worst) worst = g;
    }
  }
  return worst;
}

int oracle_sf_run(oracle_sf *s, const double *xi_bar, const double *xi0, const double *lam0,
                  int K, double *xi_out, double *lam_out, double *rp_hist, double *proj_hist,
                  double *viol) {
  if (!s || K < 0) return -1;
  oracle_am_ops ops;
  oracle_sf_ops(s, &ops);
  const int n = ops.n, m = ops.m;
  double *xi = (double *)malloc(sizeof(double) * (size_t)n);
  double *lam = (double *)malloc(sizeof(double) * (size_t)n);
  double *work = (double *)malloc(sizeof(double) * (size_t)(2 * m + n));
  double *e = (double *)malloc(sizeof(double) * (size_t)m);
  double *Fx = (double *)malloc(sizeof(double) * (size_t)m);
  memcpy(xi, xi0 ? xi0 : xi_bar, sizeof(double) * (size_t)n);
  if (lam0) memcpy(lam, lam0, sizeof(double) * (size_t)n);
  else memset(lam, 0, sizeof(double) * (size_t)n);
  for (int k = 0; k < K; ++k) {
    double pr2 = 0.0;
    oracle_am_step(&ops, s->pb.rho, xi_bar, xi, lam, e, work, &pr2);
    if (proj_hist) proj_hist[k] = sqrt(pr2);
    if (rp_hist) {
      /* Eq. (primal_residual): r_p = F xi^{k+1} - e(alpha^{k+1}, beta^{k+1}, d^{k+1}). */
      sf_apply_F(s, xi, Fx);
      double r2 = 0.0;
      for (int r = 0; r < m; ++r) { const double q = Fx[r] - e[r]; r2 += q * q; }
      rp_hist[k] = sqrt(r2);
    }
  }
  if (viol) {
    sf_apply_F(s, xi, Fx);
    *viol = violation(s, Fx);
  }
  if (xi_out) memcpy(xi_out, xi, sizeof(double) * (size_t)n);
  if (lam_out) memcpy(lam_out, lam, sizeof(double) * (size_t)n);
  free(xi); free(lam); free(work); free(e); free(Fx);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Batch entry point: samples are independent, so they are spread over threads. */
/* ------------------------------------------------------------------------- */

typedef struct {
  oracle_sf *s;
  int S, K, n;
  const double *xi_bar, *xi0, *lam0;
  double *xi_out, *lam_out, *rp_final, *rp_hist, *proj_hist;
  int next;
  pthread_mutex_t mu;
  int err;
} batch_job;

static void *batch_worker(void *arg) {
  batch_job *job = (batch_job *)arg;
  double *rp = (double *)malloc(sizeof(double) * (size_t)(job->K > 0 ? job->K : 1));
  for (;;) {
    pthread_mutex_lock(&job->mu);
    const int i = job->next++;
    pthread_mutex_unlock(&job->mu);
    if (i >= job->S) break;
    const size_t o = (size_t)i * (size_t)job->n;
    const int rc = oracle_sf_run(job->s, job->xi_bar + o, job->xi0 ? job->xi0 + o : NULL,
                                 job->lam0 ? job->lam0 + o : NULL, job->K,
                                 job->xi_out ? job->xi_out + o : NULL,
                                 job->lam_out ? job->lam_out + o : NULL, rp,
                                 job->proj_hist ? job->proj_hist + (size_t)i * job->K : NULL, NULL);
    if (rc) job->err = rc;
    if (job->rp_final) job->rp_final[i] = job->K > 0 ? rp[job->K - 1] : 0.0;
    if (job->rp_hist) memcpy(job->rp_hist + (size_t)i * job->K, rp, sizeof(double) * (size_t)job->K);
  }
  free(rp);
  return NULL;
}

int oracle_sf_run_batch(const oracle_problem *pb, const double *start, const double *goal,
                        const double *start_va, const double *goal_va, int S,
                        const double *xi_bar, const double *xi0, const double *lam0, int K,
                        double *xi_out, double *lam_out, double *rp_final, double *rp_hist,
                        double *proj_hist, int n_threads) {
  oracle_sf *s = oracle_sf_create(pb, start, goal, start_va, goal_va);
  if (!s) return -1;
  batch_job job;
  memset(&job, 0, sizeof(job));
  job.s = s; job.S = S; job.K = K; job.n = s->n;
  job.xi_bar = xi_bar; job.xi0 = xi0; job.lam0 = lam0;
  job.xi_out = xi_out; job.lam_out = lam_out; job.rp_final = rp_final;
  job.rp_hist = rp_hist; job.proj_hist = proj_hist;
  pthread_mutex_init(&job.mu, NULL);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > S) n_threads = S > 0 ? S : 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, batch_worker, &job);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&job.mu);
  oracle_sf_destroy(s);
  return job.err;
}
