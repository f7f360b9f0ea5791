"""Shared helpers of the tests: one seeded workload fed to both the FP64
oracle and the CUDA path, and the comparison metrics."""
from __future__ import annotations

import numpy as np

import swarm_inputs as si

RHO_2D = 0.3   # rho selected for the 2D N=4 workload
RHO_3D = 0.1   # rho selected for the 3D workloads

# tolerances (float32 path vs float64 oracle after K iterations)
TOL_XI_REL = 1e-4     # relative L2 of the coefficients, per sample
TOL_RESID_ABS = 1e-3  # |final ||r_p|| difference|, metres
# lambda^K: error per sample in units of the coefficient scale,
# ||lambda - lambda_ref|| / ||xi_ref||. lambda enters the xi step additively
# beside xi_bar (eta = rho F^T e + lambda + xi_bar, Eq. xi_step), so an error
# of that size moves the step's right-hand side by the same amount that the
# xi tolerance allows in xi; it is therefore held to the xi bound of each
# mode. (Relative to ||lambda_ref|| itself the bound would be undefined for
# samples whose constraints never activate, where lambda stays 0.)
TOL_LAM = TOL_XI_REL


def oracle_problem(O, spec: si.SceneSpec, rho: float, N: int | None = None, coll_b: float | None = None):
    """coll_b: the third semi-axis of the collision spheroid (a, a, b) of
    Eq. (inter_robot_con); None gives the sphere b = a."""
    return O.Problem(dim=spec.dim, n_robots=N or spec.n_robots, T=spec.T, order=spec.order,
                     t_final=spec.t_final, rho=rho, coll_a=spec.coll,
                     coll_b=spec.coll if coll_b is None else coll_b, v_max=spec.v_max, a_max=spec.a_max)


def run_oracle(O, sc: si.Scene, rho: float, K: int, idx=None, hist=False, coll_b=None):
    xb = sc.xi_bar if idx is None else sc.xi_bar[idx]
    x0 = None
    if sc.spec.init == "zero":
        x0 = np.zeros_like(xb)
    return O.run_batch(oracle_problem(O, sc.spec, rho, coll_b=coll_b), sc.start, sc.goal, xb, K=K, xi0=x0,
                       hist=hist)


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(a.shape[0], -1)
    b = np.asarray(b, np.float64).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-30)


def lam_err(lam, ref_lam, ref_xi):
    """Per-sample ||lambda - lambda_ref|| / ||xi_ref|| (see TOL_LAM)."""
    a = np.asarray(lam, np.float64).reshape(np.shape(lam)[0], -1)
    b = np.asarray(ref_lam, np.float64).reshape(a.shape[0], -1)
    x = np.asarray(ref_xi, np.float64).reshape(a.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(x, axis=1), 1e-30)
