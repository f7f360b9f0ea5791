"""P8: the oracle against an independent brute-force penalty solver on 2-3
robot instances with one brief overlap.

The penalty solver shares nothing with the oracle: its own basis (scipy
BPoly), its own constraint functions, the boundary conditions eliminated by
fixing c0..c2 and c8..c10 (zero end velocity / acceleration), and L-BFGS on
1/2 ||xi - xi_bar||^2 + mu * sum of squared violations with mu -> 1e8.

What is pinned: the oracle's converged output is feasible, it is never closer
to xi_bar than the true projection (which the penalty solver finds), and the
gap between the two is bounded. The SF's fixed point is NOT the exact
projection: its multiplier accumulates rho F^T (e - F xi) over the history,
so rows that were active early bias the final point (a property of the
iteration as printed). The measured gaps are stated in the asserts.
"""
import numpy as np
import pytest
from scipy.interpolate import BPoly
from scipy.optimize import minimize


def _basis(order, T, tf):
    tau = np.arange(T) / (T - 1)
    P, Pd, Pdd = (np.zeros((T, order + 1)) for _ in range(3))
    for k in range(order + 1):
        c = np.zeros((order + 1, 1))
        c[k, 0] = 1
        bp = BPoly(c, [0, 1])
        P[:, k] = bp(tau)
        Pd[:, k] = bp.derivative(1)(tau) / tf
        Pdd[:, k] = bp.derivative(2)(tau) / tf ** 2
    return P, Pd, Pdd


def penalty_projection(st, gl, xb, a, vmax, amax, T, tf=5.0):
    N, dim = st.shape
    P, Pd, Pdd = _basis(10, T, tf)

    def unpack(z):
        xi = np.zeros((dim, N, 11))
        xi[:, :, :3] = st.T[:, :, None]
        xi[:, :, 8:] = gl.T[:, :, None]
        xi[:, :, 3:8] = z.reshape(dim, N, 5)
        return xi

    def f(z, mu):
        xi = unpack(z)
        p = np.einsum("tk,dik->dit", P, xi)
        v = np.einsum("tk,dik->dit", Pd, xi)
        ac = np.einsum("tk,dik->dit", Pdd, xi)
        val = 0.5 * np.sum((xi - xb) ** 2)
        gp, gv, ga = np.zeros_like(p), np.zeros_like(v), np.zeros_like(ac)
        for i in range(N):
            for j in range(i + 1, N):
                D = p[:, i] - p[:, j]
                h = np.maximum(a * a - np.sum(D ** 2, 0), 0)
                val += mu * np.sum(h ** 2)
                gD = -4 * mu * h * D
                gp[:, i] += gD
                gp[:, j] -= gD
        for arr, bnd, garr in ((v, vmax, gv), (ac, amax, ga)):
            h = np.maximum(np.sum(arr ** 2, 0) - bnd * bnd, 0)
            val += mu * np.sum(h ** 2)
            garr += 4 * mu * h * arr
        g = (xi - xb) + np.einsum("tk,dit->dik", P, gp) + np.einsum("tk,dit->dik", Pd, gv) + \
            np.einsum("tk,dit->dik", Pdd, ga)
        return val, g[:, :, 3:8].reshape(-1)

    z = xb[:, :, 3:8].reshape(-1).copy()
    for mu in [1e2, 1e3, 1e4, 1e5, 1e6, 1e7, 1e8]:
        z = minimize(f, z, args=(mu,), jac=True, method="L-BFGS-B",
                     options=dict(maxiter=20000, gtol=1e-12, ftol=1e-15)).x
    return unpack(z)


def _crossing(n_rob, seed):
    """Robots crossing near the origin at mid-horizon: a brief overlap."""
    w = np.array([0, 0, 0, 0.1, 0.3, 0.5, 0.7, 0.9, 1, 1, 1.0])
    ang = np.pi * np.arange(n_rob) / n_rob
    st = np.stack([-2 * np.cos(ang), -2 * np.sin(ang), 0.1 * np.arange(n_rob)], 1)
    gl = st * np.array([-1, -1, 1.0])
    xb = np.zeros((3, n_rob, 11))
    for ax in range(3):
        for i in range(n_rob):
            xb[ax, i] = st[i, ax] + w * (gl[i, ax] - st[i, ax])
    rng = np.random.default_rng(seed)
    xb[:, :, 3:8] += rng.normal(size=(3, n_rob, 5)) * 0.05
    return st, gl, xb


@pytest.mark.parametrize("n_rob,rho,gap", [(2, 0.1, 0.01), (3, 0.1, 0.08), (2, 0.3, 0.04)])
def test_oracle_vs_penalty_solver(oracle_lib, n_rob, rho, gap):
    O = oracle_lib
    T = 60
    st, gl, xb = _crossing(n_rob, 0)
    pb = O.Problem(dim=3, n_robots=n_rob, T=T, rho=rho, coll_a=0.5, coll_b=0.5, v_max=2.0, a_max=3.0)
    out = O.OracleSF(pb, st, gl).run(xb.reshape(-1), 5000)
    xo = out["xi"].reshape(3, n_rob, 11)
    xp = penalty_projection(st, gl, xb, 0.5, 2.0, 3.0, T)
    # the instance really has an overlap to resolve
    assert np.linalg.norm(xp - xb) > 0.1
    # converged and feasible (Eq. primal_residual -> 0)
    assert out["rp_hist"][-1] < 1e-9 and out["viol"] < 1e-9
    # never closer to xi_bar than the projection
    assert np.linalg.norm(xo - xb) >= np.linalg.norm(xp - xb) - 1e-6
    # bounded gap to the true projection (measured 0.5% / 6.6% / 2.0%)
    rel = np.linalg.norm(xo - xp) / np.linalg.norm(xp)
    assert rel < gap, rel
