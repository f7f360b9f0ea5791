"""Pins of the oracle's QP layer (the decoders' differentiable QP: Eq.
(sf_form) with the equality constraints only, Sec. III-A / B) against the
optimality conditions, an independent null-space basis, the closed form,
and finite differences."""
import numpy as np
import pytest
from scipy.linalg import null_space


def _sf(O, N=4, dim=3, T=30, seed=0, va=False):
    rng = np.random.default_rng(seed)
    pb = O.Problem(dim=dim, n_robots=N, T=T, rho=0.3)
    st, gl = rng.normal(size=(N, dim)) * 2, rng.normal(size=(N, dim)) * 2
    sva = rng.normal(size=(N, 2, dim)) if va else None
    gva = rng.normal(size=(N, 2, dim)) if va else None
    return O.OracleSF(pb, st, gl, sva, gva), rng


@pytest.mark.parametrize("dim,va", [(3, False), (3, True), (2, True)])
def test_eq_projection_optimality(oracle_lib, dim, va):
    """A xi = b; xi_in - xi is orthogonal to the null space of A (scipy basis);
    a second projection changes nothing; a feasible input is returned."""
    sf, rng = _sf(oracle_lib, dim=dim, va=va)
    A, b = sf.dense_A()
    Z = null_space(A)
    for _ in range(5):
        x = rng.normal(size=sf.n) * 3
        p = sf.eq_project(x)
        np.testing.assert_allclose(A @ p, b, atol=1e-11)
        np.testing.assert_allclose(Z.T @ (x - p), 0.0, atol=1e-10)
        np.testing.assert_allclose(sf.eq_project(p), p, atol=1e-11)


def test_eq_projection_closed_form(oracle_lib):
    """Equals xi_in - A^T (A A^T)^-1 (A xi_in - b) (numpy, dense)."""
    sf, rng = _sf(oracle_lib, va=True, seed=1)
    A, b = sf.dense_A()
    for _ in range(5):
        x = rng.normal(size=sf.n)
        cf = x - A.T @ np.linalg.solve(A @ A.T, A @ x - b)
        np.testing.assert_allclose(sf.eq_project(x), cf, atol=1e-10)


def test_eq_projection_adjoint_finite_differences(oracle_lib):
    """dL/dxi_in and dL/db of L = <w, xi_out> against central differences of
    the oracle's forward (b enters through the boundary rows of the start /
    goal positions)."""
    O = oracle_lib
    N, dim = 3, 3
    rng = np.random.default_rng(2)
    st, gl = rng.normal(size=(N, dim)), rng.normal(size=(N, dim))
    pb = O.Problem(dim=dim, n_robots=N, T=25, rho=0.3)
    sf = O.OracleSF(pb, st, gl)
    x = rng.normal(size=sf.n)
    w = rng.normal(size=sf.n)
    gi, gb = sf.eq_project_adjoint(w)
    h = 1e-6
    for idx in rng.choice(sf.n, 6, replace=False):
        e = np.zeros(sf.n)
        e[idx] = h
        fd = (w @ sf.eq_project(x + e) - w @ sf.eq_project(x - e)) / (2 * h)
        assert abs(fd - gi[idx]) <= 1e-7 * max(1.0, abs(fd))
    # start position of robot i, axis ax is b[(ax * N + i) * 6 + 0]
    for i, ax in ((0, 0), (2, 1), (1, 2)):
        sp, sm = st.copy(), st.copy()
        sp[i, ax] += h
        sm[i, ax] -= h
        fd = (w @ O.OracleSF(pb, sp, gl).eq_project(x) - w @ O.OracleSF(pb, sm, gl).eq_project(x)) / (2 * h)
        assert abs(fd - gb[(ax * N + i) * 6]) <= 1e-7 * max(1.0, abs(fd))
