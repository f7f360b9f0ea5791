"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants, independent library routines, a hand-worked example, or
brute force. A plausible slip in the oracle (dropped term, wrong sign, wrong
index, transposed operand) fails at least one of them.
"""
import os

import numpy as np
import pytest
from scipy.interpolate import BPoly

import swarm_inputs as si

HERE = os.path.dirname(os.path.abspath(__file__))


def _problem(O, **kw):
    base = dict(dim=3, n_robots=3, T=40, order=10, t_final=5.0, rho=0.3, coll_a=0.5, coll_b=0.5,
                v_max=2.0, a_max=3.0)
    base.update(kw)
    return O.Problem(**base)


# --- Eq. (poly): the basis -------------------------------------------------------

def test_basis_matches_scipy_bernstein(oracle_lib):
    """Bernstein basis and derivatives against scipy's BPoly (independent)."""
    O = oracle_lib
    order, T, tf = 10, 37, 4.0
    P, Pd, Pdd = O.basis(order, T, tf)
    tau = np.arange(T) / (T - 1)
    for k in range(order + 1):
        c = np.zeros((order + 1, 1))
        c[k, 0] = 1.0
        bp = BPoly(c, [0.0, 1.0])
        np.testing.assert_allclose(P[:, k], bp(tau), atol=1e-13)
        np.testing.assert_allclose(Pd[:, k], bp.derivative(1)(tau) / tf, atol=1e-11)
        np.testing.assert_allclose(Pdd[:, k], bp.derivative(2)(tau) / tf ** 2, atol=1e-10)
    # partition of unity and its derivatives
    np.testing.assert_allclose(P.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(Pd.sum(1), 0.0, atol=1e-12)
    np.testing.assert_allclose(Pdd.sum(1), 0.0, atol=1e-11)


# --- Appendix, alpha / beta / d steps ---------------------------------------------

def test_pair_projection_is_euclidean_for_spheres(oracle_lib):
    """For a == b the closed-form steps give the Euclidean projection onto
    {||v|| >= a}: identity outside, a * v / ||v|| inside."""
    O = oracle_lib
    rng = np.random.default_rng(1)
    a = 0.6
    for dim in (2, 3):
        for _ in range(500):
            v = rng.normal(size=dim) * rng.choice([0.1, 0.5, 2.0])
            e = O.pair_project(a, a, v)
            r = np.linalg.norm(v)
            expect = v if r >= a else a * v / r
            np.testing.assert_allclose(e, expect, atol=1e-13)


def test_pair_projection_tie_break_at_zero(oracle_lib):
    """delta = 0 (either zero sign): alpha = beta = 0, d = 1."""
    O = oracle_lib
    a, b = 0.6, 0.4
    for z in (0.0, -0.0):
        np.testing.assert_array_equal(O.pair_project(a, b, np.array([z, z, z])), [0.0, 0.0, b])
        np.testing.assert_array_equal(O.pair_project(a, b, np.array([z, z])), [a, 0.0])
    np.testing.assert_array_equal(O.ball_project(2.0, np.zeros(3)), np.zeros(3))


def test_pair_projection_brute_force_argmin(oracle_lib):
    """The steps minimise ||delta - d (a ca sb, a sa sb, b cb)||^2 over the
    angles and d >= 1; compared with a dense grid search (a == b)."""
    O = oracle_lib
    rng = np.random.default_rng(2)
    a = 0.5
    al = np.linspace(-np.pi, np.pi, 721)
    be = np.linspace(0, np.pi, 361)
    A, B = np.meshgrid(al, be, indexing="ij")
    U = np.stack([np.cos(A) * np.sin(B), np.sin(A) * np.sin(B), np.cos(B)], -1)
    for _ in range(20):
        v = rng.normal(size=3) * 0.3
        # best d for every direction, clipped to [1, inf), then the AL term
        d = np.maximum((U @ v) / a, 1.0)
        val = np.sum((v - a * d[..., None] * U) ** 2, -1)
        e = O.pair_project(a, a, v)
        assert np.sum((v - e) ** 2) <= val.min() + 1e-12
        # and the grid optimum is close to the oracle's point
        i = np.unravel_index(np.argmin(val), val.shape)
        np.testing.assert_allclose(a * d[i] * U[i], e, atol=5e-3)


def test_spheroid_projection_scaled_radial(oracle_lib):
    """a != b: outside the spheroid e = delta; inside, e lies on the surface on
    the ray of delta in scaled coordinates (the scaled-beta reading)."""
    O = oracle_lib
    rng = np.random.default_rng(3)
    a, b = 0.6, 0.3
    M = np.array([a, a, b])
    for _ in range(500):
        v = rng.normal(size=3) * 0.4
        e = O.pair_project(a, b, v)
        s = np.linalg.norm(v / M)
        if s >= 1:
            np.testing.assert_allclose(e, v, atol=1e-13)
        else:
            np.testing.assert_allclose(np.linalg.norm(e / M), 1.0, atol=1e-13)
            np.testing.assert_allclose(e / M, (v / M) / s, atol=1e-13)


def test_ball_projection(oracle_lib):
    """Velocity / acceleration blocks (centre 0, d in [0, 1]) = ball projection."""
    O = oracle_lib
    rng = np.random.default_rng(4)
    for dim in (2, 3):
        for _ in range(300):
            v = rng.normal(size=dim) * 3
            e = O.ball_project(2.0, v)
            r = np.linalg.norm(v)
            np.testing.assert_allclose(e, v if r <= 2.0 else 2.0 * v / r, atol=1e-13)
    c = np.array([1.0, -2.0, 0.5])
    for _ in range(300):
        p = c + rng.normal(size=3) * 3
        e = O.spheroid_in_project(3.0, 1.5, c, p)
        s = np.linalg.norm((p - c) / np.array([3.0, 3.0, 1.5]))
        if s <= 1:
            np.testing.assert_allclose(e, p, atol=1e-13)
        else:
            np.testing.assert_allclose(np.linalg.norm((e - c) / np.array([3.0, 3.0, 1.5])), 1.0,
                                       atol=1e-13)


# --- Appendix, F, A and the KKT of the xi step -------------------------------------

def _kron_F(P, Pd, Pdd, N, dim, v_on=True, a_on=True):
    """F from the Kronecker form printed in the Appendix: F_o = [F_{o,i}] (x) P
    with F_{o,i} = [F_i, -I], F_i the (n-i) x i block with ones in column i;
    velocity and acceleration blocks I (x) Pd, I (x) Pdd; block-diagonal over
    the axes."""
    blocks = []
    for i in range(1, N):
        Fi = np.zeros((N - i, i))
        Fi[:, i - 1] = 1.0
        blocks.append(np.hstack([Fi, -np.eye(N - i)]))
    Fo = np.kron(np.vstack(blocks), P) if N > 1 else np.zeros((0, N * P.shape[1]))
    parts = [Fo]
    if v_on:
        parts.append(np.kron(np.eye(N), Pd))
    if a_on:
        parts.append(np.kron(np.eye(N), Pdd))
    Fax = np.vstack(parts)
    return np.kron(np.eye(dim), Fax)


@pytest.mark.parametrize("N,dim", [(2, 3), (3, 3), (4, 2)])
def test_dense_F_matches_kronecker_form(oracle_lib, N, dim):
    O = oracle_lib
    pb = _problem(O, n_robots=N, dim=dim, T=12)
    rng = np.random.default_rng(5)
    sf = O.OracleSF(pb, rng.normal(size=(N, dim)), rng.normal(size=(N, dim)))
    F = sf.dense_F()
    P, Pd, Pdd = O.basis(pb.order, pb.T, pb.t_final)
    Fk = _kron_F(P, Pd, Pdd, N, dim)
    np.testing.assert_allclose(F, Fk, atol=1e-14)


def test_operators_adjoint_and_laplacian(oracle_lib):
    """<F x, y> = <x, F^T y>; F^T F per axis = (N I - 1 1^T) (x) P^T P +
    I (x) (Pd^T Pd + Pdd^T Pdd) (complete-graph Laplacian identity)."""
    O = oracle_lib
    N, dim = 5, 3
    pb = _problem(O, n_robots=N, dim=dim, T=30)
    rng = np.random.default_rng(6)
    sf = O.OracleSF(pb, rng.normal(size=(N, dim)), rng.normal(size=(N, dim)))
    for _ in range(5):
        x = rng.normal(size=sf.n)
        y = rng.normal(size=sf.m)
        lhs = sf.apply("apply_F", x) @ y
        rhs = x @ sf.apply("apply_Ft", y)
        assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
    K = sf.kkt_matrix()
    P, Pd, Pdd = O.basis(pb.order, pb.T, pb.t_final)
    L = N * np.eye(N) - np.ones((N, N))
    H = np.kron(L, P.T @ P) + np.kron(np.eye(N), Pd.T @ Pd + Pdd.T @ Pdd)
    nc = N * pb.nvar
    np.testing.assert_allclose(K[:nc, :nc], np.eye(nc) + pb.rho * H, atol=1e-9, rtol=1e-12)


def test_boundary_rows_and_xi_step_solve(oracle_lib):
    """A holds (p, pdot, pddot) at t = 0 and t = H; the xi step equals the
    dense KKT solve done by numpy on F and A."""
    O = oracle_lib
    N, dim = 3, 3
    pb = _problem(O, n_robots=N, dim=dim, T=25)
    rng = np.random.default_rng(7)
    st, gl = rng.normal(size=(N, dim)), rng.normal(size=(N, dim))
    sva, gva = rng.normal(size=(N, 2, dim)), rng.normal(size=(N, 2, dim))
    sf = O.OracleSF(pb, st, gl, sva, gva)
    A, b = sf.dense_A()
    P, Pd, Pdd = O.basis(pb.order, pb.T, pb.t_final)
    rows = np.stack([P[0], Pd[0], Pdd[0], P[-1], Pd[-1], Pdd[-1]])
    for ax in range(dim):
        for i in range(N):
            r0 = (ax * N + i) * 6
            c0 = (ax * N + i) * pb.nvar
            np.testing.assert_array_equal(A[r0:r0 + 6, c0:c0 + pb.nvar], rows)
            np.testing.assert_array_equal(b[r0:r0 + 6], [st[i, ax], sva[i, 0, ax], sva[i, 1, ax],
                                                         gl[i, ax], gva[i, 0, ax], gva[i, 1, ax]])
    F = sf.dense_F()
    n = sf.n
    Kd = np.block([[np.eye(n) + pb.rho * F.T @ F, A.T], [A, np.zeros((A.shape[0], A.shape[0]))]])
    rhs = rng.normal(size=n)
    sol = np.linalg.solve(Kd, np.concatenate([rhs, b]))[:n]
    np.testing.assert_allclose(sf.apply("solve_xi", rhs), sol, atol=1e-10)


# --- Eq. (boundary_con): P1 ----------------------------------------------------------

def test_boundary_conditions_hold_after_iterations(oracle_lib):
    O = oracle_lib
    N, dim = 4, 3
    pb = _problem(O, n_robots=N, dim=dim, T=40)
    rng = np.random.default_rng(8)
    st, gl = rng.normal(size=(N, dim)) * 2, rng.normal(size=(N, dim)) * 2
    sva, gva = rng.normal(size=(N, 2, dim)) * 0.3, rng.normal(size=(N, 2, dim)) * 0.3
    sf = O.OracleSF(pb, st, gl, sva, gva)
    A, b = sf.dense_A()
    xb = rng.normal(size=sf.n) * 2
    out = sf.run(xb, 7)
    assert np.abs(A @ out["xi"] - b).max() <= 1e-12 * max(1, np.abs(b).max()) * 10


def test_bernstein_boundary_coefficients(oracle_lib):
    """With zero boundary velocity / acceleration, c0 = c1 = c2 = start and
    c8 = c9 = c10 = goal (Bernstein end-point property, order 10)."""
    O = oracle_lib
    spec = si.config_small_2d(n_samples=3)
    sc = si.scene(spec, 0)
    pb = _problem(O, dim=2, n_robots=4, T=100, coll_a=0.6, coll_b=0.6)
    sf = O.OracleSF(pb, sc.start, sc.goal)
    out = sf.run(sc.xi_bar[0], 5, xi0=np.zeros(sf.n))
    xi = out["xi"].reshape(2, 4, 11)
    for ax in range(2):
        for i in range(4):
            np.testing.assert_allclose(xi[ax, i, :3], sc.start[i, ax], atol=1e-12)
            np.testing.assert_allclose(xi[ax, i, 8:], sc.goal[i, ax], atol=1e-12)


# --- P2: an already-feasible sample comes back unchanged ---------------------------

def _feasible_lanes(N, dim, sep=2.0, length=2.0):
    """Robots on parallel lanes sep apart, moving length along x with zero end
    velocity / acceleration (c0..c2 = start, c8..c10 = goal, ramps between)."""
    w = np.array([0, 0, 0, 0.1, 0.3, 0.5, 0.7, 0.9, 1, 1, 1.0])
    st = np.zeros((N, dim))
    st[:, 1] = sep * np.arange(N)
    gl = st.copy()
    gl[:, 0] += length
    xi = np.zeros((dim, N, 11))
    for ax in range(dim):
        for i in range(N):
            xi[ax, i] = st[i, ax] + w * (gl[i, ax] - st[i, ax])
    return st, gl, xi


def test_feasible_sample_returned_unchanged(oracle_lib):
    O = oracle_lib
    N, dim = 4, 3
    pb = _problem(O, n_robots=N, dim=dim, T=50)
    st, gl, xb = _feasible_lanes(N, dim)
    sf = O.OracleSF(pb, st, gl)
    out = sf.run(xb.reshape(-1), 5)
    assert out["viol"] <= 0.0
    np.testing.assert_allclose(out["xi"], xb.reshape(-1), atol=1e-12)
    np.testing.assert_allclose(out["lam"], 0.0, atol=1e-12)
    assert out["rp_hist"].max() <= 1e-12


# --- P3: no active inequality -> affine iteration towards the equality-QP projection

def test_affine_iteration_to_equality_projection(oracle_lib):
    """Two robots far apart, loose bounds, sample init: e = F xi every step, so
    xi^{k+1} = T xi^k + c with T = S rho F^T F (S the xi-block of the KKT
    inverse) and the fixed point is the closed-form equality-QP projection
    xi_QP = xi_bar - A^T (A A^T)^{-1} (A xi_bar - b). Then
    xi^k - xi_QP = T^k (xi^0 - xi_QP) for every k."""
    O = oracle_lib
    N, dim = 2, 3
    pb = _problem(O, n_robots=N, dim=dim, T=30, v_max=50.0, a_max=50.0, rho=0.7)
    st = np.array([[0.0, 0, 0], [0, 20.0, 0]])
    gl = st + np.array([1.0, 0.5, -0.3])
    sf = O.OracleSF(pb, st, gl)
    rng = np.random.default_rng(9)
    xb = np.zeros((dim, N, 11))
    for i in range(N):
        for ax in range(dim):
            xb[ax, i] = st[i, ax] + np.linspace(0, 1, 11) * (gl[i, ax] - st[i, ax])
    xb = xb.reshape(-1) + rng.normal(size=sf.n) * 0.05
    A, b = sf.dense_A()
    xqp = xb - A.T @ np.linalg.solve(A @ A.T, A @ xb - b)
    F = sf.dense_F()
    n = sf.n
    Kd = np.block([[np.eye(n) + pb.rho * F.T @ F, A.T], [A, np.zeros((A.shape[0], A.shape[0]))]])
    Kinv = np.linalg.inv(Kd)
    Tm = Kinv[:n, :n] @ (pb.rho * F.T @ F)
    for k in (1, 2, 5, 20):
        out = sf.run(xb, k)
        assert out["viol"] <= 0
        pred = np.linalg.matrix_power(Tm, k) @ (xb - xqp)
        np.testing.assert_allclose(out["xi"] - xqp, pred, atol=1e-10)


# --- P4: symmetries ---------------------------------------------------------------------

def _swap_instance(offset=0.05):
    """Two robots swapping places head-on along x, slightly offset in y/z."""
    st = np.array([[-2.0, offset, 0.02], [2.0, -offset, -0.02]])
    gl = np.array([[2.0, offset, 0.02], [-2.0, -offset, -0.02]])
    k = np.linspace(0, 1, 11)
    xb = np.zeros((3, 2, 11))
    for ax in range(3):
        for i in range(2):
            xb[ax, i] = st[i, ax] + k * (gl[i, ax] - st[i, ax])
    return st, gl, xb


def test_mirror_symmetry_head_on_swap(oracle_lib):
    """Mirroring y -> -y (and z -> -z) of inputs mirrors the outputs."""
    O = oracle_lib
    pb = _problem(O, n_robots=2, dim=3, T=60)
    st, gl, xb = _swap_instance()
    base = O.OracleSF(pb, st, gl).run(xb.reshape(-1), 60)["xi"].reshape(3, 2, 11)
    for axes in ([1], [2], [1, 2]):
        m = np.ones(3)
        m[axes] = -1
        st2, gl2 = st * m, gl * m
        xb2 = xb * m[:, None, None]
        out = O.OracleSF(pb, st2, gl2).run(xb2.reshape(-1), 60)["xi"].reshape(3, 2, 11)
        np.testing.assert_allclose(out, base * m[:, None, None], atol=1e-12)


def test_permutation_equivariance(oracle_lib):
    """Relabelling robots permutes the outputs (pair orientation flips and
    proj(-delta) = -proj(delta))."""
    O = oracle_lib
    N = 4
    pb = _problem(O, n_robots=N, dim=3, T=40)
    spec = si.config_n16_3d(n_robots=N, n_samples=1, box=(3.0, 3.0, 1.5), min_sep=0.8)
    sc = si.scene(spec, 11)
    perm = np.array([2, 0, 3, 1])
    a = O.OracleSF(pb, sc.start, sc.goal).run(sc.xi_bar[0].reshape(-1), 40)["xi"].reshape(3, N, 11)
    b = O.OracleSF(pb, sc.start[perm], sc.goal[perm]).run(
        sc.xi_bar[0][:, perm].reshape(-1), 40)["xi"].reshape(3, N, 11)
    np.testing.assert_allclose(b, a[:, perm], atol=1e-11)


def test_time_reversal(oracle_lib):
    """Swapping start and goal and reversing c_k -> c_{10-k} reverses the
    solution (Bernstein symmetry on the symmetric grid; the velocity rows flip
    sign, the ball projections are odd)."""
    O = oracle_lib
    N = 3
    pb = _problem(O, n_robots=N, dim=3, T=41)
    spec = si.config_n16_3d(n_robots=N, n_samples=1, box=(3.0, 3.0, 1.5), min_sep=0.8)
    sc = si.scene(spec, 12)
    a = O.OracleSF(pb, sc.start, sc.goal).run(sc.xi_bar[0].reshape(-1), 30)["xi"].reshape(3, N, 11)
    b = O.OracleSF(pb, sc.goal, sc.start).run(sc.xi_bar[0][..., ::-1].reshape(-1), 30)["xi"]
    np.testing.assert_allclose(b.reshape(3, N, 11)[..., ::-1], a, atol=1e-10)


# --- P7: the scalar worked example, through the oracle's generic AM core ------------

def test_scalar_worked_example(oracle_lib):
    O = oracle_lib
    rows = []
    with open(os.path.join(HERE, "golden", "scalar_am_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    rho = 1.0
    inst = O.ScalarInstance(
        n=1, m=1, F=lambda x: x, Ft=lambda y: y, project=lambda v: np.maximum(1.0, v),
        solve=lambda rhs: rhs / (1.0 + rho))
    for x0 in (-3.0, 0.0):
        x, lam = np.array([x0]), np.array([0.0])
        seq = {}
        for k in range(1, 11):
            x, lam, _ = inst.step(rho, np.array([0.0]), x, lam)
            seq[k] = (x[0], lam[0])
        for r in rows:
            if r[0] == x0:
                assert seq[int(r[1])] == (r[2], r[3])


def test_printed_plus_sign_would_diverge(oracle_lib):
    """Documents the lambda-step sign reading: the printed '+' applied to the
    same scalar example runs away instead of converging."""
    x, lam = -3.0, 0.0
    for _ in range(30):
        e = max(1.0, x)
        lam = lam + (x - e)
        x = (e + lam) / 2.0
    assert abs(x) > 1e4


# --- the problem reaches feasibility on the workloads ---------------------------------

def test_residual_decreases_on_small_2d(oracle_lib):
    O = oracle_lib
    spec = si.config_small_2d(n_samples=4)
    sc = si.scene(spec, 0)
    pb = _problem(O, dim=2, n_robots=4, T=100, coll_a=spec.coll, coll_b=spec.coll)
    out = O.run_batch(pb, sc.start, sc.goal, sc.xi_bar, K=100, xi0=np.zeros_like(sc.xi_bar), hist=True)
    h = out["rp_hist"]
    assert np.all(h[:, -1] < 0.01 * h[:, 0])
    assert np.median(out["rp_final"]) < 2e-3


# --- Eq. (primal_residual): the residual outputs ----------------------------------------

def _dense_e(Fx, N, T, dim, a, v_max, a_max):
    """e(F xi) row by row from the dense F's row order (per axis: pair rows
    (i < j) x T, velocity rows N x T, acceleration rows N x T), with the
    Euclidean projections the closed forms reduce to for a == b."""
    npair = N * (N - 1) // 2
    R = (npair + 2 * N) * T
    X = Fx.reshape(dim, R)
    E = X.copy()
    viol = -np.inf
    for blk, (count, kind) in enumerate(((npair, "pair"), (N, "v"), (N, "a"))):
        off = (0, npair * T, (npair + N) * T)[blk]
        for r in range(count):
            for t in range(T):
                col = off + r * T + t
                d = X[:, col]
                nrm = np.linalg.norm(d)
                if kind == "pair":
                    E[:, col] = d * max(1.0, a / nrm)
                    viol = max(viol, a - nrm)
                else:
                    bound = v_max if kind == "v" else a_max
                    E[:, col] = d * min(1.0, bound / nrm)
                    viol = max(viol, nrm - bound)
    return E.reshape(-1), viol


def test_residual_outputs_match_their_definition(oracle_lib):
    """rp_hist[k] = ||F xi^{k+1} - e(F xi^k)||, proj_hist[k] = ||F xi^k -
    e(F xi^k)|| and viol = the largest violation of xi^K, evaluated here with
    the dense F (pinned against the Kronecker form of the Appendix) and the
    Euclidean projections, on an instance with active pair, velocity and
    acceleration rows. Catches a residual paired with the wrong iterate, a
    dropped block or a wrong norm."""
    O = oracle_lib
    N, dim, T, K = 3, 3, 24, 6
    pb = _problem(O, n_robots=N, dim=dim, T=T, v_max=1.2, a_max=1.5, coll_a=0.8, coll_b=0.8, rho=0.3)
    st = np.array([[-1.5, 0.1, 0.05], [1.5, -0.1, -0.05], [0.05, -1.6, 0.1]])
    gl = np.array([[1.5, 0.1, 0.05], [-1.5, -0.1, -0.05], [0.05, 1.6, 0.1]])
    rng = np.random.default_rng(31)
    xb = np.zeros((dim, N, 11))
    for i in range(N):
        for ax in range(dim):
            xb[ax, i] = np.linspace(st[i, ax], gl[i, ax], 11)
    xb = xb.reshape(-1) + rng.normal(size=dim * N * 11) * 0.3
    sf = O.OracleSF(pb, st, gl)
    F = sf.dense_F()
    out = sf.run(xb, K)
    # the iterates one step at a time (the run is deterministic)
    xs, lam = [xb.copy()], np.zeros_like(xb)
    for k in range(K):
        o = sf.run(xb, 1, xi0=xs[-1], lam0=lam)
        xs.append(o["xi"])
        lam = o["lam"]
    np.testing.assert_allclose(xs[-1], out["xi"], atol=1e-12)
    n_active = 0
    for k in range(K):
        e, _ = _dense_e(F @ xs[k], N, T, dim, 0.8, 1.2, 1.5)
        n_active += int(np.sum(np.abs(e - F @ xs[k]) > 1e-12))
        np.testing.assert_allclose(out["proj_hist"][k], np.linalg.norm(F @ xs[k] - e), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(out["rp_hist"][k], np.linalg.norm(F @ xs[k + 1] - e), rtol=1e-10, atol=1e-12)
    assert n_active > 0
    _, viol = _dense_e(F @ xs[K], N, T, dim, 0.8, 1.2, 1.5)
    np.testing.assert_allclose(out["viol"], viol, rtol=1e-10, atol=1e-12)


def test_batch_run_equals_single_sample_runs(oracle_lib):
    """The threaded batch entry point (the reference of every GPU parity test)
    returns, sample by sample and bit for bit, what single-sample runs
    return: per-sample offsets, initial iterates and history rows are
    wired correctly, and threads do not share state."""
    O = oracle_lib
    spec = si.config_n16_3d(n_robots=5, n_samples=7, T=30, box=(3.0, 3.0, 1.5), min_sep=0.8)
    sc = si.scene(spec, 17)
    pb = _problem(O, n_robots=5, T=30, coll_a=spec.coll, coll_b=spec.coll, rho=0.1)
    K = 12
    rng = np.random.default_rng(5)
    x0 = sc.xi_bar + rng.normal(size=sc.xi_bar.shape) * 0.1
    l0 = rng.normal(size=sc.xi_bar.shape) * 0.05
    out = O.run_batch(pb, sc.start, sc.goal, sc.xi_bar, K=K, xi0=x0, lam0=l0, hist=True, n_threads=3)
    sf = O.OracleSF(pb, sc.start, sc.goal)
    for s in range(sc.xi_bar.shape[0]):
        one = sf.run(sc.xi_bar[s].reshape(-1), K, xi0=x0[s].reshape(-1), lam0=l0[s].reshape(-1))
        np.testing.assert_array_equal(out["xi"][s].reshape(-1), one["xi"])
        np.testing.assert_array_equal(out["lam"][s].reshape(-1), one["lam"])
        np.testing.assert_array_equal(out["rp_hist"][s], one["rp_hist"])
        np.testing.assert_array_equal(out["proj_hist"][s], one["proj_hist"])
        assert out["rp_final"][s] == one["rp_hist"][-1]
