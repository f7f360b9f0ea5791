"""Pins of the oracle's workspace block (Eqs. workspace_con, workspace_polar;
F_w = I (x) P in the Appendix) against closed forms, brute force and
invariants other than the oracle itself."""
import numpy as np
import pytest

import swarm_inputs as si


def _problem(O, **kw):
    base = dict(dim=3, n_robots=3, T=40, order=10, t_final=5.0, rho=0.3, coll_a=0.5, coll_b=0.5,
                v_max=2.0, a_max=3.0, use_workspace=True, ws_center=(0.5, -0.25, 0.3), ws_a=4.0, ws_b=2.0)
    base.update(kw)
    return O.Problem(**base)


def test_workspace_projection_scaled_radial(oracle_lib):
    """d in [0, 1]: inside the spheroid (and at its centre) the point is kept;
    outside, it moves to the surface along the ray from the centre in scaled
    coordinates; for a_w = b_w that is the Euclidean projection onto the ball."""
    O = oracle_lib
    rng = np.random.default_rng(21)
    c = np.array([0.5, -0.25, 0.3])
    for a, b in ((3.0, 1.5), (2.0, 2.0)):
        M = np.array([a, a, b])
        for _ in range(400):
            p = c + rng.normal(size=3) * 3
            e = O.spheroid_in_project(a, b, c, p)
            s = np.linalg.norm((p - c) / M)
            if s <= 1:
                np.testing.assert_allclose(e, p, atol=1e-13)
            else:
                np.testing.assert_allclose((e - c) / M, ((p - c) / M) / s, atol=1e-12)
            if a == b:
                r = np.linalg.norm(p - c)
                np.testing.assert_allclose(e, c + (p - c) * min(1.0, a / r), atol=1e-12)
        np.testing.assert_allclose(O.spheroid_in_project(a, b, c, c), c, atol=0)
    # 2D: circle of radius a
    c2 = np.array([1.0, 2.0])
    for _ in range(200):
        p = c2 + rng.normal(size=2) * 4
        e = O.spheroid_in_project(2.5, 2.5, c2, p)
        r = np.linalg.norm(p - c2)
        np.testing.assert_allclose(e, c2 + (p - c2) * min(1.0, 2.5 / r), atol=1e-12)


def test_workspace_projection_brute_force(oracle_lib):
    """a_w != b_w: the oracle's point is feasible, and along its ray from the
    centre its d is the distance-minimising d in [0, 1] found by a grid search
    (the d step: least squares in d given the angles, clipped to [0, 1])."""
    O = oracle_lib
    a, b = 2.0, 1.0
    c = np.zeros(3)
    rng = np.random.default_rng(22)
    for _ in range(20):
        p = rng.normal(size=3) * 3
        e = O.spheroid_in_project(a, b, c, p)
        assert np.linalg.norm(e / np.array([a, a, b])) <= 1 + 1e-12
        # along the oracle's direction, d is the least-squares d clipped to [0, 1]
        u = e / max(np.linalg.norm(e / np.array([a, a, b])), 1e-300)
        ds = np.linspace(0, 1, 20001)
        best = ds[np.argmin(np.linalg.norm(ds[:, None] * u[None, :] - p[None, :], axis=1))]
        np.testing.assert_allclose(np.linalg.norm(e / np.array([a, a, b])), best, atol=1e-4)


def _kron_F_ws(P, Pd, Pdd, N, dim):
    blocks = []
    for i in range(1, N):
        Fi = np.zeros((N - i, i))
        Fi[:, i - 1] = 1.0
        blocks.append(np.hstack([Fi, -np.eye(N - i)]))
    Fo = np.kron(np.vstack(blocks), P)
    Fax = np.vstack([Fo, np.kron(np.eye(N), Pd), np.kron(np.eye(N), Pdd), np.kron(np.eye(N), P)])
    return np.kron(np.eye(dim), Fax)


@pytest.mark.parametrize("N,dim", [(3, 3), (4, 2)])
def test_dense_F_with_workspace_rows(oracle_lib, N, dim):
    """F with the workspace block F_w = I (x) P after the pair, velocity and
    acceleration blocks; F^T F per axis = (N I - 1 1^T) (x) P^T P +
    I (x) (Pd^T Pd + Pdd^T Pdd + P^T P)."""
    O = oracle_lib
    pb = _problem(O, n_robots=N, dim=dim, T=15)
    rng = np.random.default_rng(23)
    sf = O.OracleSF(pb, rng.normal(size=(N, dim)), rng.normal(size=(N, dim)))
    P, Pd, Pdd = O.basis(pb.order, pb.T, pb.t_final)
    np.testing.assert_allclose(sf.dense_F(), _kron_F_ws(P, Pd, Pdd, N, dim), atol=1e-14)
    K = sf.kkt_matrix()
    L = N * np.eye(N) - np.ones((N, N))
    H = np.kron(L, P.T @ P) + np.kron(np.eye(N), Pd.T @ Pd + Pdd.T @ Pdd + P.T @ P)
    nc = N * pb.nvar
    np.testing.assert_allclose(K[:nc, :nc], np.eye(nc) + pb.rho * H, atol=1e-9, rtol=1e-12)


def test_sample_inside_workspace_unchanged(oracle_lib):
    """A feasible, boundary-consistent sample well inside the workspace comes
    back unchanged with lambda = 0 (every workspace row has e = F xi)."""
    O = oracle_lib
    N, dim = 3, 3
    pb = _problem(O, n_robots=N, dim=dim, T=50, ws_center=(1.0, 2.0, 0.0), ws_a=20.0, ws_b=10.0)
    st = np.array([[0.0, 0.0, 0.0], [0.0, 3.0, 0.0], [0.0, 6.0, 0.0]])
    gl = st + np.array([2.0, 0.0, 0.0])
    w = np.array([0, 0, 0, 0.1, 0.3, 0.5, 0.7, 0.9, 1, 1, 1.0])
    xb = np.zeros((dim, N, 11))
    for ax in range(dim):
        for i in range(N):
            xb[ax, i] = st[i, ax] + w * (gl[i, ax] - st[i, ax])
    out = O.OracleSF(pb, st, gl).run(xb.reshape(-1), 5)
    np.testing.assert_allclose(out["xi"], xb.reshape(-1), atol=1e-12)
    np.testing.assert_allclose(out["lam"], 0.0, atol=1e-12)


def test_workspace_pulls_trajectory_inside(oracle_lib):
    """A sample whose straight path leaves a spherical workspace between
    boundary points inside it: after the iterations every position at every
    time step is inside the workspace up to a small violation, far less than
    the sample's, and the boundary conditions still hold."""
    O = oracle_lib
    N, dim = 2, 3
    pb = _problem(O, n_robots=N, dim=dim, T=60, rho=0.3, ws_center=(0.0, 0.0, 0.0), ws_a=3.0, ws_b=3.0,
                  v_max=20.0, a_max=50.0)
    st = np.array([[-2.5, 0.0, 0.0], [2.5, 1.5, 0.0]])
    gl = np.array([[-2.5, 1.5, 0.0], [2.5, 0.0, 0.0]])
    xb = np.zeros((dim, N, 11))
    for i in range(N):
        for ax in range(dim):
            xb[ax, i] = np.linspace(st[i, ax], gl[i, ax], 11)
        xb[0, i, 3:8] *= 2.0          # bulge outwards, beyond radius 3
    sf = O.OracleSF(pb, st, gl)
    P, _, _ = O.basis(pb.order, pb.T, pb.t_final)

    def worst(xi):
        x = xi.reshape(dim, N, 11)
        pos = np.einsum("tk,dnk->ntd", P, x)
        return np.max(np.linalg.norm(pos, axis=2)) - 3.0

    assert worst(xb) > 1.0
    out = sf.run(xb.reshape(-1), 400)
    assert worst(out["xi"]) < 0.02
    A, bvec = sf.dense_A()
    np.testing.assert_allclose(A @ out["xi"], bvec, atol=1e-10)


def test_scene_spec_workspace_case():
    """The seeded workload used for workspace parity keeps every start and goal
    inside the workspace sphere (so the boundary conditions are feasible)."""
    spec = si.config_n16_3d(n_samples=4, box=(6.0, 6.0, 3.0), min_sep=1.0)
    sc = si.scene(spec, 61)
    r = np.linalg.norm(np.concatenate([sc.start, sc.goal]), axis=1)
    assert r.max() < 4.8
