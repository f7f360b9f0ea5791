"""The decoders' QP layer on the GPU (sf_eq_project / _backward through the
C ABI) against the FP64 oracle's KKT solve and its adjoint, on single scenes
with and without boundary velocity / acceleration, 2D and 3D, a ragged
multi-scene batch, and through the autograd Function."""
import numpy as np
import pytest
import torch

import swarm_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    P.build()
    return P


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _oracle_sf(O, sc, sva=None, gva=None):
    spec = sc.spec
    pb = O.Problem(dim=spec.dim, n_robots=spec.n_robots, T=spec.T, order=spec.order, t_final=spec.t_final,
                   rho=0.1, coll_a=spec.coll, coll_b=spec.coll)
    return O.OracleSF(pb, sc.start, sc.goal, sva, gva)


@pytest.mark.parametrize("dim,va", [(3, False), (3, True), (2, False)])
def test_eq_project_matches_oracle(sfmod, oracle_lib, dim, va):
    spec = si.config_n16_3d(n_robots=7, n_samples=37, T=80) if dim == 3 else si.config_small_2d(n_samples=23)
    sc = si.scene(spec, 9)
    rng = np.random.default_rng(4)
    N = spec.n_robots
    sva = rng.normal(size=(N, 2, dim)) if va else None
    gva = rng.normal(size=(N, 2, dim)) if va else None
    f = sfmod.SafetyFilter(dim=dim, T=spec.T, rho=0.1, coll_a=spec.coll, max_robots=N, t_final=spec.t_final)
    xp = sc.xi_bar + rng.normal(size=sc.xi_bar.shape)          # decoder outputs off the constraints
    kw = dict(start_va=_dev(sva) if va else None, goal_va=_dev(gva) if va else None)
    out = f.eq_project(_dev(xp), _dev(sc.start), _dev(sc.goal), **kw).double().cpu().numpy()
    g = rng.normal(size=xp.shape)
    gin, gb = f.eq_project_backward(_dev(g), _dev(sc.start), _dev(sc.goal), want_grad_b=True, **kw)
    osf = _oracle_sf(oracle_lib, sc, sva, gva)
    scale = np.abs(xp).max()
    for s in range(spec.n_samples):
        ref = osf.eq_project(xp[s])
        np.testing.assert_allclose(out[s].reshape(-1), ref, atol=2e-6 * scale, rtol=0)
        rgi, rgb = osf.eq_project_adjoint(g[s])
        np.testing.assert_allclose(gin[s].double().cpu().numpy().reshape(-1), rgi, atol=2e-5, rtol=0)
        # grad_b rows of sample s: (axis, robot) order, 6 values each
        np.testing.assert_allclose(gb[s * dim * N:(s + 1) * dim * N].double().cpu().numpy().reshape(-1), rgb,
                                   atol=2e-4 * np.abs(rgb).max(), rtol=0)
    # A xi = b holds on the output (boundary rows of the basis)
    Pm, Pd, Pdd = oracle_lib.basis(10, spec.T, spec.t_final)
    pos0 = np.einsum("k,sdnk->snd", Pm[0], out)
    np.testing.assert_allclose(pos0, np.broadcast_to(sc.start, pos0.shape), atol=2e-5 * scale)


def test_eq_project_ragged_batch(sfmod, oracle_lib):
    """Several scenes of different N and S (one empty) in one call."""
    specs = [si.config_n16_3d(n_robots=n, n_samples=s, T=60) for n, s in [(3, 5), (11, 2), (5, 0), (30, 3)]]
    st = si.Stream(12)
    scenes = [si.make_scene(sp, st) for sp in specs]
    f = sfmod.SafetyFilter(dim=3, T=60, rho=0.1, coll_a=0.5, max_robots=32)
    rng = np.random.default_rng(5)
    xp = [s.xi_bar + rng.normal(size=s.xi_bar.shape) for s in scenes]
    flat = np.concatenate([x.reshape(-1) for x in xp])
    out = f.eq_project(_dev(flat), _dev(np.concatenate([s.start for s in scenes])),
                       _dev(np.concatenate([s.goal for s in scenes])),
                       n_robots=[s.spec.n_robots for s in scenes],
                       n_samples=[s.spec.n_samples for s in scenes]).double().cpu().numpy()
    c = 0
    for s, x in zip(scenes, xp):
        osf = _oracle_sf(oracle_lib, s)
        for k in range(s.spec.n_samples):
            n = x[k].size
            np.testing.assert_allclose(out[c:c + n], osf.eq_project(x[k]), atol=2e-6 * np.abs(x).max(), rtol=0)
            c += n
    assert c == out.size


def test_eq_project_autograd(sfmod):
    from paper_2501_19042_gb300.autograd import eq_project
    sc = si.scene(si.config_n16_3d(n_robots=4, n_samples=8, T=50), 3)
    f = sfmod.SafetyFilter(dim=3, T=50, rho=0.1, coll_a=0.5, max_robots=4)
    xp = _dev(sc.xi_bar + 0.3).requires_grad_(True)
    w = torch.randn(xp.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    y = eq_project(f, xp, _dev(sc.start), _dev(sc.goal))
    (w * y).sum().backward()
    gin, _ = f.eq_project_backward(w.contiguous(), _dev(sc.start), _dev(sc.goal))
    assert torch.equal(xp.grad, gin)
    # the projection is idempotent and its gradient annihilates the constraint normals
    y2 = f.eq_project(y.detach().contiguous(), _dev(sc.start), _dev(sc.goal))
    assert (y2 - y).abs().max().item() <= 1e-4
