"""Learned initialisation (3-layer MLP trained through the differentiable SF)."""
import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_3D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    from paper_2501_19042_gb300 import init_mlp as M
    P.build()
    spec = si.config_diff(n_samples=8)
    sf = P.SafetyFilter(dim=3, T=spec.T, rho=RHO_3D, coll_a=spec.coll, max_robots=16, checkpoint_every=10)
    return P, M, spec, sf


def test_untrained_network_is_the_sample_init(setup):
    P, M, spec, sf = setup
    torch.manual_seed(0)
    mlp = M.InitMLP(16).cuda()
    b = M.make_batch(spec, 123, 4, sf.device)
    xi0, lam0 = mlp(b.start_s, b.goal_s, b.xi_bar)
    assert torch.equal(xi0, b.xi_bar) and torch.count_nonzero(lam0) == 0
    kw = dict(n_robots=b.n_robots, n_samples=b.n_samples)
    a = sf.project(b.xi_bar, b.start, b.goal, 20, **kw)
    c = sf.project(b.xi_bar, b.start, b.goal, 20, xi0=xi0, lam0=lam0, **kw)
    assert torch.equal(a.xi, c.xi) and torch.equal(a.residual, c.residual)


def test_training_reduces_the_loss_and_fallback_never_worse(setup):
    P, M, spec, sf = setup
    torch.manual_seed(0)
    mlp = M.InitMLP(16).cuda()
    hist = M.train(sf, mlp, spec, K=20, n_train_scenes=40 * 16, scenes_per_step=16, lr=1e-3, max_steps=40)
    assert np.mean(hist[-5:]) < np.mean(hist[:5])
    ev = M.evaluate(sf, mlp, spec, K=20, n_scenes=8)
    assert ev["learned_with_fallback"]["median"] <= ev["sample_init"]["median"] + 1e-7
    b = M.make_batch(spec, 77, 4, sf.device)
    xi, lam, res, pick = M.project_with_fallback(sf, mlp, b.xi_bar, b.start, b.goal, b.start_s, b.goal_s, 20,
                                                 n_robots=b.n_robots, n_samples=b.n_samples)
    plain = sf.project(b.xi_bar, b.start, b.goal, 20, n_robots=b.n_robots, n_samples=b.n_samples)
    assert torch.all(res <= plain.residual)


def test_paper_init_network_and_residual_curves(setup):
    """The paper's PointNet-like initialisation network: untrained (eval mode)
    it is the sample initialisation; a few training steps through the
    differentiable SF lower the loss; the residual curves of zero, sample and
    learned initialisation come from the per-iteration history and the
    zero / sample curves equal direct sf_project histories."""
    P, M, spec, sf = setup
    torch.manual_seed(0)
    net = M.make_init_net("pointnet", 16).cuda()
    b = M.make_batch(spec, 321, 4, sf.device)
    net.eval()
    xi0, lam0 = net(b.start_s, b.goal_s, b.xi_bar)
    assert torch.equal(xi0, b.xi_bar) and torch.count_nonzero(lam0) == 0
    net.train()
    hist = M.train(sf, net, spec, K=20, n_train_scenes=30 * 16, scenes_per_step=16, lr=1e-3, max_steps=30)
    assert np.mean(hist[-5:]) < np.mean(hist[:5])
    cur = M.residual_curves(sf, {"pointnet": net}, spec, 20, n_scenes=4, at=(1, 5, 20))
    assert set(cur) == {"zero", "sample", "pointnet"}
    bb = M.make_batch(spec, 5 * 1_000_003, 4, sf.device)
    r = sf.project(bb.xi_bar, bb.start, bb.goal, 20, n_robots=bb.n_robots, n_samples=bb.n_samples, hist=True)
    assert cur["sample"]["20"] == float(r.hist.median(dim=1).values[19])
    for name in cur:
        assert 0 < cur[name]["20"] < cur[name]["1"]
