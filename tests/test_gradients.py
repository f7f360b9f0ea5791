"""Gradients of the unrolled SF.

CPU: central finite differences of the FP64 oracle pin the FP64 PyTorch
unroll (tests/torch_unroll.py) and its autograd gradients.
GPU: the hand-written adjoint kernel (sf_project_backward, through the
autograd Function) against autograd over that FP64 unroll, including the
fixed-point-residual term of Eq. (NN_loss).
"""
import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_3D
from torch_unroll import TorchSF


def _instance(N=3, S=2, T=30, seed=5):
    spec = si.config_n16_3d(n_robots=N, n_samples=S, T=T, box=(3.0, 3.0, 1.5), min_sep=0.8)
    return si.scene(spec, seed)


def _tsf(O, sc, rho=RHO_3D):
    P, Pd, Pdd = O.basis(10, sc.spec.T, sc.spec.t_final)
    return TorchSF(P, Pd, Pdd, sc.start, sc.goal, rho, sc.spec.coll, sc.spec.coll, sc.spec.v_max, sc.spec.a_max)


@pytest.mark.parametrize("ws", [None, ((0.1, 0.0, 0.0), 1.6, 1.0)])
def test_torch_unroll_forward_and_gradient_match_oracle_fd(oracle_lib, ws):
    """The FP64 unroll (with and without workspace rows) against the oracle's
    forward and central finite differences of it."""
    O = oracle_lib
    sc = _instance()
    K = 15
    P_, Pd_, Pdd_ = O.basis(10, sc.spec.T, sc.spec.t_final)
    ts = TorchSF(P_, Pd_, Pdd_, sc.start, sc.goal, RHO_3D, sc.spec.coll, sc.spec.coll, sc.spec.v_max,
                 sc.spec.a_max, workspace=ws)
    rng = np.random.default_rng(0)
    xb = torch.tensor(sc.xi_bar[:1])
    x0 = xb.clone() + torch.tensor(rng.normal(size=xb.shape) * 0.05)
    l0 = torch.tensor(rng.normal(size=xb.shape) * 0.01)
    w = torch.tensor(rng.normal(size=xb.shape))
    x0.requires_grad_(True)
    xbv = xb.clone().requires_grad_(True)
    xi, lam, _ = ts.unroll(x0, l0, xbv, K)
    wkw = {} if ws is None else dict(use_workspace=True, ws_center=ws[0], ws_a=ws[1], ws_b=ws[2])
    pb = O.Problem(dim=3, n_robots=sc.spec.n_robots, T=sc.spec.T, rho=RHO_3D, coll_a=sc.spec.coll,
                   coll_b=sc.spec.coll, **wkw)
    sf = O.OracleSF(pb, sc.start, sc.goal)
    if ws is not None:   # the workspace rows are active on this input
        P0 = np.asarray(P_)
        pos = np.einsum("tk,dnk->ntd", P0, x0.detach()[0].numpy()) - np.asarray(ws[0])
        assert (np.sqrt((pos[..., 0] ** 2 + pos[..., 1] ** 2) / ws[1] ** 2 + pos[..., 2] ** 2 / ws[2] ** 2) > 1).any()
    ref = sf.run(xb[0].numpy().reshape(-1), K, xi0=x0.detach()[0].numpy().reshape(-1), lam0=l0[0].numpy().reshape(-1))
    np.testing.assert_allclose(xi.detach().numpy().reshape(-1), ref["xi"], atol=1e-12)
    L = (w * xi).sum()
    gx0, gxb = torch.autograd.grad(L, [x0, xbv])

    def loss(x0v, xbv_):
        r = sf.run(xbv_.reshape(-1), K, xi0=x0v.reshape(-1), lam0=l0[0].numpy().reshape(-1))
        return float((w[0].numpy().reshape(-1) * r["xi"]).sum())

    h = 1e-6
    base_x0 = x0.detach()[0].numpy().copy()
    base_xb = xb[0].numpy().copy()
    for flat in rng.choice(base_x0.size, 8, replace=False):
        idx = np.unravel_index(flat, base_x0.shape)
        for which, g in (("x0", gx0), ("xb", gxb)):
            a, b = base_x0.copy(), base_xb.copy()
            arr = a if which == "x0" else b
            arr[idx] += h
            fp = loss(a, b)
            arr[idx] -= 2 * h
            fm = loss(a, b)
            fd = (fp - fm) / (2 * h)
            assert abs(fd - float(g[0][idx])) <= 1e-6 + 1e-5 * abs(fd), (which, idx, fd, float(g[0][idx]))


@pytest.mark.parametrize("coll_b", [0.35, 0.8])
def test_torch_unroll_ellipsoid_matches_oracle(oracle_lib, coll_b):
    """With unequal collision semi-axes (a, a, b) the FP64 unroll equals the
    oracle's forward (the literal atan2 / sin / cos closed forms of the
    alpha / beta / d steps) on an input whose pair rows are active."""
    O = oracle_lib
    sc = _instance(N=4, S=2, T=30, seed=5)
    K = 12
    P_, Pd_, Pdd_ = O.basis(10, sc.spec.T, sc.spec.t_final)
    ts = TorchSF(P_, Pd_, Pdd_, sc.start, sc.goal, RHO_3D, sc.spec.coll, coll_b, sc.spec.v_max, sc.spec.a_max)
    xb = torch.tensor(sc.xi_bar)
    q0 = ts.project_q(xb)["pair"]
    assert (q0.abs() > 0).any()
    xi, lam, _ = ts.unroll(xb.clone(), torch.zeros_like(xb), xb, K)
    pb = O.Problem(dim=3, n_robots=sc.spec.n_robots, T=sc.spec.T, rho=RHO_3D, coll_a=sc.spec.coll, coll_b=coll_b)
    ref = O.run_batch(pb, sc.start, sc.goal, sc.xi_bar, K=K)
    np.testing.assert_allclose(xi.numpy(), ref["xi"], atol=1e-11)
    np.testing.assert_allclose(lam.numpy(), ref["lam"], atol=1e-11)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def sfmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    P.build()
    return P


def _torch_grads(ts, xb, x0, l0, K, gxi, glam, gfp, sample_init):
    xbv = xb.clone().double().requires_grad_(True)
    if sample_init:
        xi, lam, fp = ts.unroll(xbv, torch.zeros_like(xbv), xbv, K, fp_weight=1.0)
        L = (gxi * xi).sum() + (glam * lam).sum() + (gfp * fp).sum()
        (g_xb,) = torch.autograd.grad(L, [xbv])
        return None, None, g_xb, fp
    x0v = x0.clone().double().requires_grad_(True)
    l0v = l0.clone().double().requires_grad_(True)
    xi, lam, fp = ts.unroll(x0v, l0v, xbv, K, fp_weight=1.0)
    L = (gxi * xi).sum() + (glam * lam).sum() + (gfp * fp).sum()
    return (*torch.autograd.grad(L, [x0v, l0v, xbv]), fp)


def _rel(a, b):
    a = a.detach().double().cpu().reshape(a.shape[0], -1)
    b = b.detach().double().cpu().reshape(b.shape[0], -1)
    return ((a - b).norm(dim=1) / b.norm(dim=1).clamp_min(1e-30)).max().item()


@pytest.mark.gpu
@pytest.mark.parametrize("sample_init", [False, True])
def test_adjoint_kernel_matches_autograd(sfmod, oracle_lib, sample_init):
    from paper_2501_19042_gb300.autograd import sf_unroll
    P = sfmod
    sc = _instance(N=5, S=6, T=40, seed=8)
    K = 20
    rng = np.random.default_rng(1)
    xb = torch.tensor(sc.xi_bar)
    x0 = xb + torch.tensor(rng.normal(size=xb.shape) * 0.05)
    l0 = torch.tensor(rng.normal(size=xb.shape) * 0.01)
    gxi = torch.tensor(rng.normal(size=xb.shape))
    glam = torch.tensor(rng.normal(size=xb.shape))
    gfp = torch.tensor(rng.uniform(0.1, 1.0, size=xb.shape[0]))
    ts = _tsf(oracle_lib, sc)
    r_x0, r_l0, r_xb, r_fp = _torch_grads(ts, xb, x0, l0, K, gxi, glam, gfp, sample_init)
    f = P.SafetyFilter(dim=3, T=sc.spec.T, rho=RHO_3D, coll_a=sc.spec.coll, max_robots=8, checkpoint_every=5)
    xbd = _dev(sc.xi_bar).requires_grad_(True)
    x0d = None if sample_init else _dev(x0.numpy()).requires_grad_(True)
    l0d = None if sample_init else _dev(l0.numpy()).requires_grad_(True)
    xi, lam, fp, res = sf_unroll(f, xbd, _dev(sc.start), _dev(sc.goal), K, xi0=x0d, lam0=l0d)
    np.testing.assert_allclose(fp.detach().double().cpu().numpy(), r_fp.detach().numpy(), rtol=2e-4, atol=1e-6)
    L = (_dev(gxi.numpy()) * xi).sum() + (_dev(glam.numpy()) * lam).sum() + (_dev(gfp.numpy()) * fp).sum()
    L.backward()
    assert _rel(xbd.grad, r_xb) <= 2e-3
    if not sample_init:
        assert _rel(x0d.grad, r_x0) <= 2e-3
        assert _rel(l0d.grad, r_l0) <= 2e-3


@pytest.mark.gpu
def test_adjoint_full_size_sampled(sfmod, oracle_lib):
    """The differentiation workload (N=16, S=512, K=50, checkpoint every 10)
    at full size; 3 sampled samples against FP64 autograd one by one."""
    from paper_2501_19042_gb300.autograd import sf_unroll
    P = sfmod
    spec = si.config_diff()
    sc = si.scene(spec, 5)
    K = spec.K
    rng = np.random.default_rng(2)
    gxi = rng.normal(size=sc.xi_bar.shape)
    f = P.SafetyFilter(dim=3, T=spec.T, rho=RHO_3D, coll_a=spec.coll, max_robots=16, checkpoint_every=10)
    xbd = _dev(sc.xi_bar).requires_grad_(True)
    xi, lam, fp, res = sf_unroll(f, xbd, _dev(sc.start), _dev(sc.goal), K)
    (_dev(gxi) * xi).sum().backward()
    ts = _tsf(oracle_lib, sc)
    for s in (0, 255, 511):
        xb = torch.tensor(sc.xi_bar[s:s + 1])
        _, _, r_xb, _ = _torch_grads(ts, xb, None, None, K, torch.tensor(gxi[s:s + 1]), torch.zeros_like(xb),
                                     torch.zeros(1, dtype=torch.float64), True)
        assert _rel(xbd.grad[s:s + 1], r_xb) <= 2e-3, s
