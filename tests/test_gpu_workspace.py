"""The workspace block (Eq. workspace_con, F_w = I (x) P) on the GPU: parity
of the fused and plain forms (float32, and the bf16 / fp16 tensor-memory form)
with the FP64 oracle on a seeded workload whose samples leave the workspace
spheroid, and the adjoint with workspace rows against FP64 autograd."""
import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_2D, RHO_3D, TOL_RESID_ABS, TOL_XI_REL, lam_err, rel_l2

pytestmark = pytest.mark.gpu

WS3 = ((0.2, -0.1, 0.05), 4.4, 2.2)     # centre, a_w, b_w (3D)
WS2 = ((0.1, -0.2, 0.0), 3.3, 3.3)      # a circle (2D)


@pytest.fixture(scope="module")
def sfmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    P.build()
    return P


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _oracle(O, sc, rho, K, ws, hist=False):
    spec = sc.spec
    pb = O.Problem(dim=spec.dim, n_robots=spec.n_robots, T=spec.T, order=spec.order, t_final=spec.t_final,
                   rho=rho, coll_a=spec.coll, coll_b=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                   use_workspace=True, ws_center=ws[0], ws_a=ws[1], ws_b=ws[2])
    x0 = np.zeros_like(sc.xi_bar) if spec.init == "zero" else None
    return O.run_batch(pb, sc.start, sc.goal, sc.xi_bar, K=K, xi0=x0, hist=hist)


def _run(P, sc, rho, K, ws, form="fused", prec="fp32", hist=False):
    spec = sc.spec
    f = P.SafetyFilter(dim=spec.dim, T=spec.T, rho=rho, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                       max_robots=spec.n_robots, t_final=spec.t_final, precision=prec, workspace=ws)
    x0 = _dev(np.zeros_like(sc.xi_bar)) if spec.init == "zero" else None
    out = f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), K, xi0=x0, form=form, hist=hist)
    torch.cuda.synchronize()
    f.sync_status()
    return out


def _scene3(n_robots=16, n_samples=24, T=100, seed=61, ws=WS3):
    sc = si.scene(si.config_n16_3d(n_robots=n_robots, n_samples=n_samples, T=T, box=(6.0, 6.0, 3.0),
                                   min_sep=1.0), seed)
    c, a, b = ws
    pts = np.concatenate([sc.start, sc.goal]) - np.asarray(c)
    assert np.sqrt((pts[:, 0] ** 2 + pts[:, 1] ** 2) / a ** 2 + pts[:, 2] ** 2 / b ** 2).max() < 0.95
    return sc


def _check(out, ref, tol):
    """tol bounds the xi relative L2 and lambda in units of ||xi_ref|| (the
    tolerance of the mode, as in the other parity tests)."""
    err = rel_l2(out.xi.double().cpu().numpy(), ref["xi"])
    dres = np.abs(out.residual.double().cpu().numpy() - ref["rp_final"])
    assert err.max() <= tol, f"xi rel L2 max {err.max():.3e}"
    lerr = lam_err(out.lam.double().cpu().numpy(), ref["lam"], ref["xi"])
    assert lerr.max() <= tol, f"lambda error max {lerr.max():.3e}"
    assert dres.max() <= TOL_RESID_ABS, f"residual diff max {dres.max():.3e}"


@pytest.mark.parametrize("form", ["fused", "plain"])
def test_workspace_3d_float32(sfmod, oracle_lib, form):
    sc = _scene3()
    ref = _oracle(oracle_lib, sc, RHO_3D, 60, WS3, hist=True)
    # the workload exercises the block: the samples start outside
    assert ref["proj_hist"][:, 0].min() > 0
    out = _run(sfmod, sc, RHO_3D, 60, WS3, form=form, hist=True)
    _check(out, ref, TOL_XI_REL)
    h = out.hist.double().cpu().numpy().T
    np.testing.assert_allclose(h, ref["proj_hist"], rtol=1e-3, atol=1e-4)


def test_workspace_3d_n32(sfmod, oracle_lib):
    """27 robots (the 32-robot bucket, positions staged in shared memory)."""
    ws = ((0.0, 0.0, 0.0), 5.0, 3.0)
    sc = _scene3(n_robots=27, n_samples=6, T=64, seed=63, ws=ws)
    ref = _oracle(oracle_lib, sc, RHO_3D, 40, ws, hist=True)
    assert ref["proj_hist"][:, 0].min() > 0
    _check(_run(sfmod, sc, RHO_3D, 40, ws), ref, TOL_XI_REL)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_workspace_3d_tensor_core(sfmod, oracle_lib, prec):
    sc = _scene3()
    ref = _oracle(oracle_lib, sc, RHO_3D, 60, WS3)
    _check(_run(sfmod, sc, RHO_3D, 60, WS3, prec=prec), ref, 5e-3)


@pytest.mark.parametrize("form", ["fused", "plain"])
def test_workspace_2d(sfmod, oracle_lib, form):
    sc = si.scene(si.config_small_2d(), 0)
    ref = _oracle(oracle_lib, sc, RHO_2D, 100, WS2)
    _check(_run(sfmod, sc, RHO_2D, 100, WS2, form=form), ref, TOL_XI_REL)


def test_workspace_adjoint_matches_autograd(sfmod, oracle_lib):
    """dL/dxi_bar through K iterations with workspace rows active: the adjoint
    kernel (activity masks) against autograd over the FP64 PyTorch unroll."""
    from paper_2501_19042_gb300.autograd import sf_unroll
    from torch_unroll import TorchSF
    P = sfmod
    ws = ((0.1, 0.0, 0.0), 2.0, 1.2)
    sc = si.scene(si.config_n16_3d(n_robots=5, n_samples=6, T=40, box=(3.0, 3.0, 1.5), min_sep=0.8), 12)
    pts = np.concatenate([sc.start, sc.goal]) - np.asarray(ws[0])
    assert np.sqrt((pts[:, 0] ** 2 + pts[:, 1] ** 2) / 2.0 ** 2 + pts[:, 2] ** 2 / 1.2 ** 2).max() < 0.95
    K = 20
    rng = np.random.default_rng(3)
    gxi = torch.tensor(rng.normal(size=sc.xi_bar.shape))
    Pm, Pd, Pdd = oracle_lib.basis(10, sc.spec.T, sc.spec.t_final)
    ts = TorchSF(Pm, Pd, Pdd, sc.start, sc.goal, RHO_3D, sc.spec.coll, sc.spec.coll, sc.spec.v_max,
                 sc.spec.a_max, workspace=ws)
    xbv = torch.tensor(sc.xi_bar).requires_grad_(True)
    xi_t, _, _ = ts.unroll(xbv, torch.zeros_like(xbv), xbv, K)
    (g_ref,) = torch.autograd.grad((gxi * xi_t).sum(), [xbv])
    f = P.SafetyFilter(dim=3, T=sc.spec.T, rho=RHO_3D, coll_a=sc.spec.coll, max_robots=8, checkpoint_every=5,
                       workspace=ws)
    xbd = _dev(sc.xi_bar).requires_grad_(True)
    xi, lam, fp, res = sf_unroll(f, xbd, _dev(sc.start), _dev(sc.goal), K)
    np.testing.assert_allclose(xi.detach().double().cpu().numpy(), xi_t.detach().numpy(), rtol=0, atol=2e-4)
    (_dev(gxi.numpy()) * xi).sum().backward()
    a = xbd.grad.double().cpu().reshape(6, -1)
    b = g_ref.reshape(6, -1)
    assert ((a - b).norm(dim=1) / b.norm(dim=1)).max().item() <= 2e-3


@pytest.mark.parametrize("n_robots,seed,ws", [(16, 61, WS3), (27, 63, ((0.0, 0.0, 0.0), 5.0, 3.0))])
def test_workspace_pruning_is_exact(sfmod, n_robots, seed, ws):
    """Pair and workspace-row pruning give the same xi, lambda, residual and
    history as testing every row every iteration."""
    sc = _scene3(n_robots=n_robots, n_samples=12, T=80, seed=seed, ws=ws)
    outs = []
    for prune in (True, False):
        spec = sc.spec
        f = sfmod.SafetyFilter(dim=3, T=spec.T, rho=RHO_3D, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                               max_robots=spec.n_robots, t_final=spec.t_final, workspace=ws)
        f.set_pair_pruning(prune)
        outs.append(f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 150, hist=True))
        torch.cuda.synchronize()
    a, b = outs
    assert torch.equal(a.xi, b.xi) and torch.equal(a.lam, b.lam)
    assert torch.equal(a.residual, b.residual)
    # the history sums squared residuals; above 16 robots the full test sums
    # them in block order, the candidate path in row order
    torch.testing.assert_close(a.hist, b.hist, rtol=1e-5, atol=1e-7)
