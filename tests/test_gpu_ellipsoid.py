"""The collision spheroid with unequal semi-axes (a, a, b), a != b
(Eq. inter_robot_con, M_a = diag(a, a, b)), on the GPU: the fused and plain
forms in float32 and the 16-bit tensor-memory forms against the FP64 oracle,
and the adjoint against autograd over the FP64 PyTorch unroll. For a != b
the pair rows take the scaled-coordinate closed forms of the alpha / beta /
d steps: e = delta outside the spheroid, the radial projection in scaled
coordinates inside."""
import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_3D, TOL_LAM, TOL_RESID_ABS, TOL_XI_REL, lam_err, rel_l2, run_oracle

pytestmark = pytest.mark.gpu

TOL_MIXED = 5e-3


@pytest.fixture(scope="module")
def sfmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    P.build()
    return P


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _run(P, sc, K, coll_b, form="fused", prec="fp32"):
    spec = sc.spec
    f = P.SafetyFilter(dim=3, T=spec.T, rho=RHO_3D, coll_a=spec.coll, coll_b=coll_b, v_max=spec.v_max,
                       a_max=spec.a_max, max_robots=spec.n_robots, t_final=spec.t_final, precision=prec)
    out = f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), K, form=form)
    torch.cuda.synchronize()
    f.sync_status()
    return out


def _check(out, ref, tol, idx=None):
    xi = out.xi.double().cpu().numpy()
    lam = out.lam.double().cpu().numpy()
    res = out.residual.double().cpu().numpy()
    if idx is not None:
        xi, lam, res = xi[idx], lam[idx], res[idx]
    err = rel_l2(xi, ref["xi"])
    assert err.max() <= tol, f"xi rel L2 max {err.max():.3e}"
    lerr = lam_err(lam, ref["lam"], ref["xi"])
    assert lerr.max() <= tol, f"lambda error max {lerr.max():.3e}"
    assert np.abs(res - ref["rp_final"]).max() <= TOL_RESID_ABS


def _active_pairs(sc, coll_b):
    """Pair rows of the input samples inside the spheroid (the workload
    exercises the block)."""
    import oracle as O
    P, _, _ = O.basis(10, sc.spec.T, sc.spec.t_final)
    p = np.einsum("tk,sdnk->sntd", P, sc.xi_bar)
    d = p[:, :, None] - p[:, None, :]
    a = sc.spec.coll
    s2 = (d[..., 0] ** 2 + d[..., 1] ** 2) / a ** 2 + d[..., 2] ** 2 / coll_b ** 2
    iu = np.triu_indices(sc.spec.n_robots, 1)
    return int((s2[:, iu[0], iu[1]] < 1).sum())


@pytest.mark.parametrize("form", ["fused", "plain"])
@pytest.mark.parametrize("coll_b", [0.35, 0.8])
def test_ellipsoid_small(sfmod, oracle_lib, form, coll_b):
    """N=4 in a tight box (pairs active from the start), S=8, K=60, both an
    oblate (b < a) and a prolate (b > a) spheroid."""
    sc = si.scene(si.config_n16_3d(n_robots=4, n_samples=8, T=64, box=(2.5, 2.5, 1.2), min_sep=0.7), 21)
    assert _active_pairs(sc, coll_b) > 0
    ref = run_oracle(oracle_lib, sc, RHO_3D, 60, coll_b=coll_b)
    _check(_run(sfmod, sc, 60, coll_b, form=form), ref, TOL_XI_REL)


@pytest.mark.parametrize("form", ["fused", "plain"])
def test_ellipsoid_n16(sfmod, oracle_lib, form):
    """N=16, 24 samples (several CTAs, a ragged time tail), K=60, b = 0.35."""
    sc = si.scene(si.config_n16_3d(n_samples=24), 1)
    assert _active_pairs(sc, 0.35) > 0
    ref = run_oracle(oracle_lib, sc, RHO_3D, 60, coll_b=0.35)
    _check(_run(sfmod, sc, 60, 0.35, form=form), ref, TOL_XI_REL)


def test_ellipsoid_n16_full_size_sampled(sfmod, oracle_lib):
    """The bench workload's shape (N=16, S=1024, K=200) with b = 0.35;
    6 sampled outputs against the oracle one by one."""
    sc = si.scene(si.config_n16_3d(), 1)
    out = _run(sfmod, sc, 200, 0.35)
    idx = np.array([0, 5, 333, 640, 999, 1023])
    ref = run_oracle(oracle_lib, sc, RHO_3D, 200, idx=idx, coll_b=0.35)
    _check(out, ref, TOL_XI_REL, idx)
    assert torch.isfinite(out.xi).all()


def test_ellipsoid_n32_full_size_sampled(sfmod, oracle_lib):
    """The precision workload's shape (N=32, S=2048, T=120, K=200) with
    b = 0.35 (the 32-robot bucket, positions staged in shared memory);
    4 sampled outputs."""
    sc = si.scene(si.config_n32_3d(), 3)
    out = _run(sfmod, sc, 200, 0.35)
    idx = np.array([0, 700, 1500, 2047])
    ref = run_oracle(oracle_lib, sc, RHO_3D, 200, idx=idx, coll_b=0.35)
    _check(out, ref, TOL_XI_REL, idx)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_ellipsoid_tensor_core(sfmod, oracle_lib, prec):
    sc = si.scene(si.config_n16_3d(n_samples=24), 1)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 60, coll_b=0.35)
    _check(_run(sfmod, sc, 60, 0.35, prec=prec), ref, TOL_MIXED)


@pytest.mark.parametrize("coll_b", [0.35, 0.8])
def test_ellipsoid_adjoint_matches_autograd(sfmod, oracle_lib, coll_b):
    """dL/dxi_bar through K iterations with a != b: the adjoint kernel
    against autograd over the FP64 PyTorch unroll (scaled-coordinate
    projection, its Jacobian inside the spheroid)."""
    from paper_2501_19042_gb300.autograd import sf_unroll
    from torch_unroll import TorchSF
    P = sfmod
    sc = si.scene(si.config_n16_3d(n_robots=5, n_samples=6, T=40, box=(3.0, 3.0, 1.5), min_sep=0.8), 8)
    assert _active_pairs(sc, coll_b) > 0
    K = 20
    rng = np.random.default_rng(4)
    gxi = torch.tensor(rng.normal(size=sc.xi_bar.shape))
    Pm, Pd, Pdd = oracle_lib.basis(10, sc.spec.T, sc.spec.t_final)
    ts = TorchSF(Pm, Pd, Pdd, sc.start, sc.goal, RHO_3D, sc.spec.coll, coll_b, sc.spec.v_max, sc.spec.a_max)
    xbv = torch.tensor(sc.xi_bar).requires_grad_(True)
    xi_t, _, _ = ts.unroll(xbv, torch.zeros_like(xbv), xbv, K)
    (g_ref,) = torch.autograd.grad((gxi * xi_t).sum(), [xbv])
    f = P.SafetyFilter(dim=3, T=sc.spec.T, rho=RHO_3D, coll_a=sc.spec.coll, coll_b=coll_b, max_robots=8,
                       checkpoint_every=5)
    xbd = _dev(sc.xi_bar).requires_grad_(True)
    xi, lam, fp, res = sf_unroll(f, xbd, _dev(sc.start), _dev(sc.goal), K)
    np.testing.assert_allclose(xi.detach().double().cpu().numpy(), xi_t.detach().numpy(), rtol=0, atol=2e-4)
    (_dev(gxi.numpy()) * xi).sum().backward()
    a = xbd.grad.double().cpu().reshape(6, -1)
    b = g_ref.reshape(6, -1)
    assert ((a - b).norm(dim=1) / b.norm(dim=1)).max().item() <= 2e-3
