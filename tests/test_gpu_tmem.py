"""Parity of the tensor-memory form of the fused forward (coefficient-to-state
products on tcgen05 tensor cores, accumulators in TMEM; option
SF_OPT_TENSOR_MEMORY) with the FP64 oracle on the same seeded inputs.
float32 handles (tf32 operands, three-term split): the float32 bounds
(xi relative L2 <= 1e-4, lambda <= 1e-4 ||xi_ref||, final ||r_p|| within
1e-3); bf16 / fp16 handles: the mixed-precision bounds (5e-3)."""
import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_2D, RHO_3D, TOL_RESID_ABS, TOL_XI_REL, lam_err, rel_l2, run_oracle

pytestmark = pytest.mark.gpu

TOL = {"fp32": TOL_XI_REL, "bf16": 5e-3, "fp16": 5e-3}


@pytest.fixture(scope="module")
def sfmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    P.build()
    return P


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _filter(P, spec, rho, prec="fp32", max_robots=None, coll_b=None, tm=True):
    f = P.SafetyFilter(dim=spec.dim, T=spec.T, rho=rho, coll_a=spec.coll, coll_b=coll_b, v_max=spec.v_max,
                       a_max=spec.a_max, max_robots=max_robots or spec.n_robots, t_final=spec.t_final,
                       precision=prec)
    f.set_tensor_memory(tm)
    return f


def _run(P, sc, rho, K, prec="fp32", hist=False, coll_b=None):
    f = _filter(P, sc.spec, rho, prec, coll_b=coll_b)
    x0 = _dev(np.zeros_like(sc.xi_bar)) if sc.spec.init == "zero" else None
    out = f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), K, xi0=x0, hist=hist)
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
    assert err.max() <= tol, f"xi rel L2 max {err.max():.3e} median {np.median(err):.3e}"
    lerr = lam_err(lam, ref["lam"], ref["xi"])
    assert lerr.max() <= tol, f"lambda error max {lerr.max():.3e}"
    dres = np.abs(res - ref["rp_final"])
    assert dres.max() <= TOL_RESID_ABS, f"residual diff max {dres.max():.3e}"
    return err


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_small_2d_zero_init(sfmod, oracle_lib, prec):
    """2D, N=4, zero init (every pair at delta = 0 in iteration 1), with the
    residual history."""
    sc = si.scene(si.config_small_2d(), 0)
    ref = run_oracle(oracle_lib, sc, RHO_2D, 100, hist=True)
    out = _run(sfmod, sc, RHO_2D, 100, prec, hist=True)
    _check(out, ref, TOL[prec])
    h = out.hist.double().cpu().numpy().T
    if prec == "fp32":
        np.testing.assert_allclose(h, ref["proj_hist"], rtol=1e-3, atol=1e-4)
    else:
        assert np.abs(h - ref["proj_hist"]).max() <= 5e-3


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_n16_3d_small_batch(sfmod, oracle_lib, prec):
    """3D, N=16, 24 samples (several CTAs, a ragged time tail), K=60."""
    sc = si.scene(si.config_n16_3d(n_samples=24), 1)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 60)
    _check(_run(sfmod, sc, RHO_3D, 60, prec), ref, TOL[prec])


@pytest.mark.parametrize("N,T", [(1, 50), (2, 33), (5, 64), (9, 31), (17, 97), (27, 120)])
def test_edge_sizes(sfmod, oracle_lib, N, T):
    """Robot counts across the buckets and off the lane quarters, time steps
    below, at and off the chunk and 8-step block sizes."""
    spec = si.config_n16_3d(n_robots=N, n_samples=5, T=T, box=(6.0, 6.0, 3.0), min_sep=0.8)
    sc = si.scene(spec, 40 + N)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 30)
    _check(_run(sfmod, sc, RHO_3D, 30), ref, TOL_XI_REL)


def test_n32_t120(sfmod, oracle_lib):
    sc = si.scene(si.config_n32_3d(n_samples=16), 3)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 40)
    _check(_run(sfmod, sc, RHO_3D, 40), ref, TOL_XI_REL)


def test_ellipsoid(sfmod, oracle_lib):
    sc = si.scene(si.config_n16_3d(n_samples=24), 1)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 60, coll_b=0.35)
    _check(_run(sfmod, sc, RHO_3D, 60, coll_b=0.35), ref, TOL_XI_REL)


def test_n16_full_size_sampled(sfmod, oracle_lib):
    """The bench workload at full size (S=1024, K=200): 8 sampled outputs
    against the oracle one by one, and the median final residual below 1e-3."""
    sc = si.scene(si.config_n16_3d(), 1)
    out = _run(sfmod, sc, RHO_3D, 200)
    idx = np.array([0, 1, 137, 300, 511, 700, 901, 1023])
    ref = run_oracle(oracle_lib, sc, RHO_3D, 200, idx=idx)
    _check(out, ref, TOL_XI_REL, idx)
    assert torch.isfinite(out.xi).all() and float(out.residual.median()) < 1e-3


def test_ragged_multi_scene_batch(sfmod, oracle_lib):
    """Scenes of every bucket (one empty) in one call, each against its own
    oracle run."""
    P = sfmod
    specs = [si.config_n16_3d(n_robots=n, n_samples=s, K=25) for n, s in
             [(8, 7), (13, 3), (16, 0), (24, 5), (32, 2), (3, 9)]]
    st = si.Stream(7)
    scenes = [si.make_scene(sp, st) for sp in specs]
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=32)
    f.set_tensor_memory(True)
    xb = np.concatenate([s.xi_bar.reshape(-1) for s in scenes])
    nr = [s.spec.n_robots for s in scenes]
    ns = [s.spec.n_samples for s in scenes]
    out = f.project(_dev(xb), _dev(np.concatenate([s.start for s in scenes])),
                    _dev(np.concatenate([s.goal for s in scenes])), 25, n_robots=nr, n_samples=ns)
    torch.cuda.synchronize()
    f.sync_status()
    xi = out.xi.double().cpu().numpy()
    lam = out.lam.double().cpu().numpy()
    res = out.residual.double().cpu().numpy()
    c0 = s0 = 0
    for s in scenes:
        S, N = s.spec.n_samples, s.spec.n_robots
        n = S * 3 * N * 11
        if S:
            ref = run_oracle(oracle_lib, s, RHO_3D, 25)
            assert rel_l2(xi[c0:c0 + n].reshape(S, -1), ref["xi"]).max() <= TOL_XI_REL, N
            assert lam_err(lam[c0:c0 + n].reshape(S, -1), ref["lam"], ref["xi"]).max() <= TOL_XI_REL, N
            assert np.abs(res[s0:s0 + S] - ref["rp_final"]).max() <= TOL_RESID_ABS
        c0 += n
        s0 += S


def test_pruning_is_exact_in_tensor_memory_form(sfmod):
    """With the tensor-memory form too, testing only candidate pair rows
    between full tests gives the same xi, lambda and residual as testing
    every row."""
    P = sfmod
    sc = si.scene(si.config_n16_3d(n_samples=40), 1)
    outs = []
    for prune in (True, False):
        f = _filter(P, sc.spec, RHO_3D)
        f.set_pair_pruning(prune)
        outs.append(f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 120))
        torch.cuda.synchronize()
    a, b = outs
    assert torch.equal(a.xi, b.xi) and torch.equal(a.lam, b.lam) and torch.equal(a.residual, b.residual)


def test_deterministic(sfmod):
    P = sfmod
    sc = si.scene(si.config_n16_3d(n_samples=40), 9)
    f = _filter(P, sc.spec, RHO_3D)
    a = f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 20)
    b = f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 20)
    torch.cuda.synchronize()
    assert torch.equal(a.xi, b.xi) and torch.equal(a.lam, b.lam) and torch.equal(a.residual, b.residual)


def _torch_ref_grads(oracle_lib, sc, K, gxi, glam, gfp):
    from torch_unroll import TorchSF
    Pm, Pd, Pdd = oracle_lib.basis(10, sc.spec.T, sc.spec.t_final)
    ts = TorchSF(Pm, Pd, Pdd, sc.start, sc.goal, RHO_3D, sc.spec.coll, sc.spec.coll, sc.spec.v_max, sc.spec.a_max)
    xbv = torch.tensor(sc.xi_bar).requires_grad_(True)
    xi, lam, fp = ts.unroll(xbv, torch.zeros_like(xbv), xbv, K, fp_weight=1.0)
    L = (gxi * xi).sum() + (glam * lam).sum() + (gfp * fp).sum()
    (g,) = torch.autograd.grad(L, [xbv])
    return g, fp.detach()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_training_forward_and_adjoint(sfmod, oracle_lib, prec):
    """The differentiable SF with the tensor-memory training forward
    (checkpoints, activity masks and the fixed-point residual sum written by
    the MMA form) and the float32 adjoint: dL/dxi_bar against autograd over
    the FP64 PyTorch unroll (relative L2 <= 2e-3, the float32 adjoint's bound,
    in every mode), the fixed-point residual against the unroll's."""
    from paper_2501_19042_gb300.autograd import sf_unroll
    P = sfmod
    sc = si.scene(si.config_n16_3d(n_robots=5, n_samples=6, T=40, box=(3.0, 3.0, 1.5), min_sep=0.8), 8)
    K = 20
    rng = np.random.default_rng(1)
    gxi = torch.tensor(rng.normal(size=sc.xi_bar.shape))
    glam = torch.tensor(rng.normal(size=sc.xi_bar.shape))
    gfp = torch.tensor(rng.uniform(0.1, 1.0, size=sc.xi_bar.shape[0]))
    g_ref, fp_ref = _torch_ref_grads(oracle_lib, sc, K, gxi, glam, gfp)
    f = P.SafetyFilter(dim=3, T=sc.spec.T, rho=RHO_3D, coll_a=sc.spec.coll, max_robots=8, checkpoint_every=5,
                       precision=prec)
    f.set_tensor_memory(True)
    xbd = _dev(sc.xi_bar).requires_grad_(True)
    xi, lam, fp, res = sf_unroll(f, xbd, _dev(sc.start), _dev(sc.goal), K)
    f.sync_status()
    np.testing.assert_allclose(fp.detach().double().cpu().numpy(), fp_ref.numpy(), rtol=2e-3, atol=1e-5)
    L = (_dev(gxi.numpy()) * xi).sum() + (_dev(glam.numpy()) * lam).sum() + (_dev(gfp.numpy()) * fp).sum()
    L.backward()
    a = xbd.grad.double().cpu().reshape(6, -1)
    b = g_ref.reshape(6, -1)
    assert ((a - b).norm(dim=1) / b.norm(dim=1)).max().item() <= 2e-3


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_training_forward_full_size_sampled(sfmod, oracle_lib, prec):
    """The differentiation workload (N=16, S=512, K=50, checkpoint every 10)
    through the tensor-memory training forward and the adjoint; 2 sampled
    samples against FP64 autograd one by one."""
    from paper_2501_19042_gb300.autograd import sf_unroll
    from torch_unroll import TorchSF
    P = sfmod
    spec = si.config_diff()
    sc = si.scene(spec, 5)
    K = spec.K
    rng = np.random.default_rng(2)
    gxi = rng.normal(size=sc.xi_bar.shape)
    f = P.SafetyFilter(dim=3, T=spec.T, rho=RHO_3D, coll_a=spec.coll, max_robots=16, checkpoint_every=10,
                       precision=prec)
    f.set_tensor_memory(True)
    xbd = _dev(sc.xi_bar).requires_grad_(True)
    xi, lam, fp, res = sf_unroll(f, xbd, _dev(sc.start), _dev(sc.goal), K)
    (_dev(gxi) * xi).sum().backward()
    f.sync_status()
    Pm, Pd, Pdd = oracle_lib.basis(10, spec.T, spec.t_final)
    ts = TorchSF(Pm, Pd, Pdd, sc.start, sc.goal, RHO_3D, spec.coll, spec.coll, spec.v_max, spec.a_max)
    for s in (0, 511):
        xb = torch.tensor(sc.xi_bar[s:s + 1]).requires_grad_(True)
        x, _, _ = ts.unroll(xb, torch.zeros_like(xb), xb, K)
        (g,) = torch.autograd.grad((torch.tensor(gxi[s:s + 1]) * x).sum(), [xb])
        a = xbd.grad[s:s + 1].double().cpu().reshape(-1)
        assert ((a - g.reshape(-1)).norm() / g.norm()).item() <= 2e-3, s


def test_default_form_per_bucket(sfmod):
    """A float32 handle's default (SF_OPT_TENSOR_MEMORY = 2) takes the
    tensor-memory form for 3D scenes of 9..24 robots when its launch shape
    fills at least 96 TMEM lanes per CTA, the float32 form otherwise; each
    launch gives the bits of the explicit choice."""
    P = sfmod
    cases = [(3, 16, 1024, 50, True), (3, 12, 1024, 100, True), (3, 20, 1024, 50, True),
             (3, 16, 64, 100, False), (3, 8, 1024, 100, False), (3, 32, 256, 50, False),
             (2, 16, 1024, 100, False)]
    for dim, N, S, K, want in cases:
        spec = si.config_n16_3d(n_robots=N, n_samples=S) if dim == 3 else \
            si.config_small_2d(n_robots=N, n_samples=S, circle_radius=5.0)
        sc = si.scene(spec, 9)
        args = (_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal))
        f = _filter(P, spec, RHO_3D, tm="auto")
        out = f.project(*args, K)
        f.sync_status()
        assert f.launch_shape()["tensor_memory"] == want, (dim, N, S, K)
        g = _filter(P, spec, RHO_3D, tm=want)
        ref = g.project(*args, K)
        g.sync_status()
        assert torch.equal(out.xi, ref.xi) and torch.equal(out.lam, ref.lam), (dim, N, S, K)
