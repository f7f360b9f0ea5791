"""Parity of the tensor-memory form (bf16 / fp16 MMA operands, float32
accumulation) with the FP64 oracle on the same seeded inputs: per-sample
relative L2 of xi^K <= 5e-3, ||lambda^K - lambda_ref|| <= 5e-3 ||xi_ref||
and final ||r_p|| within 1e-3 (absolute) of the oracle's. The float32 form's
bound (1e-4) is not asked of these modes."""
import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_2D, RHO_3D, TOL_RESID_ABS, lam_err, rel_l2, run_oracle

pytestmark = pytest.mark.gpu

TOL_XI_REL_MIXED = 5e-3
TOL_LAM_MIXED = TOL_XI_REL_MIXED   # lambda in units of ||xi_ref||, as in the float32 tests
PRECS = ("bf16", "fp16")


@pytest.fixture(scope="module")
def sfmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    P.build()
    return P


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _run(P, sc, rho, K, prec, max_robots=None, hist=False):
    spec = sc.spec
    f = P.SafetyFilter(dim=spec.dim, T=spec.T, rho=rho, coll_a=spec.coll, v_max=spec.v_max,
                       a_max=spec.a_max, max_robots=max_robots or spec.n_robots, t_final=spec.t_final,
                       precision=prec)
    x0 = _dev(np.zeros_like(sc.xi_bar)) if spec.init == "zero" else None
    out = f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), K, xi0=x0, hist=hist)
    torch.cuda.synchronize()
    f.sync_status()
    return out


def _check(out, ref, idx=None):
    xi = out.xi.double().cpu().numpy()
    lam = out.lam.double().cpu().numpy()
    res = out.residual.double().cpu().numpy()
    if idx is not None:
        xi, lam, res = xi[idx], lam[idx], res[idx]
    err = rel_l2(xi, ref["xi"])
    dres = np.abs(res - ref["rp_final"])
    assert err.max() <= TOL_XI_REL_MIXED, f"xi rel L2 max {err.max():.3e} median {np.median(err):.3e}"
    lerr = lam_err(lam, ref["lam"], ref["xi"])
    assert lerr.max() <= TOL_LAM_MIXED, f"lambda error max {lerr.max():.3e} median {np.median(lerr):.3e}"
    assert dres.max() <= TOL_RESID_ABS, f"residual diff max {dres.max():.3e}"
    return err, dres


@pytest.mark.parametrize("prec", PRECS)
def test_small_2d_zero_init(sfmod, oracle_lib, prec):
    sc = si.scene(si.config_small_2d(), 0)
    ref = run_oracle(oracle_lib, sc, RHO_2D, 100)
    _check(_run(sfmod, sc, RHO_2D, 100, prec), ref)


@pytest.mark.parametrize("prec", PRECS)
def test_n16_3d_small_batch(sfmod, oracle_lib, prec):
    """24 samples (several CTAs, a ragged time tail), K=60, with the
    residual history checked against the oracle's projection residual."""
    sc = si.scene(si.config_n16_3d(n_samples=24), 1)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 60, hist=True)
    out = _run(sfmod, sc, RHO_3D, 60, prec, hist=True)
    _check(out, ref)
    h = out.hist.double().cpu().numpy().T          # [S][K]
    assert np.abs(h - ref["proj_hist"]).max() <= 5e-3


@pytest.mark.parametrize("prec", PRECS)
def test_n32_t120(sfmod, oracle_lib, prec):
    sc = si.scene(si.config_n32_3d(n_samples=16), 3)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 40)
    _check(_run(sfmod, sc, RHO_3D, 40, prec), ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,T", [(1, 50), (2, 33), (5, 64), (9, 31), (17, 97)])
def test_edge_sizes(sfmod, oracle_lib, prec, N, T):
    spec = si.config_n16_3d(n_robots=N, n_samples=5, T=T, box=(6.0, 6.0, 3.0), min_sep=0.8)
    sc = si.scene(spec, 40 + N)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 30)
    _check(_run(sfmod, sc, RHO_3D, 30, prec), ref)


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_multi_scene_batch(sfmod, oracle_lib, prec):
    """Scenes with different N and S (one empty) in one call; each scene
    against its own oracle run."""
    P = sfmod
    specs = [si.config_n16_3d(n_robots=n, n_samples=s, K=25) for n, s in
             [(8, 7), (13, 3), (16, 0), (24, 5), (32, 2), (3, 9)]]
    st = si.Stream(7)
    scenes = [si.make_scene(sp, st) for sp in specs]
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=32, precision=prec)
    xb = np.concatenate([s.xi_bar.reshape(-1) for s in scenes])
    nr = [s.spec.n_robots for s in scenes]
    ns = [s.spec.n_samples for s in scenes]
    out = f.project(_dev(xb), _dev(np.concatenate([s.start for s in scenes])),
                    _dev(np.concatenate([s.goal for s in scenes])), 25, n_robots=nr, n_samples=ns)
    torch.cuda.synchronize()
    xi = out.xi.double().cpu().numpy()
    lam = out.lam.double().cpu().numpy()
    res = out.residual.double().cpu().numpy()
    c0 = s0 = 0
    for s in scenes:
        n = s.spec.n_samples * 3 * s.spec.n_robots * 11
        if s.spec.n_samples:
            ref = run_oracle(oracle_lib, s, RHO_3D, 25)
            err = rel_l2(xi[c0:c0 + n].reshape(s.xi_bar.shape), ref["xi"])
            assert err.max() <= TOL_XI_REL_MIXED, (s.spec.n_robots, err.max())
            lerr = lam_err(lam[c0:c0 + n].reshape(s.xi_bar.shape), ref["lam"], ref["xi"])
            assert lerr.max() <= TOL_LAM_MIXED, (s.spec.n_robots, lerr.max())
            assert np.abs(res[s0:s0 + s.spec.n_samples] - ref["rp_final"]).max() <= TOL_RESID_ABS
        c0 += n
        s0 += s.spec.n_samples


@pytest.mark.parametrize("prec", PRECS)
def test_n32_full_size_sampled(sfmod, oracle_lib, prec):
    """The precision workload at full size (N=32, S=2048, T=120, K=200, one
    launch); 8 sampled outputs against the oracle one by one."""
    sc = si.scene(si.config_n32_3d(), 3)
    out = _run(sfmod, sc, RHO_3D, 200, prec)
    idx = np.array([0, 1, 250, 777, 1024, 1500, 2046, 2047])
    ref = run_oracle(oracle_lib, sc, RHO_3D, 200, idx=idx)
    _check(out, ref, idx)
    assert torch.isfinite(out.xi).all() and torch.isfinite(out.residual).all()


def test_unsupported_combinations(sfmod):
    """The plain form is float32 only: a 16-bit handle refuses it with
    SF_ERR_UNSUPPORTED. (The 16-bit training forward runs in the
    tensor-memory form; its gradients are tested in test_gpu_tmem.py.)"""
    P = sfmod
    sc = si.scene(si.config_n16_3d(n_samples=2), 1)
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=16, precision="bf16",
                       checkpoint_every=10)
    args = (_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 5)
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        f.project(*args, form="plain")
    out, fp, ck = f.project_train(*args)
    torch.cuda.synchronize()
    f.sync_status()
    assert torch.isfinite(out.xi).all() and torch.isfinite(fp).all()
