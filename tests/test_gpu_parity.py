"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs. Float32 path: per-sample relative L2 of xi^K <= 1e-4,
||lambda^K - lambda_ref|| <= 1e-4 ||xi_ref|| and final ||r_p|| within 1e-3
(absolute) of the oracle's. The single-scene cases run the float32 form
(the tensor-memory form has tests of its own); the multi-scene cases run the
library's default choice of form per robot-count bucket."""
import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_2D, RHO_3D, TOL_LAM, TOL_RESID_ABS, TOL_XI_REL, lam_err, rel_l2, run_oracle

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


def _gpu_run(P, sc, rho, K, form="fused", idx=None, hist=False, max_robots=None):
    spec = sc.spec
    f = P.SafetyFilter(dim=spec.dim, T=spec.T, rho=rho, coll_a=spec.coll, v_max=spec.v_max,
                       a_max=spec.a_max, max_robots=max_robots or spec.n_robots, t_final=spec.t_final)
    f.set_tensor_memory(False)
    xb = sc.xi_bar if idx is None else sc.xi_bar[idx]
    x0 = _dev(np.zeros_like(xb)) if spec.init == "zero" else None
    out = f.project(_dev(xb), _dev(sc.start), _dev(sc.goal), K, xi0=x0, form=form, hist=hist)
    torch.cuda.synchronize()
    f.sync_status()
    return out


def _check(out, ref, tol_xi=TOL_XI_REL, min_pass=1.0, idx=None):
    xi = out.xi.double().cpu().numpy()
    lam = out.lam.double().cpu().numpy()
    res = out.residual.double().cpu().numpy()
    if idx is not None:
        xi, lam, res = xi[idx], lam[idx], res[idx]
    err = rel_l2(xi, ref["xi"])
    dres = np.abs(res - ref["rp_final"])
    frac = np.mean(err <= tol_xi)
    assert frac >= min_pass, f"xi rel L2: max {err.max():.3e}, median {np.median(err):.3e}, pass {frac:.3f}"
    lerr = lam_err(lam, ref["lam"], ref["xi"])
    assert lerr.max() <= TOL_LAM, f"lambda error max {lerr.max():.3e}, median {np.median(lerr):.3e}"
    assert dres.max() <= TOL_RESID_ABS, f"residual diff max {dres.max():.3e}"
    return err, dres


@pytest.mark.parametrize("form", ["fused", "plain"])
def test_small_2d_zero_init(sfmod, oracle_lib, form):
    """2D, N=4 on a circle, S=16, K=100, zero init (every pair is at delta = 0 in
    the first iteration: the tie-break)."""
    sc = si.scene(si.config_small_2d(), 0)
    ref = run_oracle(oracle_lib, sc, RHO_2D, 100, hist=True)
    out = _gpu_run(sfmod, sc, RHO_2D, 100, form=form, hist=True)
    _check(out, ref)
    h = out.hist.double().cpu().numpy().T
    np.testing.assert_allclose(h, ref["proj_hist"], rtol=1e-3, atol=1e-4)


@pytest.mark.parametrize("form", ["fused", "plain"])
def test_n16_3d_small_batch(sfmod, oracle_lib, form):
    """3D, N=16, 24 samples (several CTAs, a T=100 ragged time tail), K=60."""
    sc = si.scene(si.config_n16_3d(n_samples=24), 1)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 60)
    out = _gpu_run(sfmod, sc, RHO_3D, 60, form=form)
    _check(out, ref)


def test_n16_full_size_sampled(sfmod, oracle_lib):
    """The benchmark workload at full size (S=1024, K=200, the launch the bench
    times); 8 sampled outputs against the oracle one by one."""
    sc = si.scene(si.config_n16_3d(), 1)
    out = _gpu_run(sfmod, sc, RHO_3D, 200)
    idx = np.array([0, 1, 137, 300, 511, 700, 901, 1023])
    ref = run_oracle(oracle_lib, sc, RHO_3D, 200, idx=idx)
    _check(out, ref, idx=idx)
    # properties at any size: finite, boundary conditions, residual small
    assert torch.isfinite(out.xi).all() and torch.isfinite(out.residual).all()
    assert float(out.residual.median()) < 1e-3


def test_n32_t120(sfmod, oracle_lib):
    """N=32 (496 pairs), T=120, 16 samples, K=40."""
    sc = si.scene(si.config_n32_3d(n_samples=16), 3)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 40)
    out = _gpu_run(sfmod, sc, RHO_3D, 40)
    _check(out, ref)


def test_n32_t120_full_size_sampled(sfmod, oracle_lib):
    """The precision workload at full size in float32 (N=32, S=2048, T=120,
    K=200, one launch); 12 sampled outputs against the oracle one by one."""
    sc = si.scene(si.config_n32_3d(), 3)
    out = _gpu_run(sfmod, sc, RHO_3D, 200)
    idx = np.array([0, 1, 2, 3, 250, 511, 777, 1024, 1500, 1901, 2046, 2047])
    ref = run_oracle(oracle_lib, sc, RHO_3D, 200, idx=idx)
    _check(out, ref, idx=idx)
    assert torch.isfinite(out.xi).all() and torch.isfinite(out.residual).all()


@pytest.mark.parametrize("N,T", [(1, 50), (2, 33), (5, 64), (9, 31), (17, 97)])
def test_edge_sizes(sfmod, oracle_lib, N, T):
    """Single robot (no pairs), two robots, robot counts off the block size,
    time steps below, at and just off multiples of 32."""
    spec = si.config_n16_3d(n_robots=N, n_samples=5, T=T, box=(6.0, 6.0, 3.0), min_sep=0.8)
    sc = si.scene(spec, 40 + N)
    ref = run_oracle(oracle_lib, sc, RHO_3D, 30)
    for form in ("fused", "plain"):
        out = _gpu_run(sfmod, sc, RHO_3D, 30, form=form)
        _check(out, ref)


def test_ragged_multi_scene_batch(sfmod, oracle_lib):
    """Several scenes with different N and S (one of them empty) in one call."""
    P = sfmod
    O = oracle_lib
    specs = [si.config_n16_3d(n_robots=n, n_samples=s, K=25) for n, s in
             [(8, 7), (13, 3), (16, 0), (24, 5), (32, 2), (3, 9)]]
    st = si.Stream(7)
    scenes = [si.make_scene(sp, st) for sp in specs]
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=32)
    xb = np.concatenate([s.xi_bar.reshape(-1) for s in scenes])
    starts = np.concatenate([s.start for s in scenes])
    goals = np.concatenate([s.goal for s in scenes])
    nr = [s.spec.n_robots for s in scenes]
    ns = [s.spec.n_samples for s in scenes]
    for form in ("fused", "plain"):
        out = f.project(_dev(xb), _dev(starts), _dev(goals), 25, n_robots=nr, n_samples=ns, form=form)
        torch.cuda.synchronize()
        xi = out.xi.double().cpu().numpy()
        lam = out.lam.double().cpu().numpy()
        res = out.residual.double().cpu().numpy()
        c0 = s0 = 0
        for sc in scenes:
            S, N = sc.spec.n_samples, sc.spec.n_robots
            n = S * 3 * N * 11
            if S:
                ref = run_oracle(O, sc, RHO_3D, 25)
                err = rel_l2(xi[c0:c0 + n].reshape(S, -1), ref["xi"])
                assert err.max() <= TOL_XI_REL, (N, err)
                assert lam_err(lam[c0:c0 + n].reshape(S, -1), ref["lam"], ref["xi"]).max() <= TOL_LAM, N
                assert np.abs(res[s0:s0 + S] - ref["rp_final"]).max() <= TOL_RESID_ABS
            c0 += n
            s0 += S


def test_deterministic_and_host_path(sfmod):
    """Two runs are bit-identical; sf_project_host (host buffers, copies inside
    the call) gives the same bits as sf_project."""
    P = sfmod
    sc = si.scene(si.config_n16_3d(n_samples=40), 9)
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=16)
    a = f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 20)
    b = f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 20)
    torch.cuda.synchronize()
    assert torch.equal(a.xi, b.xi) and torch.equal(a.lam, b.lam) and torch.equal(a.residual, b.residual)
    h = f.project_host(torch.tensor(sc.xi_bar, dtype=torch.float32).contiguous(),
                       torch.tensor(sc.start, dtype=torch.float32), torch.tensor(sc.goal, dtype=torch.float32), 20)
    assert torch.equal(h.xi, a.xi.cpu()) and torch.equal(h.residual, a.residual.cpu())


def test_invalid_arguments(sfmod):
    P = sfmod
    from paper_2501_19042_gb300._native import SfError
    with pytest.raises(SfError):
        P.SafetyFilter(dim=4)
    with pytest.raises(SfError):
        P.SafetyFilter(order=7)
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=8)
    sc = si.scene(si.config_n16_3d(n_samples=2), 1)
    with pytest.raises(SfError):       # N=16 > max_robots
        f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 5)
    sc8 = si.scene(si.config_n16_3d(n_robots=8, n_samples=2), 1)
    with pytest.raises(SfError):       # K = 0
        f.project(_dev(sc8.xi_bar), _dev(sc8.start), _dev(sc8.goal), 0)
    with pytest.raises(ValueError):    # size mismatch caught in marshalling
        f.project(_dev(sc8.xi_bar), _dev(sc8.start[:4]), _dev(sc8.goal), 5)
    n0 = f.launch_count()
    f.project(_dev(sc8.xi_bar), _dev(sc8.start), _dev(sc8.goal), 5)
    assert f.launch_count() == n0 + 1


def _ragged_inputs(scenes):
    xb = np.concatenate([s.xi_bar.reshape(-1) for s in scenes])
    starts = np.concatenate([s.start for s in scenes])
    goals = np.concatenate([s.goal for s in scenes])
    nr = [s.spec.n_robots for s in scenes]
    ns = [s.spec.n_samples for s in scenes]
    return xb, starts, goals, nr, ns


def test_graph_replay_and_in_place_update(sfmod):
    """A captured graph of a multi-bucket batch (concurrent branches) replays
    bit-identically to the direct call, also after the inputs change in place."""
    P = sfmod
    st = si.Stream(31)
    scenes = [si.make_scene(si.config_n16_3d(n_robots=n, n_samples=s, K=30), st)
              for n, s in [(6, 9), (12, 20), (20, 7), (31, 4)]]
    xb, starts, goals, nr, ns = _ragged_inputs(scenes)
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=32)
    dxb, dst, dgl = _dev(xb), _dev(starts), _dev(goals)
    ref = f.project(dxb, dst, dgl, 30, n_robots=nr, n_samples=ns, hist=True)
    g = f.capture(dxb, dst, dgl, 30, n_robots=nr, n_samples=ns, hist=True)
    for _ in range(2):
        out = g.launch()
        torch.cuda.synchronize()
        assert torch.equal(out.xi, ref.xi) and torch.equal(out.lam, ref.lam)
        assert torch.equal(out.residual, ref.residual) and torch.equal(out.hist, ref.hist)
    dxb.mul_(0.9)
    ref2 = f.project(dxb, dst, dgl, 30, n_robots=nr, n_samples=ns, hist=True)
    out = g.launch()
    torch.cuda.synchronize()
    assert torch.equal(out.xi, ref2.xi) and not torch.equal(ref2.xi, ref.xi)
    g.close()


def test_ragged_64_scenes_full_size_sampled(sfmod, oracle_lib):
    """The batching workload at full size: 64 scenes, N ~ U{8..32},
    S ~ U{128..512}, K=150, autotuned and replayed from one captured graph;
    sampled outputs against the oracle one by one."""
    P = sfmod
    scenes = si.ragged_batch(2)
    xb, starts, goals, nr, ns = _ragged_inputs(scenes)
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=32)
    dxb, dst, dgl = _dev(xb), _dev(starts), _dev(goals)
    f.autotune(dxb, dst, dgl, K_probe=5, n_candidates=4, n_robots=nr, n_samples=ns)
    g = f.capture(dxb, dst, dgl, 150, n_robots=nr, n_samples=ns)
    out = g.launch()
    torch.cuda.synchronize()
    f.sync_status()
    xi = out.xi.double().cpu().numpy()
    lam = out.lam.double().cpu().numpy()
    res = out.residual.double().cpu().numpy()
    assert np.isfinite(xi).all() and np.isfinite(res).all()
    offs_c = np.cumsum([0] + [s * 3 * n * 11 for n, s in zip(nr, ns)])
    offs_s = np.cumsum([0] + ns)
    picks = [(0, 0), (17, 5), (40, 100), (63, None)]
    for q, smp in picks:
        sc = scenes[q]
        S, N = sc.spec.n_samples, sc.spec.n_robots
        smp = S - 1 if smp is None else min(smp, S - 1)
        ref = run_oracle(oracle_lib, sc, RHO_3D, 150, idx=np.array([smp]))
        got = xi[offs_c[q]:offs_c[q + 1]].reshape(S, -1)[smp:smp + 1]
        assert rel_l2(got, ref["xi"]).max() <= TOL_XI_REL, (q, N)
        got_l = lam[offs_c[q]:offs_c[q + 1]].reshape(S, -1)[smp:smp + 1]
        assert lam_err(got_l, ref["lam"], ref["xi"]).max() <= TOL_LAM, (q, N)
        assert abs(res[offs_s[q] + smp] - ref["rp_final"][0]) <= TOL_RESID_ABS
    g.close()


@pytest.mark.parametrize("form,prec", [("fused", "fp32"), ("plain", "fp32"), ("fused", "bf16")])
def test_nonfinite_input_is_reported_and_contained(sfmod, form, prec):
    """A NaN in one sample's coefficients: sf_sync_status reports
    SF_ERR_NONFINITE (and clears the word), every other sample's output is
    bit-identical to a run without the bad sample's NaN, and the next clean
    call reports no error."""
    P = sfmod
    sc = si.scene(si.config_n16_3d(n_samples=20), 1)
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=sc.spec.coll, max_robots=16, precision=prec)
    clean = f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 15, form=form)
    f.sync_status()
    bad = sc.xi_bar.copy()
    bad[7, 1, 3, 5] = np.nan
    out = f.project(_dev(bad), _dev(sc.start), _dev(sc.goal), 15, form=form)
    with pytest.raises(RuntimeError, match="NONFINITE"):
        f.sync_status()
    keep = [s for s in range(20) if s != 7]
    assert torch.equal(out.xi[keep], clean.xi[keep]) and torch.equal(out.residual[keep], clean.residual[keep])
    assert not torch.isfinite(out.residual[7])
    f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), 15, form=form)
    f.sync_status()


@pytest.mark.parametrize("N,S,K,T,seed", [(16, 64, 200, 100, 1), (27, 8, 60, 64, 3), (5, 12, 80, 40, 9),
                                          (9, 20, 150, 97, 4)])
def test_pair_pruning_is_exact(sfmod, N, S, K, T, seed):
    """Testing only the candidate pair rows between full tests gives the same
    xi, lambda and final residual as testing every pair every iteration (the
    drift bound excludes every other row), and the same per-iteration history
    up to the order of its sum."""
    P = sfmod
    sc = si.scene(si.config_n16_3d(n_robots=N, n_samples=S, T=T), seed)
    outs = []
    for prune in (True, False):
        f = P.SafetyFilter(dim=3, T=T, rho=RHO_3D, coll_a=sc.spec.coll, max_robots=N)
        f.set_pair_pruning(prune)
        outs.append(f.project(_dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal), K, hist=True))
        torch.cuda.synchronize()
    a, b = outs
    assert torch.equal(a.xi, b.xi) and torch.equal(a.lam, b.lam)
    assert torch.equal(a.residual, b.residual)
    # the history sums squared residuals; above 16 robots the full test sums
    # them in block order, the candidate path in row order
    torch.testing.assert_close(a.hist, b.hist, rtol=1e-5, atol=1e-7)


def test_pair_pruning_training_forward_and_gradients(sfmod):
    """The training forward (checkpoints and activity masks) and the adjoint
    give identical results with and without pair pruning."""
    from paper_2501_19042_gb300.autograd import sf_unroll
    P = sfmod
    sc = si.scene(si.config_diff(n_samples=24), 5)
    g = torch.randn(sc.xi_bar.shape, generator=torch.Generator().manual_seed(1)).cuda()
    res = []
    for prune in (True, False):
        f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=sc.spec.coll, max_robots=16, checkpoint_every=10)
        f.set_pair_pruning(prune)
        xb = _dev(sc.xi_bar).requires_grad_(True)
        xi, lam, fp, r = sf_unroll(f, xb, _dev(sc.start), _dev(sc.goal), 50)
        ((g * xi).sum() + fp.sum()).backward()
        res.append((xi.detach(), fp.detach(), xb.grad.detach()))
    for u, v in zip(*res):
        assert torch.equal(u, v)
