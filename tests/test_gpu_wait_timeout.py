"""The tensor-memory form's only device-side wait (for its own MMA group,
tcgen05.commit to an mbarrier) is bounded in time. The test makes that wait
run out without a fault: with SF_OPT_TEST_WAIT_TIMEOUT the first MMA group of
every CTA is never issued, so nothing ever completes the phase the threads
wait on. The call must end, report SF_ERR_TIMEOUT through sf_sync_status,
and leave the context usable: the next normal call on the same handle gives
the same outputs as a fresh handle."""
import time

import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_3D

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


def _filter(P, spec, prec):
    f = P.SafetyFilter(dim=spec.dim, T=spec.T, rho=RHO_3D, coll_a=spec.coll, v_max=spec.v_max,
                       a_max=spec.a_max, max_robots=spec.n_robots, t_final=spec.t_final, precision=prec)
    f.set_tensor_memory(True)
    return f


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mma_wait_runs_out_and_context_survives(sfmod, prec):
    from paper_2501_19042_gb300._native import SfError
    spec = si.config_n16_3d()
    sc = si.scene(spec, 4)
    S = 40
    args = (_dev(sc.xi_bar[:S]), _dev(sc.start), _dev(sc.goal))
    K = 6
    f = _filter(sfmod, spec, prec)
    f.set_wait_timeout_test(2000)   # 2 ms per wait
    t0 = time.perf_counter()
    f.project(*args, K)
    with pytest.raises(SfError) as e:
        f.sync_status()
    took = time.perf_counter() - t0
    assert e.value.code == 4, e.value   # SF_ERR_TIMEOUT
    assert took < 5.0, f"the abandoned wait took {took:.2f} s"
    # the status word was cleared and the context still works
    f.sync_status()
    f.set_wait_timeout_test(0)
    out = f.project(*args, K)
    f.sync_status()
    g = _filter(sfmod, spec, prec)
    ref = g.project(*args, K)
    g.sync_status()
    assert torch.equal(out.xi, ref.xi) and torch.equal(out.lam, ref.lam)
    assert torch.equal(out.residual, ref.residual)
    assert torch.isfinite(out.xi).all()


def test_option_rejects_bad_values(sfmod):
    from paper_2501_19042_gb300._native import SfError
    f = _filter(sfmod, si.config_n16_3d(), "fp32")
    for bad in (-1, 1000001):
        with pytest.raises(SfError) as e:
            f.set_wait_timeout_test(bad)
        assert e.value.code == 1
