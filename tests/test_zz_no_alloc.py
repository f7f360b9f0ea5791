"""sf_project_plain_noalloc: the plain form on the library's built-in scratch
buffer, for callers that may not allocate device memory when they call in
(for example a plug-in whose host framework owns every device allocation,
or a control loop that cannot afford a call that may synchronise the
device). Called through the C ABI; its output must match the regular
plain-form entry point (caller-provided workspace) on two calls in a row.
This file is collected last so that a failure here cannot hide the others.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import swarm_inputs as si
from sfcase import RHO_3D, TOL_RESID_ABS, TOL_XI_REL, rel_l2

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    P.build()
    from paper_2501_19042_gb300 import _native as nat
    return P, nat


def test_noalloc_matches_plain_form_on_two_calls(setup):
    P, nat = setup
    st = si.Stream(21)
    scenes = [si.make_scene(si.config_n16_3d(n_robots=n, n_samples=s), st) for n, s in [(16, 24), (7, 10)]]
    K = 40
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=16)
    xb = _dev(np.concatenate([s.xi_bar.reshape(-1) for s in scenes]))
    starts = _dev(np.concatenate([s.start for s in scenes]))
    goals = _dev(np.concatenate([s.goal for s in scenes]))
    nr = [s.spec.n_robots for s in scenes]
    ns = [s.spec.n_samples for s in scenes]
    ref = f.project(xb, starts, goals, K, n_robots=nr, n_samples=ns, form="plain", hist=True)
    torch.cuda.synchronize()

    lib = nat.load()
    b, keep, ncoef, nsamp = f._batch(xb, starts, goals, nr, ns, None, None)
    stream = torch.cuda.current_stream()
    for call in range(2):
        xi = torch.full_like(xb, float("nan"))
        lam = torch.full_like(xb, float("nan"))
        res = torch.full((nsamp,), float("nan"), device="cuda")
        hist = torch.full((K, nsamp), float("nan"), device="cuda")
        code = lib.sf_project_plain_noalloc(f._h, C.c_void_p(stream.cuda_stream), C.byref(b), K, None, None,
                                            C.c_void_p(xi.data_ptr()), C.c_void_p(lam.data_ptr()),
                                            C.c_void_p(res.data_ptr()), C.c_void_p(hist.data_ptr()))
        nat.check(lib, f._h, code)
        torch.cuda.synchronize()
        off = 0
        for n, s in zip(nr, ns):
            m = s * 3 * n * 11
            a = xi[off:off + m].double().cpu().numpy().reshape(s, -1)
            r = ref.xi[off:off + m].double().cpu().numpy().reshape(s, -1)
            assert rel_l2(a, r).max() <= TOL_XI_REL, f"call {call}"
            la = lam[off:off + m].double().cpu().numpy().reshape(s, -1)
            lr = ref.lam[off:off + m].double().cpu().numpy().reshape(s, -1)
            assert np.abs(la - lr).max() <= 1e-4 * max(1.0, np.abs(lr).max()), f"call {call}"
            off += m
        assert (res - ref.residual).abs().max().item() <= TOL_RESID_ABS, f"call {call}"
        assert torch.allclose(hist, ref.hist, rtol=1e-4, atol=1e-5), f"call {call}"
    del keep


def test_noalloc_rejects_batches_beyond_the_buffer(setup):
    P, nat = setup
    sc = si.scene(si.config_n16_3d(n_samples=400), 3)      # about 48 MB of scratch > 32 MiB
    f = P.SafetyFilter(dim=3, T=100, rho=RHO_3D, coll_a=0.5, max_robots=16)
    xb, stt, gl = _dev(sc.xi_bar), _dev(sc.start), _dev(sc.goal)
    lib = nat.load()
    b, keep, ncoef, nsamp = f._batch(xb, stt, gl, None, None, None, None)
    out = torch.zeros_like(xb)
    res = torch.zeros(nsamp, device="cuda")
    code = lib.sf_project_plain_noalloc(f._h, None, C.byref(b), 10, None, None, C.c_void_p(out.data_ptr()),
                                        C.c_void_p(out.data_ptr()), C.c_void_p(res.data_ptr()), None)
    assert code == 1
    assert b"built-in buffer" in lib.sf_last_error(f._h)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
    del keep
