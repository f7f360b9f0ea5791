"""The debug build of the library (``build(debug=True)``, compiled with
-DSF_DEBUG_CHECKS=1): shared-memory canary words after the head and at the
end of every sample block, checked after every phase, and index checks at
the computed-index accesses of the fused kernels (pair decode, chunk-buffer
rows, TMEM columns, MMA tables). No check traps: a failure is reported by
sf_sync_status as SF_ERR_DEBUG_CHECK. The child process
(tests/debug_checks_child.py) runs tiny cases (N = 2, 3; T = 8, 37) against
the FP64 oracle element by element, the bench shape, N = 32, a training
forward and the adjoint, in every form; all must pass their checks and the
tiny cases must match the oracle. A canary word planted on purpose (an
in-bounds write of a wrong value, SF_OPT_TEST_CANARY) must be reported, and
the next call without it must be clean."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DS_CANARY_BLOCK = 8


@pytest.fixture(scope="module")
def child_result():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_19042_gb300.build import build
    build(debug=True)
    env = dict(os.environ, SF_GB300_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_checks_child.py")], capture_output=True,
                       text=True, timeout=1200, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_no_check_fires_and_tiny_cases_match_the_oracle(child_result):
    for key, v in child_result.items():
        if key.startswith("planted/"):
            continue
        assert v["status"] == 0, (key, v["msg"])
        if "xi_err" in v:
            tol = 1e-4 if "/fp32/" in key else 5e-3
            assert v["xi_err"] <= tol, (key, v)
            assert v["lam_err"] <= tol, (key, v)
            assert v["resid_diff"] <= 1e-3, (key, v)


def test_planted_canary_is_reported(child_result):
    planted = {k: v for k, v in child_result.items() if k.startswith("planted/")}
    assert len(planted) == 4
    for key, v in planted.items():
        assert v["status"] == 8, (key, v)   # SF_ERR_DEBUG_CHECK
        assert f"site {DS_CANARY_BLOCK}" in v["msg"], (key, v)
        assert v["after"] == 0, (key, v)


def test_release_library_rejects_the_canary_option():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_19042_gb300 as P
    P.build()
    f = P.SafetyFilter(dim=3, T=100, max_robots=16)
    assert f._lib.sf_set_option(f._h, 4, 1) == 6   # SF_ERR_UNSUPPORTED
