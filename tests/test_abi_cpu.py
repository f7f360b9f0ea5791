"""CPU-side checks of the C ABI: the library builds, loads without a GPU,
exports every function include/sf.h declares, and rejects bad problems
before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2501_19042_gb300 as P
    from paper_2501_19042_gb300 import _native
    P.build()
    return _native.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "sf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sf_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_function(lib):
    from paper_2501_19042_gb300 import _native
    declared = _declared()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(_native.EXPORTS) == declared


def test_create_validates_before_device(lib):
    from paper_2501_19042_gb300 import _native as nat
    pb = nat.SfProblem()
    pb.dim, pb.order, pb.T, pb.t_final, pb.rho = 3, 10, 100, 5.0, 0.1
    pb.coll_a = pb.coll_b = 0.5
    pb.v_max, pb.a_max, pb.max_robots = 2.0, 3.0, 16
    h = C.c_void_p()
    bad = nat.SfProblem.from_buffer_copy(pb)
    bad.dim = 4
    assert lib.sf_create(C.byref(bad), 0, C.byref(h)) == 1 and not h.value
    bad = nat.SfProblem.from_buffer_copy(pb)
    bad.rho = -1.0
    assert lib.sf_create(C.byref(bad), 0, C.byref(h)) == 1
    bad = nat.SfProblem.from_buffer_copy(pb)
    bad.max_robots = 33
    assert lib.sf_create(C.byref(bad), 0, C.byref(h)) == 1
    bad = nat.SfProblem.from_buffer_copy(pb)
    bad.order = 9
    assert lib.sf_create(C.byref(bad), 0, C.byref(h)) == 6
    assert lib.sf_create(C.byref(pb), 0, None) == 1
    # NULL handle arguments are rejected, not dereferenced
    assert lib.sf_project(None, None, None, 1, 0, None, None, None, None, None, None, None, 0, None) == 1
    assert lib.sf_workspace_bytes(None, None, 0, 1) == 0
    assert lib.sf_launch_count(None) == 0
    assert lib.sf_set_option(None, 1, 1) == 1
    assert lib.sf_eq_project(None, None, None, None) == 1
    assert lib.sf_eq_project_backward(None, None, None, None, None, None) == 1
    # workspace block: semi-axes must be positive and the centre finite
    bad = nat.SfProblem.from_buffer_copy(pb)
    bad.use_workspace, bad.ws_a, bad.ws_b = 1, 0.0, 1.0
    assert lib.sf_create(C.byref(bad), 0, C.byref(h)) == 1
    bad = nat.SfProblem.from_buffer_copy(pb)
    bad.use_workspace, bad.ws_a, bad.ws_b = 1, 2.0, 1.0
    bad.ws_center[1] = float("nan")
    assert lib.sf_create(C.byref(bad), 0, C.byref(h)) == 1
    bad = nat.SfProblem.from_buffer_copy(pb)
    bad.use_workspace = 2
    assert lib.sf_create(C.byref(bad), 0, C.byref(h)) == 1
    lib.sf_destroy(None)


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle and has no CPU implementation."""
    pkg = os.path.join(ROOT, "paper_2501_19042_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                s = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in s and "from oracle" not in s, f
