"""ctypes declarations of the C ABI in ``include/sf.h`` (marshalling only).

Loading fails loudly when ``libsf_gb300.so`` has not been built: there is no
fallback implementation of any step.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# SF_GB300_DEBUG=1 loads the debug build (canaries and index checks in the
# fused kernels; ``build(debug=True)`` makes it)
DEBUG = os.environ.get("SF_GB300_DEBUG") == "1"
LIB_PATH = os.path.join(HERE, "libsf_gb300_debug.so" if DEBUG else "libsf_gb300.so")

SF_OK = 0
STATUS_NAMES = {0: "SF_OK", 1: "SF_ERR_INVALID_ARG", 2: "SF_ERR_CUDA", 3: "SF_ERR_OOM",
                4: "SF_ERR_TIMEOUT", 5: "SF_ERR_NONFINITE", 6: "SF_ERR_UNSUPPORTED",
                7: "SF_ERR_WORKSPACE", 8: "SF_ERR_DEBUG_CHECK"}
PREC = {"fp32": 0, "bf16": 1, "fp16": 2}
FORM = {"fused": 0, "plain": 1}

# every function include/sf.h declares
EXPORTS = ("sf_create", "sf_destroy", "sf_last_error", "sf_workspace_bytes", "sf_checkpoint_bytes",
           "sf_project", "sf_host_staging_bytes", "sf_project_host", "sf_launch_count",
           "sf_project_plain_noalloc", "sf_set_launch_shape", "sf_get_launch_shape",
           "sf_project_train", "sf_backward_workspace_bytes", "sf_project_backward",
           "sf_autotune", "sf_graph_capture", "sf_graph_launch", "sf_graph_destroy", "sf_sync_status",
           "sf_eq_project", "sf_eq_project_backward", "sf_set_option", "sf_plan_launch",
           "sf_lane_peaks", "sf_get_launch_form")


class SfProblem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("order", C.c_int), ("T", C.c_int), ("t_final", C.c_double),
        ("rho", C.c_double), ("coll_a", C.c_double), ("coll_b", C.c_double),
        ("v_max", C.c_double), ("a_max", C.c_double), ("use_workspace", C.c_int),
        ("ws_center", C.c_double * 3), ("ws_a", C.c_double), ("ws_b", C.c_double),
        ("max_robots", C.c_int), ("precision", C.c_int), ("checkpoint_every", C.c_int),
    ]


class SfBatch(C.Structure):
    _fields_ = [
        ("n_scenes", C.c_int), ("n_robots", C.POINTER(C.c_int)), ("n_samples", C.POINTER(C.c_int)),
        ("start", C.c_void_p), ("goal", C.c_void_p), ("start_va", C.c_void_p),
        ("goal_va", C.c_void_p), ("xi_bar", C.c_void_p),
    ]


class SfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Loads the CUDA library; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = C.CDLL(path)
        vp, sz = C.c_void_p, C.c_size_t
        lib.sf_create.argtypes = [C.POINTER(SfProblem), C.c_int, C.POINTER(vp)]
        lib.sf_create.restype = C.c_int
        lib.sf_destroy.argtypes = [vp]
        lib.sf_destroy.restype = None
        lib.sf_last_error.argtypes = [vp]
        lib.sf_last_error.restype = C.c_char_p
        lib.sf_workspace_bytes.argtypes = [vp, C.POINTER(SfBatch), C.c_int, C.c_int]
        lib.sf_workspace_bytes.restype = sz
        lib.sf_checkpoint_bytes.argtypes = [vp, C.POINTER(SfBatch), C.c_int]
        lib.sf_checkpoint_bytes.restype = sz
        lib.sf_project.argtypes = [vp, vp, C.POINTER(SfBatch), C.c_int, C.c_int, vp, vp, vp, vp, vp,
                                   vp, vp, sz, vp]
        lib.sf_project.restype = C.c_int
        lib.sf_host_staging_bytes.argtypes = [vp, C.POINTER(SfBatch), C.c_int, C.c_int]
        lib.sf_host_staging_bytes.restype = sz
        lib.sf_project_host.argtypes = [vp, vp, C.POINTER(SfBatch), C.c_int, C.c_int, vp, vp, vp, vp,
                                        vp, vp, sz]
        lib.sf_project_host.restype = C.c_int
        lib.sf_launch_count.argtypes = [vp]
        lib.sf_launch_count.restype = C.c_ulonglong
        lib.sf_project_plain_noalloc.argtypes = [vp, vp, C.POINTER(SfBatch), C.c_int, vp, vp, vp, vp,
                                                 vp, vp]
        lib.sf_project_plain_noalloc.restype = C.c_int
        lib.sf_set_launch_shape.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        lib.sf_set_launch_shape.restype = C.c_int
        lib.sf_get_launch_shape.argtypes = [vp, C.POINTER(C.c_int)]
        lib.sf_get_launch_shape.restype = C.c_int
        lib.sf_get_launch_form.argtypes = [vp, C.POINTER(C.c_int)]
        lib.sf_get_launch_form.restype = C.c_int
        lib.sf_project_train.argtypes = [vp, vp, C.POINTER(SfBatch), C.c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.sf_project_train.restype = C.c_int
        lib.sf_backward_workspace_bytes.argtypes = [vp, C.POINTER(SfBatch), C.c_int]
        lib.sf_backward_workspace_bytes.restype = sz
        lib.sf_project_backward.argtypes = [vp, vp, C.POINTER(SfBatch), C.c_int, C.c_int, vp, vp, vp, vp, vp,
                                            vp, vp, vp, sz]
        lib.sf_project_backward.restype = C.c_int
        lib.sf_set_option.argtypes = [vp, C.c_int, C.c_int]
        lib.sf_set_option.restype = C.c_int
        ip = C.POINTER(C.c_int)
        lib.sf_plan_launch.argtypes = [C.c_int, C.c_int, C.c_int, ip, ip, C.c_int, C.c_int, sz, ip,
                                       C.POINTER(sz)]
        lib.sf_plan_launch.restype = C.c_int
        lib.sf_eq_project.argtypes = [vp, vp, C.POINTER(SfBatch), vp]
        lib.sf_eq_project.restype = C.c_int
        lib.sf_eq_project_backward.argtypes = [vp, vp, C.POINTER(SfBatch), vp, vp, vp]
        lib.sf_eq_project_backward.restype = C.c_int
        lib.sf_autotune.argtypes = [vp, vp, C.POINTER(SfBatch), C.c_int, C.c_int, vp, vp, vp]
        lib.sf_autotune.restype = C.c_int
        lib.sf_graph_capture.argtypes = [vp, C.POINTER(SfBatch), C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp,
                                         sz, C.POINTER(vp)]
        lib.sf_graph_capture.restype = C.c_int
        lib.sf_graph_launch.argtypes = [vp, vp]
        lib.sf_graph_launch.restype = C.c_int
        lib.sf_graph_destroy.argtypes = [vp]
        lib.sf_graph_destroy.restype = None
        lib.sf_sync_status.argtypes = [vp, vp]
        lib.sf_sync_status.restype = C.c_int
        dp = C.POINTER(C.c_double)
        lib.sf_lane_peaks.argtypes = [C.c_int, dp, dp, dp]
        lib.sf_lane_peaks.restype = C.c_int
        _lib = lib
        return lib


def check(lib, handle, code: int):
    if code != SF_OK:
        msg = lib.sf_last_error(handle).decode() if handle else ""
        raise SfError(code, msg)
