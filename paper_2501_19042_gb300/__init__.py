"""GB300-native batched safety filter (SF) of Swarm-Gen, arXiv 2501.19042.

The solver is the CUDA library ``libsf_gb300.so`` (C ABI in ``include/sf.h``);
``SafetyFilter`` is its Python front end. Importing this package does not load
the library; creating a ``SafetyFilter`` does, and fails if it is not built.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("SafetyFilter", "ProjectResult", "plan_launch", "lane_peaks"):
        from . import safety_filter
        return getattr(safety_filter, name)
    raise AttributeError(name)
