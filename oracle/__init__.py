"""FP64 CPU oracle of the Swarm-Gen safety filter (arXiv 2501.19042).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers. Nothing in the product
package imports this module, and this module imports nothing from it.

The arithmetic lives in ``sf_oracle.c`` (plain C, double precision, one
rounding per operation). This file only compiles it with gcc and marshals
numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sf_oracle.c")
_HDR = os.path.join(_HERE, "sf_oracle.h")
_LIB = os.path.join(_HERE, "liboracle_sf.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
          "-D_POSIX_C_SOURCE=200809L"]


def build(force: bool = False) -> str:
    """Compile ``liboracle_sf.so`` next to the source (idempotent)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm", "-lpthread"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OracleProblem(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n_robots", C.c_int), ("order", C.c_int), ("T", C.c_int),
        ("t_final", C.c_double), ("rho", C.c_double), ("coll_a", C.c_double),
        ("coll_b", C.c_double), ("v_max", C.c_double), ("a_max", C.c_double),
        ("use_workspace", C.c_int), ("ws_center", C.c_double * 3), ("ws_a", C.c_double),
        ("ws_b", C.c_double),
    ]


_VEC = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double))


class AmOps(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("ctx", C.c_void_p),
                ("apply_F", _VEC), ("apply_Ft", _VEC), ("project", _VEC), ("solve_xi", _VEC)]


_dp = C.POINTER(C.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            lib.oracle_basis.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp, _dp]
            lib.oracle_basis.restype = C.c_int
            lib.oracle_pair_project.argtypes = [C.c_double, C.c_double, C.c_int, _dp, _dp]
            lib.oracle_ball_project.argtypes = [C.c_double, C.c_int, _dp, _dp]
            lib.oracle_spheroid_in_project.argtypes = [C.c_double, C.c_double, C.c_int, _dp, _dp, _dp]
            lib.oracle_rows_per_axis.argtypes = [C.POINTER(OracleProblem)]
            lib.oracle_rows_per_axis.restype = C.c_int
            lib.oracle_sf_create.argtypes = [C.POINTER(OracleProblem), _dp, _dp, _dp, _dp]
            lib.oracle_sf_create.restype = C.c_void_p
            lib.oracle_sf_destroy.argtypes = [C.c_void_p]
            lib.oracle_sf_ops.argtypes = [C.c_void_p, C.POINTER(AmOps)]
            lib.oracle_sf_dense_F.argtypes = [C.c_void_p, _dp]
            lib.oracle_sf_dense_F.restype = C.c_int
            lib.oracle_sf_dense_A.argtypes = [C.c_void_p, _dp, _dp]
            lib.oracle_sf_kkt_size.argtypes = [C.c_void_p]
            lib.oracle_sf_kkt_size.restype = C.c_int
            lib.oracle_sf_kkt_matrix.argtypes = [C.c_void_p, _dp]
            lib.oracle_eq_project.argtypes = [C.c_void_p, _dp, _dp]
            lib.oracle_eq_project.restype = C.c_int
            lib.oracle_eq_project_adjoint.argtypes = [C.c_void_p, _dp, _dp, _dp]
            lib.oracle_eq_project_adjoint.restype = C.c_int
            lib.oracle_sf_run.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp, _dp]
            lib.oracle_sf_run.restype = C.c_int
            lib.oracle_sf_run_batch.argtypes = [C.POINTER(OracleProblem), _dp, _dp, _dp, _dp, C.c_int,
                                                _dp, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_int]
            lib.oracle_sf_run_batch.restype = C.c_int
            lib.oracle_am_step.argtypes = [C.POINTER(AmOps), C.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Problem:
    """Problem constants (paper Sec. II and Appendix); see ``sf_oracle.h``."""
    dim: int
    n_robots: int
    T: int
    order: int = 10
    t_final: float = 5.0
    rho: float = 1.0
    coll_a: float = 0.5
    coll_b: float = 0.5
    v_max: float = 2.0
    a_max: float = 3.0
    use_workspace: bool = False
    ws_center: tuple = (0.0, 0.0, 0.0)
    ws_a: float = 1.0
    ws_b: float = 1.0

    @property
    def nvar(self) -> int:
        return self.order + 1

    def c(self) -> OracleProblem:
        p = OracleProblem()
        p.dim, p.n_robots, p.order, p.T = self.dim, self.n_robots, self.order, self.T
        p.t_final, p.rho = self.t_final, self.rho
        p.coll_a, p.coll_b, p.v_max, p.a_max = self.coll_a, self.coll_b, self.v_max, self.a_max
        p.use_workspace = int(bool(self.use_workspace))
        for i in range(3):
            p.ws_center[i] = float(self.ws_center[i]) if i < len(self.ws_center) else 0.0
        p.ws_a, p.ws_b = self.ws_a, self.ws_b
        return p


def basis(order: int, T: int, t_final: float):
    """Bernstein P, Pd, Pdd, each [T][order+1] (Eq. poly)."""
    lib = _lib_handle()
    nv = order + 1
    P, Pd, Pdd = (np.zeros((T, nv)) for _ in range(3))
    if lib.oracle_basis(order, T, float(t_final), _ptr(P), _ptr(Pd), _ptr(Pdd)) != 0:
        raise ValueError("bad basis arguments")
    return P, Pd, Pdd


def pair_project(a: float, b: float, delta) -> np.ndarray:
    lib = _lib_handle()
    d = _f64(delta)
    e = np.zeros_like(d)
    lib.oracle_pair_project(float(a), float(b), int(d.size), _ptr(d), _ptr(e))
    return e


def ball_project(r: float, v) -> np.ndarray:
    lib = _lib_handle()
    d = _f64(v)
    e = np.zeros_like(d)
    lib.oracle_ball_project(float(r), int(d.size), _ptr(d), _ptr(e))
    return e


def spheroid_in_project(a: float, b: float, center, p) -> np.ndarray:
    lib = _lib_handle()
    pp = _f64(p)
    cc = _f64(np.asarray(center, dtype=np.float64)[: pp.size])
    e = np.zeros_like(pp)
    lib.oracle_spheroid_in_project(float(a), float(b), int(pp.size), _ptr(cc), _ptr(pp), _ptr(e))
    return e


def rows_per_axis(pb: Problem) -> int:
    p = pb.c()
    return _lib_handle().oracle_rows_per_axis(C.byref(p))


class OracleSF:
    """One scene (starts, goals, optional boundary velocity/acceleration)."""

    def __init__(self, pb: Problem, start, goal, start_va=None, goal_va=None):
        self.pb = pb
        self._lib = _lib_handle()
        self._keep = [_f64(start), _f64(goal), _f64(start_va), _f64(goal_va)]
        cp = pb.c()
        self._h = self._lib.oracle_sf_create(C.byref(cp), *(_ptr(a) for a in self._keep))
        if not self._h:
            raise ValueError("oracle_sf_create failed (bad problem)")
        self.n = pb.dim * pb.n_robots * pb.nvar
        self.m = pb.dim * rows_per_axis(pb)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_sf_destroy(h)
            self._h = None

    def dense_F(self) -> np.ndarray:
        F = np.zeros((self.m, self.n))
        if self._lib.oracle_sf_dense_F(self._h, _ptr(F)) != 0:
            raise ValueError("problem too large for a dense F")
        return F

    def dense_A(self):
        rows = self.pb.dim * self.pb.n_robots * 6
        A = np.zeros((rows, self.n))
        b = np.zeros(rows)
        self._lib.oracle_sf_dense_A(self._h, _ptr(A), _ptr(b))
        return A, b

    def kkt_matrix(self) -> np.ndarray:
        k = self._lib.oracle_sf_kkt_size(self._h)
        K = np.zeros((k, k))
        self._lib.oracle_sf_kkt_matrix(self._h, _ptr(K))
        return K

    def ops(self) -> AmOps:
        o = AmOps()
        self._lib.oracle_sf_ops(self._h, C.byref(o))
        return o

    def apply(self, name: str, x) -> np.ndarray:
        """Calls one of the SF operators (apply_F, apply_Ft, project, solve_xi)."""
        o = self.ops()
        xin = _f64(x)
        out_len = self.m if name in ("apply_F", "project") else self.n
        out = np.zeros(out_len)
        getattr(o, name)(o.ctx, _ptr(xin), _ptr(out))
        return out

    def eq_project(self, xi_in) -> np.ndarray:
        """QP layer of the decoders: argmin ||xi - xi_in||^2 s.t. A xi = b."""
        x = _f64(xi_in).reshape(-1)
        out = np.zeros(self.n)
        if self._lib.oracle_eq_project(self._h, _ptr(x), _ptr(out)) != 0:
            raise RuntimeError("oracle_eq_project failed")
        return out

    def eq_project_adjoint(self, g):
        """(dL/dxi_in, dL/db) of the QP layer for dL/dxi_out = g."""
        gg = _f64(g).reshape(-1)
        gi = np.zeros(self.n)
        gb = np.zeros(self.pb.dim * self.pb.n_robots * 6)
        if self._lib.oracle_eq_project_adjoint(self._h, _ptr(gg), _ptr(gi), _ptr(gb)) != 0:
            raise RuntimeError("oracle_eq_project_adjoint failed")
        return gi, gb

    def run(self, xi_bar, K: int, xi0=None, lam0=None):
        """K iterations for one sample. Returns dict with xi, lam, rp_hist,
        proj_hist and viol (see ``oracle_sf_run``)."""
        xb = _f64(xi_bar).reshape(-1)
        x0 = _f64(xi0)
        l0 = _f64(lam0)
        xi = np.zeros(self.n)
        lam = np.zeros(self.n)
        rp = np.zeros(max(K, 1))
        ph = np.zeros(max(K, 1))
        viol = np.zeros(1)
        rc = self._lib.oracle_sf_run(self._h, _ptr(xb), _ptr(x0), _ptr(l0), int(K), _ptr(xi),
                                     _ptr(lam), _ptr(rp), _ptr(ph), _ptr(viol))
        if rc != 0:
            raise RuntimeError("oracle_sf_run failed")
        return {"xi": xi, "lam": lam, "rp_hist": rp[:K], "proj_hist": ph[:K], "viol": float(viol[0])}


def run_batch(pb: Problem, start, goal, xi_bar, K: int, xi0=None, lam0=None, start_va=None,
              goal_va=None, n_threads: int | None = None, hist: bool = False):
    """K iterations for S samples of one scene on host threads.

    xi_bar: [S][dim][N][nvar]. Returns dict with xi, lam ([S][dim][N][nvar]),
    rp_final [S] and, if hist, rp_hist / proj_hist [S][K]."""
    lib = _lib_handle()
    xb = _f64(xi_bar)
    S = xb.shape[0]
    n = pb.dim * pb.n_robots * pb.nvar
    xb = xb.reshape(S, n)
    xi = np.zeros((S, n))
    lam = np.zeros((S, n))
    rpf = np.zeros(S)
    rph = np.zeros((S, K)) if hist else None
    pph = np.zeros((S, K)) if hist else None
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    cp = pb.c()
    st, gl, sva, gva = _f64(start), _f64(goal), _f64(start_va), _f64(goal_va)
    x0 = None if xi0 is None else _f64(xi0).reshape(S, n)
    l0 = None if lam0 is None else _f64(lam0).reshape(S, n)
    rc = lib.oracle_sf_run_batch(C.byref(cp), _ptr(st), _ptr(gl), _ptr(sva), _ptr(gva), int(S),
                                 _ptr(xb), _ptr(x0), _ptr(l0), int(K), _ptr(xi), _ptr(lam),
                                 _ptr(rpf), _ptr(rph), _ptr(pph), int(n_threads))
    if rc != 0:
        raise RuntimeError("oracle_sf_run_batch failed")
    shape = (S, pb.dim, pb.n_robots, pb.nvar)
    out = {"xi": xi.reshape(shape), "lam": lam.reshape(shape), "rp_final": rpf}
    if hist:
        out["rp_hist"], out["proj_hist"] = rph, pph
    return out


@dataclass
class ScalarInstance:
    """A flat problem given by Python callables, run through the oracle's
    generic AM core (``oracle_am_step``). Used by tests to drive the core on
    small hand-made instances."""
    n: int
    m: int
    F: callable
    Ft: callable
    project: callable
    solve: callable
    _cbs: list = field(default_factory=list)

    def step(self, rho: float, xi_bar, xi, lam):
        lib = _lib_handle()

        def wrap(fn, nin, nout):
            def cb(_ctx, xin, xout):
                a = np.ctypeslib.as_array(xin, shape=(nin,)).copy()
                r = np.asarray(fn(a), dtype=np.float64).reshape(nout)
                for i in range(nout):
                    xout[i] = float(r[i])
            return _VEC(cb)

        o = AmOps()
        o.n, o.m, o.ctx = self.n, self.m, None
        cbs = [wrap(self.F, self.n, self.m), wrap(self.Ft, self.m, self.n),
               wrap(self.project, self.m, self.m), wrap(self.solve, self.n, self.n)]
        o.apply_F, o.apply_Ft, o.project, o.solve_xi = cbs
        self._cbs = cbs
        xb = _f64(xi_bar).reshape(self.n).copy()
        x = _f64(xi).reshape(self.n).copy()
        lm = _f64(lam).reshape(self.n).copy()
        work = np.zeros(2 * self.m + self.n)
        e = np.zeros(self.m)
        r2 = np.zeros(1)
        lib.oracle_am_step(C.byref(o), float(rho), _ptr(xb), _ptr(x), _ptr(lm), _ptr(e), _ptr(work),
                           _ptr(r2))
        return x, lm, e
