"""Python front end of the GB300 safety filter (argument marshalling only).

Every step of the solver runs in the CUDA library behind ``include/sf.h``;
this module allocates device tensors with PyTorch, passes raw pointers and
the caller's CUDA stream, and turns status codes into exceptions.

Shapes (float32, contiguous):
  single scene:  xi_bar [S, dim, N, nvar], start / goal [N, dim]
  many scenes:   xi_bar flat [sum_s S_s * dim * N_s * nvar], start / goal
                 [sum_s N_s, dim], with ``n_robots`` / ``n_samples`` lists.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _native as nat

NVAR = 11


@dataclass
class ProjectResult:
    xi: torch.Tensor
    lam: torch.Tensor
    residual: torch.Tensor
    hist: torch.Tensor | None = None


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())



def plan_launch(dim: int, T: int, n_robots, n_samples, precision: str = "fp32", num_sms: int = 152,
                smem_per_block_optin: int = 232448) -> dict:
    """``sf_plan_launch``: the fused launch shape the cost model picks for one
    launch group (scenes in one robot-count bucket), without a device."""
    lib = nat.load()
    n = len(n_robots)
    if n != len(n_samples):
        raise ValueError("n_robots and n_samples differ in length")
    nr = (C.c_int * max(n, 1))(*[int(x) for x in n_robots])
    ns = (C.c_int * max(n, 1))(*[int(x) for x in n_samples])
    out = (C.c_int * 4)()
    smem = C.c_size_t(0)
    code = lib.sf_plan_launch(int(dim), int(T), n, nr, ns, nat.PREC[precision], int(num_sms),
                              C.c_size_t(smem_per_block_optin), out, C.byref(smem))
    if code != nat.SF_OK:
        raise nat.SfError(code, "sf_plan_launch failed")
    return {"G": out[0], "warps": out[1], "tc": out[2], "nq": out[3], "smem": int(smem.value)}

def lane_peaks(device: int = 0) -> dict:
    """``sf_lane_peaks``: measured float32 FMA and rsqrt throughput of the
    GPU (per second) and the lane clock that the FMA rate implies."""
    lib = nat.load()
    f, m, c = C.c_double(), C.c_double(), C.c_double()
    code = lib.sf_lane_peaks(int(device), C.byref(f), C.byref(m), C.byref(c))
    if code != nat.SF_OK:
        raise nat.SfError(code, "sf_lane_peaks failed")
    return {"fma_per_s": f.value, "mufu_per_s": m.value, "lane_mhz": c.value}


class SafetyFilter:
    """Handle over ``sf_create`` / ``sf_project`` / ``sf_destroy``."""

    def __init__(self, dim: int = 3, T: int = 100, rho: float = 0.1, coll_a: float = 0.5,
                 coll_b: float | None = None, v_max: float = 2.0, a_max: float = 3.0,
                 max_robots: int = 32, order: int = 10, t_final: float = 5.0,
                 precision: str = "fp32", checkpoint_every: int = 0, device=None,
                 workspace=None):
        """workspace: None, or (centre, a_w, b_w) of the spheroid every
        position must stay in (Eq. workspace_con)."""
        self._lib = nat.load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", device if isinstance(device, int) else torch.device(device).index or 0)
        pb = nat.SfProblem()
        pb.dim, pb.order, pb.T, pb.t_final, pb.rho = dim, order, T, t_final, rho
        pb.coll_a = coll_a
        pb.coll_b = coll_a if coll_b is None else coll_b
        pb.v_max, pb.a_max = v_max, a_max
        pb.use_workspace = 0
        if workspace is not None:
            centre, wa, wb = workspace
            pb.use_workspace = 1
            for i in range(3):
                pb.ws_center[i] = float(centre[i]) if i < len(centre) else 0.0
            pb.ws_a, pb.ws_b = float(wa), float(wb)
        pb.max_robots = max_robots
        pb.precision = nat.PREC[precision]
        pb.checkpoint_every = checkpoint_every
        self.pb = pb
        self.dim, self.T, self.order = dim, T, order
        self.nvar = order + 1
        h = C.c_void_p()
        code = self._lib.sf_create(C.byref(pb), self.device.index, C.byref(h))
        if code != nat.SF_OK:
            raise nat.SfError(code, "sf_create failed")
        self._h = h
        self._ws = None

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.sf_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- batch marshalling ---------------------------------------------------------
    def _batch(self, xi_bar, start, goal, n_robots, n_samples, start_va, goal_va):
        if n_robots is None:
            S, dim, N, nv = xi_bar.shape
            if dim != self.dim or nv != self.nvar:
                raise ValueError(f"xi_bar must be [S, {self.dim}, N, {self.nvar}]")
            n_robots, n_samples = [N], [S]
        nr = (C.c_int * len(n_robots))(*[int(v) for v in n_robots])
        ns = (C.c_int * len(n_samples))(*[int(v) for v in n_samples])
        for name, t in (("xi_bar", xi_bar), ("start", start), ("goal", goal), ("start_va", start_va),
                        ("goal_va", goal_va)):
            if t is not None:
                if t.dtype != torch.float32 or not t.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous float32 tensor")
                if t.device != self.device:
                    raise ValueError(f"{name} must live on {self.device}")
        tot_r = sum(int(v) for v in n_robots)
        tot_c = sum(int(s) * self.dim * int(n) * self.nvar for n, s in zip(n_robots, n_samples))
        if start.numel() != tot_r * self.dim or goal.numel() != tot_r * self.dim:
            raise ValueError("start / goal size does not match n_robots")
        if xi_bar.numel() != tot_c:
            raise ValueError("xi_bar size does not match n_robots / n_samples")
        b = nat.SfBatch()
        b.n_scenes = len(n_robots)
        b.n_robots, b.n_samples = nr, ns
        b.start, b.goal = start.data_ptr(), goal.data_ptr()
        b.start_va = start_va.data_ptr() if start_va is not None else None
        b.goal_va = goal_va.data_ptr() if goal_va is not None else None
        b.xi_bar = xi_bar.data_ptr()
        keep = (nr, ns)
        return b, keep, tot_c, sum(int(s) for s in n_samples)

    def workspace_bytes(self, xi_bar, start, goal, K, form="fused", n_robots=None, n_samples=None):
        b, _keep, _, _ = self._batch(xi_bar, start, goal, n_robots, n_samples, None, None)
        return int(self._lib.sf_workspace_bytes(self._h, C.byref(b), nat.FORM[form], int(K)))

    def _workspace(self, nbytes):
        if nbytes == 0:
            return None
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self._ws

    def project(self, xi_bar, start, goal, K: int, n_robots=None, n_samples=None, xi0=None, lam0=None,
                start_va=None, goal_va=None, form: str = "fused", hist: bool = False,
                out: ProjectResult | None = None, stream=None) -> ProjectResult:
        """K iterations of the SF on device tensors, asynchronously on ``stream``
        (default: the current PyTorch stream)."""
        b, keep, ncoef, nsamp = self._batch(xi_bar, start, goal, n_robots, n_samples, start_va, goal_va)
        for name, t in (("xi0", xi0), ("lam0", lam0)):
            if t is not None and (t.numel() != ncoef or t.dtype != torch.float32 or not t.is_contiguous()):
                raise ValueError(f"{name} must match xi_bar")
        if out is None:
            out = ProjectResult(
                xi=torch.empty_like(xi_bar), lam=torch.empty_like(xi_bar),
                residual=torch.empty(nsamp, dtype=torch.float32, device=self.device),
                hist=torch.empty((K, nsamp), dtype=torch.float32, device=self.device) if hist else None)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        wsb = int(self._lib.sf_workspace_bytes(self._h, C.byref(b), nat.FORM[form], int(K)))
        ws = self._workspace(wsb)
        code = self._lib.sf_project(self._h, C.c_void_p(stream.cuda_stream), C.byref(b), int(K),
                                    nat.FORM[form], _ptr(xi0), _ptr(lam0), _ptr(out.xi), _ptr(out.lam),
                                    _ptr(out.residual), _ptr(out.hist), _ptr(ws), C.c_size_t(wsb), None)
        del keep
        nat.check(self._lib, self._h, code)
        return out

    def project_host(self, xi_bar, start, goal, K: int, n_robots=None, n_samples=None, xi0=None,
                     lam0=None, start_va=None, goal_va=None, form: str = "fused", out=None, stream=None):
        """``sf_project_host``: host (preferably pinned) float32 tensors in and out;
        the host-to-device and device-to-host copies happen inside the call, which
        returns after synchronising the stream."""
        if n_robots is None:
            S, _, N, _ = xi_bar.shape
            n_robots, n_samples = [N], [S]
        nr = (C.c_int * len(n_robots))(*[int(v) for v in n_robots])
        ns = (C.c_int * len(n_samples))(*[int(v) for v in n_samples])
        for t in (xi_bar, start, goal, start_va, goal_va, xi0, lam0):
            if t is not None and (t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous()):
                raise ValueError("host tensors must be contiguous float32 on the CPU")
        b = nat.SfBatch()
        b.n_scenes = len(n_robots)
        b.n_robots, b.n_samples = nr, ns
        b.start, b.goal = start.data_ptr(), goal.data_ptr()
        b.start_va = start_va.data_ptr() if start_va is not None else None
        b.goal_va = goal_va.data_ptr() if goal_va is not None else None
        b.xi_bar = xi_bar.data_ptr()
        nsamp = sum(int(v) for v in n_samples)
        if out is None:
            pin = torch.cuda.is_available()
            out = ProjectResult(xi=torch.empty(xi_bar.shape, pin_memory=pin),
                                lam=torch.empty(xi_bar.shape, pin_memory=pin),
                                residual=torch.empty(nsamp, pin_memory=pin))
        nb = int(self._lib.sf_host_staging_bytes(self._h, C.byref(b), nat.FORM[form], int(K)))
        if nb == 0:
            nat.check(self._lib, self._h, 1)
        stg = self._workspace(nb)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        code = self._lib.sf_project_host(self._h, C.c_void_p(stream.cuda_stream), C.byref(b), int(K),
                                         nat.FORM[form], _ptr(xi0), _ptr(lam0), _ptr(out.xi),
                                         _ptr(out.lam), _ptr(out.residual), _ptr(stg), C.c_size_t(nb))
        nat.check(self._lib, self._h, code)
        return out

    def set_launch_shape(self, samples_per_cta: int = 0, warps: int = 0, time_chunk: int = 0):
        nat.check(self._lib, self._h, self._lib.sf_set_launch_shape(self._h, samples_per_cta, warps, time_chunk))

    def set_pair_pruning(self, on: bool):
        """``sf_set_option(SF_OPT_PAIR_PRUNING)``: exact pruning of far pair
        rows between full tests (default on)."""
        nat.check(self._lib, self._h, self._lib.sf_set_option(self._h, 1, int(bool(on))))

    def set_tensor_memory(self, on):
        """``sf_set_option(SF_OPT_TENSOR_MEMORY)``: True puts the forward's
        coefficient-to-state products on tcgen05 tensor cores through tensor
        memory (tf32 operands in float32, the handle's 16-bit type otherwise),
        False keeps them on the float32 lanes, "auto" (the default) takes the
        form measured faster per robot-count bucket."""
        value = 2 if on == "auto" else int(bool(on))
        nat.check(self._lib, self._h, self._lib.sf_set_option(self._h, 2, value))

    def set_wait_timeout_test(self, microseconds: int):
        """``sf_set_option(SF_OPT_TEST_WAIT_TIMEOUT)``: for testing the
        timeout path only. Nonzero: the tensor-memory form skips its first
        MMA group and bounds each MMA wait by this many microseconds, so the
        next ``sync_status`` raises SF_ERR_TIMEOUT; 0 restores normal calls."""
        nat.check(self._lib, self._h, self._lib.sf_set_option(self._h, 3, int(microseconds)))

    def launch_shape(self):
        out = (C.c_int * 4)()
        nat.check(self._lib, self._h, self._lib.sf_get_launch_shape(self._h, out))
        form = C.c_int(0)
        nat.check(self._lib, self._h, self._lib.sf_get_launch_form(self._h, C.byref(form)))
        return {"G": out[0], "warps": out[1], "tc": out[2], "nq": out[3], "tensor_memory": bool(form.value)}

    def checkpoint_bytes(self, xi_bar, start, goal, K, n_robots=None, n_samples=None) -> int:
        b, _keep, _, _ = self._batch(xi_bar, start, goal, n_robots, n_samples, None, None)
        return int(self._lib.sf_checkpoint_bytes(self._h, C.byref(b), int(K)))

    def project_train(self, xi_bar, start, goal, K, n_robots=None, n_samples=None, xi0=None, lam0=None,
                      start_va=None, goal_va=None, stream=None):
        """``sf_project_train``: forward that also returns the fixed-point
        residual sum per sample and the checkpoints for the backward."""
        b, keep, ncoef, nsamp = self._batch(xi_bar, start, goal, n_robots, n_samples, start_va, goal_va)
        nck = int(self._lib.sf_checkpoint_bytes(self._h, C.byref(b), int(K)))
        ckpt = torch.empty(nck // 4, dtype=torch.float32, device=self.device)
        out = ProjectResult(xi=torch.empty_like(xi_bar), lam=torch.empty_like(xi_bar),
                            residual=torch.empty(nsamp, dtype=torch.float32, device=self.device))
        fp = torch.empty(nsamp, dtype=torch.float32, device=self.device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        code = self._lib.sf_project_train(self._h, C.c_void_p(stream.cuda_stream), C.byref(b), int(K), _ptr(xi0),
                                          _ptr(lam0), _ptr(out.xi), _ptr(out.lam), _ptr(out.residual), _ptr(fp),
                                          _ptr(ckpt))
        del keep
        nat.check(self._lib, self._h, code)
        return out, fp, ckpt

    def project_backward(self, xi_bar, start, goal, K, ckpt, grad_xi=None, grad_lam=None, grad_fp=None,
                         init_from_xi_bar=True, n_robots=None, n_samples=None, start_va=None, goal_va=None,
                         stream=None):
        """``sf_project_backward``: returns (dL/dxi0, dL/dlambda0, dL/dxi_bar)."""
        b, keep, ncoef, nsamp = self._batch(xi_bar, start, goal, n_robots, n_samples, start_va, goal_va)
        nws = int(self._lib.sf_backward_workspace_bytes(self._h, C.byref(b), int(K)))
        ws = torch.empty(max(nws, 4) // 4, dtype=torch.float32, device=self.device)
        gx0 = torch.empty_like(xi_bar)
        gl0 = torch.empty_like(xi_bar)
        gxb = torch.empty_like(xi_bar)
        for t in (grad_xi, grad_lam, grad_fp):
            if t is not None and (t.dtype != torch.float32 or not t.is_contiguous() or t.device != self.device):
                raise ValueError("gradients must be contiguous float32 on the device")
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        code = self._lib.sf_project_backward(self._h, C.c_void_p(stream.cuda_stream), C.byref(b), int(K),
                                             int(bool(init_from_xi_bar)), _ptr(ckpt), _ptr(grad_xi), _ptr(grad_lam),
                                             _ptr(grad_fp), _ptr(gx0), _ptr(gl0), _ptr(gxb), _ptr(ws),
                                             C.c_size_t(nws))
        del keep
        nat.check(self._lib, self._h, code)
        return gx0, gl0, gxb

    def eq_project(self, xi_prime, start, goal, n_robots=None, n_samples=None, start_va=None, goal_va=None,
                   stream=None, out=None):
        """``sf_eq_project``: the decoders' QP layer, the projection of xi'
        onto the boundary conditions of every robot (layout of xi_bar)."""
        b, keep, ncoef, nsamp = self._batch(xi_prime, start, goal, n_robots, n_samples, start_va, goal_va)
        if out is None:
            out = torch.empty_like(xi_prime)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        code = self._lib.sf_eq_project(self._h, C.c_void_p(stream.cuda_stream), C.byref(b), _ptr(out))
        del keep
        nat.check(self._lib, self._h, code)
        return out

    def eq_project_backward(self, grad_out, start, goal, n_robots=None, n_samples=None, start_va=None,
                            goal_va=None, want_grad_b=False, stream=None):
        """``sf_eq_project_backward``: (dL/dxi', dL/db per coefficient row or None)."""
        b, keep, ncoef, nsamp = self._batch(grad_out, start, goal, n_robots, n_samples, start_va, goal_va)
        gin = torch.empty_like(grad_out)
        gb = torch.empty((ncoef // self.nvar, 6), dtype=torch.float32, device=self.device) if want_grad_b else None
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        code = self._lib.sf_eq_project_backward(self._h, C.c_void_p(stream.cuda_stream), C.byref(b),
                                                _ptr(grad_out), _ptr(gin), _ptr(gb))
        del keep
        nat.check(self._lib, self._h, code)
        return gin, gb

    def autotune(self, xi_bar, start, goal, K_probe=10, n_candidates=8, n_robots=None, n_samples=None,
                 start_va=None, goal_va=None, stream=None):
        """``sf_autotune``: times the cost model's best launch shapes for this
        scene mix and keeps the fastest for later calls."""
        b, keep, ncoef, nsamp = self._batch(xi_bar, start, goal, n_robots, n_samples, start_va, goal_va)
        scratch = ProjectResult(xi=torch.empty_like(xi_bar), lam=torch.empty_like(xi_bar),
                                residual=torch.empty(nsamp, dtype=torch.float32, device=self.device))
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        code = self._lib.sf_autotune(self._h, C.c_void_p(stream.cuda_stream), C.byref(b), int(K_probe),
                                     int(n_candidates), _ptr(scratch.xi), _ptr(scratch.lam), _ptr(scratch.residual))
        del keep
        nat.check(self._lib, self._h, code)

    def capture(self, xi_bar, start, goal, K, n_robots=None, n_samples=None, xi0=None, lam0=None,
                start_va=None, goal_va=None, form="fused", hist=False):
        """``sf_graph_capture``: a replayable CUDA graph of one ``project`` call
        on fixed buffers. Returns a ``SFGraph`` whose ``out`` holds the outputs."""
        b, keep, ncoef, nsamp = self._batch(xi_bar, start, goal, n_robots, n_samples, start_va, goal_va)
        out = ProjectResult(
            xi=torch.empty_like(xi_bar), lam=torch.empty_like(xi_bar),
            residual=torch.empty(nsamp, dtype=torch.float32, device=self.device),
            hist=torch.empty((K, nsamp), dtype=torch.float32, device=self.device) if hist else None)
        wsb = int(self._lib.sf_workspace_bytes(self._h, C.byref(b), nat.FORM[form], int(K)))
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=self.device) if wsb else None
        g = C.c_void_p()
        code = self._lib.sf_graph_capture(self._h, C.byref(b), int(K), nat.FORM[form], _ptr(xi0), _ptr(lam0),
                                          _ptr(out.xi), _ptr(out.lam), _ptr(out.residual), _ptr(out.hist),
                                          _ptr(ws), C.c_size_t(wsb), C.byref(g))
        del keep
        nat.check(self._lib, self._h, code)
        return SFGraph(self, g, out, (xi_bar, start, goal, xi0, lam0, start_va, goal_va, ws))

    def launch_count(self) -> int:
        return int(self._lib.sf_launch_count(self._h))

    def sync_status(self, stream=None):
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        nat.check(self._lib, self._h, self._lib.sf_sync_status(self._h, C.c_void_p(stream.cuda_stream)))


class SFGraph:
    """A captured sf_project call (``sf_graph_*``). Inputs captured by pointer:
    update them in place and call ``launch()``."""

    def __init__(self, sf: SafetyFilter, g, out: ProjectResult, keep):
        self._sf, self._g, self.out, self._keep = sf, g, out, keep

    def launch(self, stream=None):
        if stream is None:
            stream = torch.cuda.current_stream(self._sf.device)
        nat.check(self._sf._lib, self._sf._h,
                  self._sf._lib.sf_graph_launch(self._g, C.c_void_p(stream.cuda_stream)))
        return self.out

    def close(self):
        if getattr(self, "_g", None):
            self._sf._lib.sf_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
