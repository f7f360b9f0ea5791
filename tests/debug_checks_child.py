"""Runs in a child process with SF_GB300_DEBUG=1, so that the library loaded
is the debug build (shared-memory canaries and index checks compiled into
the fused kernels). Prints one JSON object: per case the outcome of
sf_sync_status and, for the tiny cases, the largest deviation from the FP64
oracle. Called by tests/test_gpu_debug_checks.py."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import swarm_inputs as si  # noqa: E402
from sfcase import lam_err, rel_l2, run_oracle  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def main():
    assert os.environ.get("SF_GB300_DEBUG") == "1"
    from paper_2501_19042_gb300 import _native as nat
    from paper_2501_19042_gb300._native import SfError
    from paper_2501_19042_gb300.safety_filter import SafetyFilter
    import oracle
    oracle.build()
    assert nat.LIB_PATH.endswith("libsf_gb300_debug.so")
    res = {}

    def status(f):
        try:
            f.sync_status()
            return 0, ""
        except SfError as e:
            return e.code, str(e)

    def make(spec, rho, prec, tm, ck=0):
        f = SafetyFilter(dim=spec.dim, T=spec.T, rho=rho, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                         max_robots=spec.n_robots, t_final=spec.t_final, precision=prec, checkpoint_every=ck)
        f.set_tensor_memory(tm)
        return f

    forms = [("fp32", False), ("fp32", True), ("bf16", True), ("fp16", True)]
    # tiny cases compared elementwise with the oracle
    tiny = [("d2_n2_T8", si.config_small_2d(n_robots=2, T=8, n_samples=8), 0.3, 40),
            ("d3_n3_T8", si.config_n16_3d(n_robots=3, T=8, n_samples=8, box=(2.0, 2.0, 1.0), min_sep=0.5), 0.1, 40),
            ("d3_n3_T37", si.config_n16_3d(n_robots=3, T=37, n_samples=11, box=(2.0, 2.0, 1.0), min_sep=0.5), 0.1,
             60)]
    for name, spec, rho, K in tiny:
        sc = si.scene(spec, 3)
        ref = run_oracle(oracle, sc, rho, K)
        x0 = dev(np.zeros_like(sc.xi_bar)) if spec.init == "zero" else None
        for prec, tm in forms:
            f = make(spec, rho, prec, tm)
            out = f.project(dev(sc.xi_bar), dev(sc.start), dev(sc.goal), K, xi0=x0)
            code, msg = status(f)
            xi = out.xi.double().cpu().numpy()
            res[f"{name}/{prec}/tm{int(tm)}"] = {
                "status": code, "msg": msg,
                "xi_err": float(rel_l2(xi, ref["xi"]).max()),
                "lam_err": float(lam_err(out.lam.double().cpu().numpy(), ref["lam"], ref["xi"]).max()),
                "resid_diff": float(np.abs(out.residual.double().cpu().numpy() - ref["rp_final"]).max())}
    # larger launches: the bench shape (several chunks, pruning), N=32, a
    # training forward and the adjoint
    big = [("n16", si.config_n16_3d(n_samples=64), 0.1, 30),
           ("n32", si.config_n32_3d(n_samples=16), 0.1, 20)]
    for name, spec, rho, K in big:
        sc = si.scene(spec, 5)
        args = (dev(sc.xi_bar), dev(sc.start), dev(sc.goal))
        for prec, tm in forms:
            f = make(spec, rho, prec, tm, ck=10)
            f.project(*args, K, hist=True)
            code, msg = status(f)
            out, fp, ck = f.project_train(*args, K)
            code2, msg2 = status(f)
            g = torch.ones_like(out.xi)
            f.project_backward(*args, K, ck, grad_xi=g)
            code3, msg3 = status(f)
            res[f"{name}/{prec}/tm{int(tm)}"] = {"status": max(code, code2, code3), "msg": msg + msg2 + msg3}
    # the checks fire: a wrong canary word planted by the kernels
    spec = si.config_n16_3d(n_samples=32)
    sc = si.scene(spec, 6)
    args = (dev(sc.xi_bar), dev(sc.start), dev(sc.goal))
    for prec, tm in forms:
        f = make(spec, 0.1, prec, tm)
        f._lib.sf_set_option(f._h, 4, 1)
        f.project(*args, 10)
        code, msg = status(f)
        f._lib.sf_set_option(f._h, 4, 0)
        f.project(*args, 10)
        after, _ = status(f)
        res[f"planted/{prec}/tm{int(tm)}"] = {"status": code, "msg": msg, "after": after}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
