#!/usr/bin/env python3
"""Benchmark of the batched safety filter on the N=16 robots 3D workload.

A step is one sf_project call: K=200 iterations of f_FP over S=1024 sampled
trajectories of one scene (16 robots, 3D, T=100, Bernstein order 10, sample
init, rho=0.1), inputs resident in HBM. Metric: SF-projected samples/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--form fused|plain]

Prints one JSON line (rank 0). Under torchrun the global batch holds one
1024-sample scene per rank and is split into contiguous sample ranges
(sharding.shard_batch), one per rank (weak scaling, no collective on the
data path); the timed region is bracketed by a barrier and a synchronize,
and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import swarm_inputs as si  # noqa: E402

RHO = 0.1
METRIC = "SF-projected samples/s (16 robots 3D, residual<=1e-3), chosen vs plain form"
UNIT = "samples/s"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the fused kernel on the bench workload, per (form, tensor memory,
# precision), from ncu captures of the current kernels (summaries under
# profiles/); a kernel changed since its capture has no entry
FWD_TRAFFIC = {
    ("fused", True, "fp32"): (2391040, "ncu --set full of tm_fwd_kernel<3,16,384,tf32> on this workload, "
                                        "one launch (summary under profiles/)"),
}
# warp-instructions executed by one launch of the fused kernel on the bench
# workload (smsp__inst_executed.sum of the same ncu captures), for the
# executed-instruction fraction beside the algorithmic one
FWD_EXECUTED = {
    ("fused", True, "fp32"): 1366195759,
}
DTYPES = {"fp32": "f32", "bf16": "f32 (bf16 tensor products)", "fp16": "f32 (fp16 tensor products)"}


def ops_per_sample_iter(N: int, T: int, dim: int, nv: int = 11, use_v: bool = True, use_a: bool = True):
    """Algorithmic float32 lane operations of one iteration of one sample
    (an FMA counts once; rsqrt counts once)."""
    blocks = 1 + int(use_v) + int(use_a)
    contractions = 2 * blocks * T * nv * dim * N          # states and F^T of the residual
    c_pair = 19 if dim == 3 else 14
    c_ball = 9 if dim == 3 else 7
    pairs = N * (N - 1) // 2 * T * c_pair                   # alpha/beta/d steps + accumulation
    balls = (int(use_v) + int(use_a)) * N * T * c_ball      # velocity / acceleration blocks
    solve = dim * (N * 2 * nv * nv + 2 * nv * nv) + dim * N * nv * 5  # lambda step and xi step
    return contractions + pairs + balls + solve


def state_macs_per_sample_iter(N: int, T: int, dim: int, nv: int = 11):
    """Multiply-adds of the velocity and acceleration states of one iteration
    of one sample (Pd c, Pdd c for every robot, axis and time step): the part
    of the count that the tensor-memory form runs on the tensor cores."""
    return 2 * T * nv * dim * N


def mufu_per_sample_iter(N: int, T: int):
    """Algorithmic special-function operations of one iteration of one
    sample: one reciprocal square root per pair row and per ball row."""
    return N * (N - 1) // 2 * T + 2 * N * T


def roofline(spec, S, K, ms, tm, precision, form, lane, dev):
    """The fused kernel against the pipes that bound it. FP32 lanes:
    algorithmic lane operations (ops_per_sample_iter; in the tensor-memory
    form without the velocity / acceleration states) over the launch time,
    against the FMA rate measured in this run by sf_lane_peaks. Tensor
    cores (tensor-memory form): the states' algorithmic flops against the
    measured dense bf16 peak of MEASURED_PEAKS.json times the nominal ratio
    of the operand type (tf32 1/2, bf16 / fp16 1). MUFU: one rsqrt per pair
    and ball row against the measured rsqrt rate."""
    N, T, dim = spec.n_robots, spec.T, spec.dim
    peaks = measured_peaks()
    sec = ms * 1e-3
    lane_ops = ops_per_sample_iter(N, T, dim)
    macs = state_macs_per_sample_iter(N, T, dim)
    if tm:
        lane_ops -= macs
    achieved = lane_ops * S * K / sec / 1e12
    peak = lane["fma_per_s"] / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
           "ops_per_sample_iteration": lane_ops,
           "peak_source": (f"sf_lane_peaks in this run: FMA microbenchmark {lane['fma_per_s'] / 1e12:.2f} T/s "
                           f"(lane clock {lane['lane_mhz']:.0f} MHz), of measured"),
           "kernel": ("tm_fwd_kernel" if tm else "fused_fwd_kernel") if form == "fused"
           else "plain form (several kernels)",
           "traffic": None, "traffic_unit": "DRAM bytes per launch (ncu)"}
    cap = FWD_TRAFFIC.get((form, tm, precision))
    if cap is not None:
        out["traffic"] = cap[0]
        out["traffic_source"] = cap[1]
    inst = FWD_EXECUTED.get((form, tm, precision))
    if inst is not None and dev is not None:
        # issue slots: 4 schedulers per SM, one warp-instruction each per
        # cycle, at the clock the FMA microbenchmark ran at
        import torch
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        slots = sec * sms * 4 * lane["lane_mhz"] * 1e6
        out["executed"] = {"warp_instructions_per_launch": inst, "issue_frac": inst / slots,
                           "source": "smsp__inst_executed.sum of one ncu capture of this kernel on this workload; "
                                     "issue_frac = that count / (launch time x SMs x 4 x lane clock)"}
    mufu = mufu_per_sample_iter(N, T) * S * K / sec / 1e12
    out["mufu"] = {"achieved": mufu, "peak": lane["mufu_per_s"] / 1e12, "unit": "Tops/s",
                   "frac": mufu / (lane["mufu_per_s"] / 1e12), "ops_per_sample_iteration": mufu_per_sample_iter(N, T)}
    if tm and form == "fused":
        ratio = 0.5 if precision == "fp32" else 1.0
        bf16 = float(peaks.get("bf16_tflops", 0.0)) or 1900.0
        tpeak = bf16 * ratio
        tach = 2.0 * macs * S * K / sec / 1e12
        out["tensor"] = {"achieved": tach, "peak": tpeak, "unit": "TFLOP/s", "frac": tach / tpeak,
                         "flops_per_sample_iteration": 2 * macs,
                         "operands": {"fp32": "tf32", "bf16": "bf16", "fp16": "fp16"}[precision],
                         "peak_source": f"MEASURED_PEAKS.json bf16 burst {bf16:.1f} TFLOP/s x {ratio} (nominal "
                                        "ratio of the operand type), of measured"}
    return out


def workload_spec():
    return si.config_n16_3d()


def workload_name(spec):
    return (f"{spec.dim}D N={spec.n_robots} robots, S={spec.n_samples} samples, T={spec.T}, "
            f"K={spec.K}, Bernstein order {spec.order}, sample init, rho={RHO}, robot radius "
            f"{spec.radius} m, |v|<={spec.v_max}, |a|<={spec.a_max}")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def run_gpu(args):
    import torch
    import paper_2501_19042_gb300 as P
    from paper_2501_19042_gb300.sharding import max_over_ranks

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    P.build()
    spec = workload_spec()
    # the global batch: one scene of the workload per rank (seeds 1..world),
    # split into contiguous sample ranges by shard_batch; each rank projects
    # its own range with no collective on the data path
    from paper_2501_19042_gb300.sharding import shard_batch
    scenes = [si.scene(spec, 1 + q) for q in range(world)]
    host = lambda arrs: torch.tensor(np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in arrs]))
    sh = shard_batch(host([s.xi_bar for s in scenes]), host([s.start for s in scenes]).reshape(-1, spec.dim),
                     host([s.goal for s in scenes]).reshape(-1, spec.dim), [spec.n_robots] * world,
                     [spec.n_samples] * world, spec.dim, rank, world)
    assert sh.n_robots == [spec.n_robots] and sh.n_samples == [spec.n_samples]
    sc = scenes[sh.scenes[0][0]]
    S, K = spec.n_samples, spec.K
    f = P.SafetyFilter(dim=spec.dim, T=spec.T, rho=RHO, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                       max_robots=spec.n_robots, t_final=spec.t_final, precision=args.precision, device=dev.index)
    f.set_tensor_memory("auto" if args.tensor_memory == 2 else bool(args.tensor_memory))
    xb = sh.xi_bar.reshape(sc.xi_bar.shape).to(dev)
    st, gl = sh.start.contiguous().to(dev), sh.goal.contiguous().to(dev)
    stream = torch.cuda.current_stream(dev)
    out = f.project(xb, st, gl, K, form=args.form)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        f.project(xb, st, gl, K, form=args.form, out=out)
    torch.cuda.synchronize()

    # the float32-lane peaks of this GPU, measured now (FMA and rsqrt microbenchmarks)
    lane = P.lane_peaks(dev.index)
    f.project(xb, st, gl, K, form=args.form, out=out)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clk = ClockSampler(dev.index)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    n_launch0 = f.launch_count()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                       # L2 flushed between timed steps, outside the events
        starts[i].record(stream)
        f.project(xb, st, gl, K, form=args.form, out=out)
        stops[i].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    launches = f.launch_count() - n_launch0
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, stops)]
    ms = float(np.mean(step_ms))
    ms = max_over_ranks(ms, device=dev)
    f.sync_status()

    # residual condition of the metric
    med_res = float(out.residual.median())

    # end to end through sf_project_host: pinned host inputs, copies inside the call
    hx = torch.tensor(sc.xi_bar, dtype=torch.float32).contiguous().pin_memory()
    hs = torch.tensor(sc.start, dtype=torch.float32).contiguous().pin_memory()
    hg = torch.tensor(sc.goal, dtype=torch.float32).contiguous().pin_memory()
    hout = f.project_host(hx, hs, hg, K, form=args.form)
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        f.project_host(hx, hs, hg, K, form=args.form, out=hout)
    barrier()
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, device=dev)
    h2d = (hx.numel() + hs.numel() + hg.numel()) * 4
    d2h = (2 * hx.numel() + S) * 4

    if rank == 0:
        tm = args.form == "fused" and f.launch_shape()["tensor_memory"]   # the form that ran
        value = world * S / (ms * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic (seeded swarm generator)", "impl": "gb300", "form": args.form,
            "config": {"workload": workload_name(spec), "global_batch": world * S, "per_gpu_samples": S,
                       "parallelism": f"contiguous sample ranges (shard_batch) on {world} GPU(s)",
                       "l2": "flushed between timed steps by a 256 MiB write outside the events",
                       "tensor_memory": tm,
                       "form_choice": {0: "float32 lanes", 1: "tensor memory",
                                       2: "per robot-count bucket (library default)"}[args.tensor_memory],
                       "state_products": ({"fp32": "tf32", "bf16": "bf16", "fp16": "fp16"}[args.precision]
                                          + " three-term MMAs (tcgen05, TMEM)") if tm else "float32 lanes"},
            "median_final_residual": med_res,
            "roofline": roofline(spec, S, K, ms, tm, args.precision, args.form, lane, dev),
            "e2e": {"value": world * S / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "api": "sf_project_host"},
            "gpu_launches": int(launches),
            "wall_s_timed": wall,
            "clocks": clocks,
        }
        if args.form == "fused" and not args.no_plain_form:
            line["plain_form"] = plain_form_timing(f, xb, st, gl, K, flush, stream, ms, S)
        if not args.no_diff:
            line["differentiation"] = diff_timing(P, dev)
        if not args.no_batching:
            line["batching"] = batching_timing(P, dev)
        if not args.no_precision:
            line["precision"] = precision_timing(P, dev)
        if not args.no_init:
            line["init"] = init_timing(P, dev)
        if not args.no_workspace:
            line["workspace"] = workspace_timing(P, dev)
        if not args.no_sweep:
            line["sweep"] = sweep_timing(P, dev)
        if not args.no_qp:
            line["qp_layer"] = qp_layer_timing(P, dev)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(spec, sc, args.cpu_samples)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def plain_form_timing(f, xb, st, gl, K, flush, stream, fused_ms, S, steps: int = 3):
    """The plain form (states / project / transpose / solve / residual
    kernels, time-domain arrays in HBM) on the bench workload and handle, with
    the same warm-up, L2 flush and event timing as the headline number."""
    import torch
    out = f.project(xb, st, gl, K, form="plain")
    for _ in range(2):
        f.project(xb, st, gl, K, form="plain", out=out)
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        f.project(xb, st, gl, K, form="plain", out=out)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    f.sync_status()
    ms = float(np.mean(ts))
    return {"ms_per_step": ms, "samples_per_s": S / (ms * 1e-3), "chosen_over_plain": ms / fused_ms,
            "median_final_residual": float(out.residual.median()), "steps": steps}


def diff_timing(P, dev):
    """Forward / backward times of the differentiable SF on the
    differentiation workload (N=16 3D, S=512, T=100, K=50, checkpoint every
    10), CUDA events, mean of 5 after one warm-up call, per mode: float32
    (lane products), float32 with the tensor-memory form (tf32 products) and
    the bf16 / fp16 modes (tensor-memory form). The adjoint is float32 in
    every mode; the training forward writes checkpoints and activity masks."""
    import torch
    spec = si.config_diff()
    sc = si.scene(spec, 5)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    xb, st, gl = t(sc.xi_bar), t(sc.start), t(sc.goal)
    g = torch.randn(xb.shape, generator=torch.Generator().manual_seed(0)).to(dev)

    def timed(fn, n=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    modes = {}
    for name, prec, tm in (("fp32", "fp32", False), ("fp32_tensor_memory", "fp32", True), ("bf16", "bf16", True),
                           ("fp16", "fp16", True)):
        f = P.SafetyFilter(dim=3, T=spec.T, rho=RHO, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                           max_robots=spec.n_robots, checkpoint_every=10, device=dev.index, precision=prec)
        f.set_tensor_memory(tm)
        fwd = timed(lambda: f.project(xb, st, gl, spec.K))
        trn = timed(lambda: f.project_train(xb, st, gl, spec.K))
        _, _, ck = f.project_train(xb, st, gl, spec.K)
        bwd = timed(lambda: f.project_backward(xb, st, gl, spec.K, ck, grad_xi=g))
        f.sync_status()
        modes[name] = {"fwd_ms": fwd, "train_fwd_ms": trn, "bwd_ms": bwd, "bwd_over_fwd": bwd / fwd}
    out = {"workload": f"3D N={spec.n_robots}, S={spec.n_samples}, T={spec.T}, K={spec.K}, checkpoint every 10",
           "modes": modes}
    out.update(modes["fp32"])
    return out


def init_timing(P, dev, steps: int = 300, eval_scenes: int = 64):
    """The learned initialisations (Sec. III-C, Eq. NN_loss; Sec. V,
    initialisation efficacy) on the differentiation workload's shape (3D
    N=16, T=100, 8 samples per scene): the 3-layer MLP and the paper's
    PointNet-like network, each trained for `steps` steps of 64 seeded scenes
    through the differentiable SF (K=50, checkpoint every 10), then the
    held-out median final ||r_p|| after K=50 for the sample, zero and learned
    initialisations, and the median projection residual at k = 1, 5, 20, 50."""
    import torch
    from paper_2501_19042_gb300 import init_mlp as im
    spec = si.config_diff(n_samples=8, K=50)
    sf = P.SafetyFilter(dim=3, T=spec.T, rho=RHO, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                        max_robots=spec.n_robots, checkpoint_every=10, device=dev.index)
    out, nets = {}, {}
    for arch in ("mlp", "pointnet"):
        torch.manual_seed(0)
        net = im.make_init_net(arch, spec.n_robots).to(dev)
        t0 = time.perf_counter()
        hist = im.train(sf, net, spec, K=spec.K, n_train_scenes=steps * 64, scenes_per_step=64, max_steps=steps)
        torch.cuda.synchronize()
        ev = im.evaluate(sf, net, spec, spec.K, n_scenes=eval_scenes)
        out[arch] = {"train_steps": len(hist), "train_scenes": len(hist) * 64,
                     "train_seconds": time.perf_counter() - t0, "loss_first": hist[0], "loss_last": hist[-1],
                     "heldout_median_rp_K50": ev["learned_init"]["median"],
                     "better_than_sample_init_frac": ev["learned_better_frac"]}
        out["sample_init_median_rp_K50"] = ev["sample_init"]["median"]
        out["zero_init_median_rp_K50"] = ev["zero_init"]["median"]
        nets[arch] = net
    out["residual_curves_median"] = im.residual_curves(sf, nets, spec, spec.K, n_scenes=eval_scenes, at=(1, 5, 20, 50))
    out["workload"] = (f"3D N={spec.n_robots}, T={spec.T}, 8 samples per scene, K={spec.K}; held-out "
                       f"{eval_scenes} scenes ({eval_scenes * 8} samples)")
    return out


def precision_timing(P, dev, n_check: int = 64, steps: int = 3):
    """The precision workload: N=32 robots 3D (496 pairs), S=2048, T=120,
    K=200, sample init. Per precision mode of the fused forward: time per
    call (CUDA events, mean of `steps` after one warm-up), median final
    ||r_p|| over all samples, and against the FP64 oracle on samples
    0..n_check-1: relative L2 of xi^K per sample and |final ||r_p|| difference|."""
    import torch
    import oracle
    spec = si.config_n32_3d()
    sc = si.scene(spec, 3)
    oracle.build()
    pb = oracle.Problem(dim=3, n_robots=spec.n_robots, T=spec.T, order=spec.order, t_final=spec.t_final,
                        rho=RHO, coll_a=spec.coll, coll_b=spec.coll, v_max=spec.v_max, a_max=spec.a_max)
    t_or = time.perf_counter()
    ref = oracle.run_batch(pb, sc.start, sc.goal, sc.xi_bar[:n_check], K=spec.K, n_threads=os.cpu_count() or 1)
    t_or = time.perf_counter() - t_or
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    xb, st, gl = t(sc.xi_bar), t(sc.start), t(sc.goal)
    xr = np.asarray(ref["xi"]).reshape(n_check, -1)
    modes = {}
    for name, prec, tm in (("fp32", "fp32", False), ("fp32_tensor_memory", "fp32", True), ("bf16", "bf16", True),
                           ("fp16", "fp16", True)):
        try:
            f = P.SafetyFilter(dim=3, T=spec.T, rho=RHO, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                               max_robots=spec.n_robots, t_final=spec.t_final, precision=prec, device=dev.index)
            f.set_tensor_memory(tm)
            out = f.project(xb, st, gl, spec.K)
        except Exception as e:  # a mode this library does not build
            modes[name] = {"unavailable": str(e).splitlines()[0][:160]}
            continue
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            f.project(xb, st, gl, spec.K, out=out)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        f.sync_status()
        xi = out.xi[:n_check].double().cpu().numpy().reshape(n_check, -1)
        err = np.linalg.norm(xi - xr, axis=1) / np.linalg.norm(xr, axis=1)
        lam = out.lam[:n_check].double().cpu().numpy().reshape(n_check, -1)
        lerr = np.linalg.norm(lam - np.asarray(ref["lam"]).reshape(n_check, -1), axis=1) / np.linalg.norm(xr, axis=1)
        dres = np.abs(out.residual[:n_check].double().cpu().numpy() - np.asarray(ref["rp_final"]))
        modes[name] = {"ms": ms, "samples_per_s": spec.n_samples / (ms * 1e-3),
                       "median_final_residual": float(out.residual.median()),
                       "xi_rel_l2_median": float(np.median(err)), "xi_rel_l2_max": float(err.max()),
                       "lambda_err_max": float(lerr.max()),
                       "resid_absdiff_max": float(dres.max()), "launch_shape": f.launch_shape()}
    return {"workload": f"3D N={spec.n_robots}, S={spec.n_samples}, T={spec.T}, K={spec.K}, sample init, "
                        f"rho={RHO}; errors vs the FP64 oracle on samples 0..{n_check - 1}",
            "oracle_seconds": t_or, "modes": modes}


def workspace_timing(P, dev, n_check: int = 16, steps: int = 3):
    """The bench workload (N=16 3D, S=1024, T=100, K=200, seed 1) with the
    workspace block on: a spheroid centred at the origin with b_w = a_w / 2
    and a_w 8 % larger than needed to hold every start and goal. Time per call
    against the same call without the block, the median final ||r_p||, the
    share of (sample, robot, t) positions outside the workspace in the
    input, and errors against the FP64 oracle on samples 0..n_check-1."""
    import torch
    import oracle
    spec = workload_spec()
    sc = si.scene(spec, 1)
    pts = np.concatenate([sc.start, sc.goal])
    a_w = 1.08 * float(np.sqrt(pts[:, 0] ** 2 + pts[:, 1] ** 2 + (2.0 * pts[:, 2]) ** 2).max())
    ws = ((0.0, 0.0, 0.0), a_w, a_w / 2)
    Pm = oracle.basis(spec.order, spec.T, spec.t_final)[0]
    pos = np.einsum("tk,sdnk->sntd", Pm, sc.xi_bar)
    outside = float(((pos[..., 0] ** 2 + pos[..., 1] ** 2) / a_w ** 2 + pos[..., 2] ** 2 / (a_w / 2) ** 2 > 1).mean())
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    xb, st, gl = t(sc.xi_bar), t(sc.start), t(sc.goal)
    res = {}
    for name, w in (("without", None), ("with", ws)):
        f = P.SafetyFilter(dim=3, T=spec.T, rho=RHO, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                           max_robots=spec.n_robots, t_final=spec.t_final, workspace=w, device=dev.index)
        out = f.project(xb, st, gl, spec.K)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            f.project(xb, st, gl, spec.K, out=out)
        b.record()
        torch.cuda.synchronize()
        res[name] = (a.elapsed_time(b) / steps, out)
    oracle.build()
    pb = oracle.Problem(dim=3, n_robots=spec.n_robots, T=spec.T, order=spec.order, t_final=spec.t_final,
                        rho=RHO, coll_a=spec.coll, coll_b=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                        use_workspace=True, ws_center=ws[0], ws_a=ws[1], ws_b=ws[2])
    ref = oracle.run_batch(pb, sc.start, sc.goal, sc.xi_bar[:n_check], K=spec.K, n_threads=os.cpu_count() or 1)
    ms, out = res["with"]
    xi = out.xi[:n_check].double().cpu().numpy().reshape(n_check, -1)
    xr = np.asarray(ref["xi"]).reshape(n_check, -1)
    err = np.linalg.norm(xi - xr, axis=1) / np.linalg.norm(xr, axis=1)
    dres = np.abs(out.residual[:n_check].double().cpu().numpy() - np.asarray(ref["rp_final"]))
    return {"workload": f"3D N={spec.n_robots}, S={spec.n_samples}, T={spec.T}, K={spec.K}, workspace spheroid "
                        f"a_w={a_w:.3f} m, b_w={a_w / 2:.3f} m at the origin",
            "input_positions_outside": outside, "ms": ms, "samples_per_s": spec.n_samples / (ms * 1e-3),
            "ms_without_workspace": res["without"][0], "median_final_residual": float(out.residual.median()),
            "xi_rel_l2_max": float(err.max()), "resid_absdiff_max": float(dres.max()),
            "oracle_samples": n_check}


def sweep_timing(P, dev, reps: int = 3):
    """SF-only computation time in the layout of the paper's computation-time
    figure: per swarm size N in {4, 8, 16} (3D, the bench's box scene, T=100),
    time per sf_project call against the batch size (10..200 samples, K=200)
    and against the number of iterations (K=10..400, 10 samples). CUDA
    events, mean of `reps` calls after one warm-up call."""
    import torch
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    out = {"workload": "3D, T=100, sample init, rho=0.1, box 8x8x4 m; per N: ms per call vs batch "
                       "(K=200) and vs K (batch 10)", "by_N": {}}
    for N in (4, 8, 16):
        spec = si.config_n16_3d(n_robots=N, n_samples=200)
        sc = si.scene(spec, 100 + N)
        f = P.SafetyFilter(dim=3, T=spec.T, rho=RHO, coll_a=spec.coll, v_max=spec.v_max, a_max=spec.a_max,
                           max_robots=N, t_final=spec.t_final, device=dev.index)
        st, gl = t(sc.start), t(sc.goal)

        def timed(batch, K):
            xb = t(sc.xi_bar[:batch])
            r = f.project(xb, st, gl, K)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                f.project(xb, st, gl, K, out=r)
            b.record()
            torch.cuda.synchronize()
            return round(a.elapsed_time(b) / reps, 4)

        out["by_N"][str(N)] = {"ms_vs_batch_K200": {str(bs): timed(bs, 200) for bs in (10, 25, 50, 100, 200)},
                               "ms_vs_K_batch10": {str(K): timed(10, K) for K in (10, 50, 100, 200, 400)}}
    return out


def qp_layer_timing(P, dev, n_samples: int = 65536, reps: int = 20):
    """The decoders' QP layer (sf_eq_project) on a batch of decoder outputs:
    N=16 robots 3D, 65,536 samples (3.1M coefficient rows of 11 floats, 276
    MB read + written per call). HBM-bound: achieved = (44 B read + 44 B
    written) per row / CUDA-event time per call, against the measured copy
    bandwidth; the input is larger than L2, so no flush is needed."""
    import torch
    spec = workload_spec()
    sc = si.scene(si.config_n16_3d(n_samples=8), 1)     # the scene's starts and goals
    f = P.SafetyFilter(dim=3, T=spec.T, rho=RHO, coll_a=spec.coll, max_robots=spec.n_robots, device=dev.index)
    g = torch.Generator(device=dev).manual_seed(0)
    xp = torch.randn((n_samples, 3, spec.n_robots, 11), generator=g, device=dev)
    st = torch.as_tensor(sc.start, dtype=torch.float32, device=dev)
    gl = torch.as_tensor(sc.goal, dtype=torch.float32, device=dev)
    out = f.eq_project(xp, st, gl)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        f.eq_project(xp, st, gl, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    gin, _ = f.eq_project_backward(out, st, gl)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        f.eq_project_backward(out, st, gl)
    b.record()
    torch.cuda.synchronize()
    ms_b = a.elapsed_time(b) / reps
    rows = n_samples * 3 * spec.n_robots
    gbs = rows * 88 / (ms * 1e-3) / 1e9
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    return {"workload": f"3D N={spec.n_robots}, {n_samples} samples of decoder outputs ({rows} rows of 11)",
            "ms": ms, "samples_per_s": n_samples / (ms * 1e-3), "backward_ms": ms_b,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "algorithmic_bytes_per_row": 88, "kernel": "eq_kernel"}}


def batching_timing(P, dev):
    """The ragged batching workload: 64 scenes, N ~ U{8..32}, S ~ U{128..512},
    K=150, 3D. Aggregate: one captured graph (all robot-count groups, autotuned
    shapes), CUDA events, mean of 3 after a warm-up. Per scene: each scene
    alone through sf_project."""
    import torch
    scenes = si.ragged_batch(2)
    K = 150
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    xb = t(np.concatenate([s.xi_bar.reshape(-1) for s in scenes]))
    st = t(np.concatenate([s.start for s in scenes]))
    gl = t(np.concatenate([s.goal for s in scenes]))
    nr = [s.spec.n_robots for s in scenes]
    ns = [s.spec.n_samples for s in scenes]
    f = P.SafetyFilter(dim=3, T=100, rho=RHO, coll_a=scenes[0].spec.coll, max_robots=32, device=dev.index)
    f.autotune(xb, st, gl, K_probe=5, n_candidates=6, n_robots=nr, n_samples=ns)
    g = f.capture(xb, st, gl, K, n_robots=nr, n_samples=ns)
    g.launch()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = f.launch_count()
    a.record()
    for _ in range(3):
        g.launch()
    b.record()
    torch.cuda.synchronize()
    agg_ms = a.elapsed_time(b) / 3
    per = []
    for s in scenes:
        xs, ss, gs = t(s.xi_bar), t(s.start), t(s.goal)
        out = f.project(xs, ss, gs, K)
        torch.cuda.synchronize()
        a.record()
        f.project(xs, ss, gs, K, out=out)
        b.record()
        torch.cuda.synchronize()
        per.append({"N": s.spec.n_robots, "S": s.spec.n_samples,
                    "samples_per_s": s.spec.n_samples / (a.elapsed_time(b) * 1e-3)})
    g.close()
    tot = sum(ns)
    return {"workload": "64 scenes, N ~ U{8..32}, S ~ U{128..512}, T=100, K=150, 3D, one captured graph",
            "total_samples": tot, "aggregate_ms": agg_ms, "aggregate_samples_per_s": tot / (agg_ms * 1e-3),
            "per_scene_alone_sum_ms": float(sum(p["S"] / p["samples_per_s"] * 1e3 for p in per)),
            "per_scene": per}


def cpu_baseline(spec, sc, n_samples):
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    pb = oracle.Problem(dim=spec.dim, n_robots=spec.n_robots, T=spec.T, order=spec.order, t_final=spec.t_final,
                        rho=RHO, coll_a=spec.coll, coll_b=spec.coll, v_max=spec.v_max, a_max=spec.a_max)
    xb = sc.xi_bar[:n_samples]
    t0 = time.perf_counter()
    oracle.run_batch(pb, sc.start, sc.goal, xb, K=spec.K, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n_samples / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n_samples} of the {spec.n_samples} samples, K={spec.K}, FP64 C oracle, "
                      f"{dt:.1f} s wall on {cores} threads"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the machine's host cores."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    spec = workload_spec()
    sc = si.scene(spec, 1)
    cores = os.cpu_count() or 1
    n = args.cpu_samples
    pb = oracle.Problem(dim=spec.dim, n_robots=spec.n_robots, T=spec.T, order=spec.order, t_final=spec.t_final,
                        rho=RHO, coll_a=spec.coll, coll_b=spec.coll, v_max=spec.v_max, a_max=spec.a_max)
    for _ in range(args.warmup):
        oracle.run_batch(pb, sc.start, sc.goal, sc.xi_bar[:cores], K=5, n_threads=cores)
    times = []
    for i in range(args.steps):
        xb = sc.xi_bar[(i * n) % spec.n_samples:][:n]
        t0 = time.perf_counter()
        oracle.run_batch(pb, sc.start, sc.goal, xb, K=spec.K, n_threads=cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = n / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded swarm generator)", "impl": "reference",
        "config": {"workload": workload_name(spec), "global_batch": n,
                   "parallelism": f"{cores} host threads", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} samples of the {spec.n_samples}-sample workload per step, K={spec.K}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--form", default="fused", choices=["fused", "plain"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="contraction precision of the timed forward (the metric is quoted in fp32)")
    ap.add_argument("--tensor-memory", type=int, default=2, choices=[0, 1, 2],
                    help="1: coefficient-to-state products on tcgen05 tensor cores through TMEM; 0: on the "
                         "float32 lanes; 2 (default): the library's choice per robot-count bucket")
    ap.add_argument("--cpu-samples", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-diff", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-init", action="store_true")
    ap.add_argument("--no-workspace", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-qp", action="store_true")
    ap.add_argument("--no-plain-form", action="store_true",
                    help="skip the plain-form timing on the bench workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
