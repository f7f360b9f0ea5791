"""The multi-rank (one process per GPU) path on CPU with the gloo backend,
world size 2: the sample sharding covers every sample exactly once with the
right coefficients and boundary rows, the timing reduction gives every rank
the slowest rank's time, and the reference arm of the bench prints one line
from rank 0 only under torchrun."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import swarm_inputs as si
from paper_2501_19042_gb300.sharding import max_over_ranks, sample_ranges, shard_batch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    scenes = si.ragged_batch(11, n_scenes=5, s_lo=3, s_hi=9, K=5)
    xb = np.concatenate([s.xi_bar.reshape(-1) for s in scenes]).astype(np.float32)
    st = np.concatenate([s.start for s in scenes]).astype(np.float32)
    gl = np.concatenate([s.goal for s in scenes]).astype(np.float32)
    return scenes, xb, st, gl


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scenes, xb, st, gl = _batch()
    nr = [s.spec.n_robots for s in scenes]
    ns = [s.spec.n_samples for s in scenes]
    sh = shard_batch(torch.from_numpy(xb), torch.from_numpy(st), torch.from_numpy(gl), nr, ns, 3, rank, world)
    owned = []
    for (q, lo, hi), g0 in zip(sh.scenes, sh.sample_offset):
        owned += [(q, k) for k in range(lo, hi)]
    # the shard's coefficients are the owned samples' rows of the full batch
    c = 0
    ok = True
    for (q, lo, hi) in sh.scenes:
        s = scenes[q]
        per = 3 * s.spec.n_robots * 11
        ok &= np.array_equal(sh.xi_bar[c: c + (hi - lo) * per].numpy(),
                             s.xi_bar[lo:hi].reshape(-1).astype(np.float32))
        c += (hi - lo) * per
    ok &= c == sh.xi_bar.numel()
    r = 0
    for (q, _, _), N in zip(sh.scenes, sh.n_robots):
        ok &= np.array_equal(sh.start[r: r + N].numpy(), scenes[q].start.astype(np.float32))
        r += N
    gathered = [None] * world
    dist.all_gather_object(gathered, {"owned": owned, "ok": bool(ok)})
    slowest = max_over_ranks(1.5 + rank)
    if rank == 0:
        with open(os.path.join(out_dir, "result.json"), "w") as f:
            json.dump({"gathered": gathered, "slowest": slowest}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_sample_ranges_partition():
    ns = [5, 0, 7, 1, 12]
    for world in (1, 2, 3, 7, 30):
        seen = []
        for rank in range(world):
            rr = sample_ranges(ns, rank, world)
            assert len(rr) == len(ns)
            for q, (lo, hi) in enumerate(rr):
                assert 0 <= lo <= hi <= ns[q]
                seen += [(q, k) for k in range(lo, hi)]
        assert sorted(seen) == [(q, k) for q, s in enumerate(ns) for k in range(s)]
        sizes = [sum(hi - lo for lo, hi in sample_ranges(ns, r, world)) for r in range(world)]
        assert max(sizes) - min(sizes) <= 1


def test_two_ranks_gloo(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = json.load(open(tmp_path / "result.json"))
    scenes, _, _, _ = _batch()
    all_ids = sorted((q, k) for q, s in enumerate(scenes) for k in range(s.spec.n_samples))
    owned = [tuple(x) for g in res["gathered"] for x in g["owned"]]
    assert all(g["ok"] for g in res["gathered"])
    assert sorted(owned) == all_ids and len(owned) == len(set(owned))
    assert res["slowest"] == 2.5


def test_reference_arm_under_torchrun():
    """bench.py --impl reference with two ranks: rank 0 prints one JSON line,
    rank 1 exits 0 without work."""
    pytest.importorskip("torch.distributed.run")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--cpu-samples", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0
